#!/usr/bin/env python3
"""Benchmark of the DQO-MAP GPU optimisation hot path on GB300.

One step = one keyframe iteration of the paper's GPU-side optimisation (Sec. III-D):
  forward render with the fused colour / depth / instance losses (Eq. 7-10, 15),
  the full backward to the Gaussian parameters, and the bbox loss + gradient of the
  keyframe's 30 dual quadrics over their views (Eq. 12),
on the indoor-keyframe workload: 300k Gaussians on 30 ellipsoidal objects plus room
walls, a 1200x680 RGB-D keyframe, seeded synthetic data.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` = keyframe iterations per second over all ranks (device
time, CUDA events, L2 flushed between steps); `e2e` = the same through the C ABI with
the step's inputs copied from pinned host memory and its loss and gradients copied
back inside the timed region; `roofline` = the dominant kernel against the FP32 pipe
peak; `cpu_baseline` / `--impl reference` = the FP64 CPU oracle on a bounded sample.
Multi-GPU (torchrun): every rank runs its own keyframe replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd keyframe iters/s (300k Gaussians,1200×680) & quadric fits/s vs plain"
UNIT = "iters/s"
SEED = 1002
NUM_OBJECTS = 31                 # ids 0 (room) .. 30
FP32_LANES = 128                 # FP32 lanes per SM (context figure beside the measured peak)
# Algorithmic FP32 flops per (pixel, Gaussian) evaluation (FMA = 2 flops, the exponential
# counted on its own pipe): forward ~20 (offset, quadratic form, alpha, transmittance,
# weight, colour / depth / alpha accumulation), backward ~50 (the forward's evaluation
# again, the upstream dot product, dL/dalpha, the ten per-Gaussian partials and their
# sums).  The kernels' own instruction count is higher (25 + 55: instance channel, id
# bookkeeping); the roofline uses the algorithmic count.
FLOPS_PER_EVAL = {"blend_fwd": 20, "blend_bwd": 50, "blend_step": 70}
FLOPS_PER_EVAL_KERNEL = {"blend_fwd": 25, "blend_bwd": 55, "blend_step": 80}
# Quadric step: ~700 FP32 flops per (quadric, view) pair per forward + backward (Q* build
# share, C* = P Q* P^T, tangent-line box, IoU and the adjoint back through them).
QUADRIC_FLOPS_PER_PAIR = 700
FIT_ITERS = 100
KERNEL_SRC = {"blend_fwd": "k_blend.cu", "blend_bwd": "k_blend.cu", "blend_step": "k_blend.cu"}
# Learned proposal: algorithmic flops per sample of one training step (FMA = 2): forward
# 2 (128*128 + 128*128 + 9*128); backward dH2 and dW3 2 (9*128) each, dH1, dW2, dW1
# 2 (128*128) each.
MLP_FLOPS_PER_SAMPLE = 2 * (128 * 128 + 128 * 128 + 9 * 128) + 2 * (2 * 9 * 128 + 3 * 128 * 128)
# Bytes each HBM-bound phase of the step moves (design bytes, counted from the kernels):
# projection: reads means 12, log-scales 12, quaternion 16, logit 4, rgb 12, id 4, flags 1;
#   writes 3 x float4 48, rect 8, tiles 4, depth key 4, value 4, id 4        -> 133 B/Gaussian
# depth sort: one histogram kernel reads the keys 4; 4 radix passes read key+value 8 and
#   write 8                                                                  -> 68 B/Gaussian
# binning: the emission (which also scans the pair counts in depth order) reads order 4 and
#   rect 8 per Gaussian and writes 4 per pair; the pair sort covers the tile bits only:
#   histogram read 4 + 2 passes of (read 4, write 4); ranges read key 4 and the order 4,
#   write the list 4 per pair                                                -> 12 B/Gaussian + 36 B/pair
#   (the algorithmic minimum: write each pair's value once and read it once in the blend,
#   8 B/pair, plus 16 B/Gaussian)
# projection adjoint: reads the 10 inputs 61, tiles 4, moment record 48; read-modify-write of
#   the 14 gradient floats 112                                              -> 225 B/Gaussian
REF_BUDGET_S = 240.0   # the reference arm's K + W steps take about this long
HBM_BYTES = {"project": (133, 0), "depth_sort": (68, 0), "binning": (12, 36), "project_bwd": (225, 0)}
SORT_MIN_BYTES = (16, 8)
MLP_TRAIN_SAMPLES = 1 << 20
MLP_EPOCHS = 40
MLP_BATCH = 4096


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--tile", default="16x16")
    p.add_argument("--batch", type=int, default=256)
    p.add_argument("--no-learned", action="store_true", help="skip the learned-proposal section")
    p.add_argument("--no-batched", action="store_true", help="skip the batched-keyframes section")
    p.add_argument("--no-adjoint-1m", action="store_true", help="skip the 1M-Gaussian adjoint section")
    p.add_argument("--no-tune", action="store_true",
                   help="fixed step configuration (--tile, per-keyframe blend schedule) instead of the autotuner; "
                        "for profiling, where the tuner's timings are distorted")
    return p.parse_args()


# Fallback denominators when no measured peaks file is present (one earlier measurement
# on a GB300: STREAM-style copy, cuBLAS bf16 burst and sustained).
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def measured_peaks() -> tuple[dict, str]:
    """(peaks, basis): the measured peaks file, else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


def cpu_model() -> str:
    """The host CPU's model name (x86 'model name', or the Arm implementer/part fields)."""
    try:
        txt = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model name", "cpu model"):
        for ln in txt.splitlines():
            if ln.split(":")[0].strip() == key:
                return ln.split(":", 1)[1].strip()
    fields = {}
    for ln in txt.splitlines():
        if ":" in ln:
            k, v = ln.split(":", 1)
            fields.setdefault(k.strip(), v.strip())
    if "CPU part" in fields:
        return f"Arm implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    return "unknown"


def alu_peaks(dqo, dev, stream, smi_id) -> dict:
    """Measured FP32 FMA (TFLOP/s) and ex2 (T exponentials/s) throughput of this GPU: the
    library's probe kernels, each launch filling every SM for about 5 ms, best of 5 timed
    launches (burst, like the blend kernels inside a sub-millisecond step), CUDA events on
    the launching stream, SM clocks sampled meanwhile."""
    import torch
    sink = torch.zeros(1, device=dev)
    out = {}
    clocks = ClockSampler(smi_id)
    clocks.start()
    for kind, name in ((dqo.ALU_FMA, "fp32_fma_tflops"), (dqo.ALU_EX2, "ex2_tops")):
        iters = 64
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):                   # size the launch to about 5 ms
            e0.record(stream)
            dqo.dqo_alu_probe(kind, iters, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            iters = max(1, int(iters * 5.0 / max(e0.elapsed_time(e1), 1e-3)))
        best = 0.0
        for _ in range(5):
            e0.record(stream)
            ops = dqo.dqo_alu_probe(kind, iters, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            best = max(best, ops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[name] = best
    out["clocks"] = clocks.stop()
    return out


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.uuid = device_uuid
        self.proc = None
        self.lines = []

    def start(self):
        sel = [f"--id={self.uuid}"] if self.uuid else []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- workload

def make_workload():
    from paper_2503_02223_gb300 import synth
    kf = synth.indoor_keyframe(SEED)
    targets = synth.raycast_targets(kf)
    return kf, targets


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values of x (the job lasts as long as its slowest rank);
    x itself on one rank.  device: where the process group's backend reduces (cuda for
    NCCL, cpu for gloo)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, total_ms: float) -> float:
    """Whole-job units per second: every rank runs `steps` steps of one unit (weak
    scaling), the job taking total_ms (the slowest rank's time)."""
    return world * steps / (total_ms / 1e3)


def oracle_full_parallel(kf, targets, threads: int, bands=None) -> tuple[float, int]:
    """FP64 oracle forward + backward of the whole image (or of the given (first row, rows)
    bands) with its rows split into bands of whole tile rows run concurrently on `threads`
    host threads (the oracle's calls release the interpreter lock; each band projects all
    Gaussians).  Returns (seconds, bands)."""
    import numpy as np

    import oracle
    cam = kf["camera"]
    H = cam["height"]
    rows = max(16, -(-H // threads) // 16 * 16 + (16 if (-(-H // threads)) % 16 else 0))
    st = oracle.settings(num_objects=NUM_OBJECTS)
    oracle.build()
    if bands is None:
        bands = [(r0, min(rows, H - r0)) for r0 in range(0, H, rows)]

    def run(band):
        r0, nr = band
        cam2 = dict(cam, height=nr, cy=cam["cy"] - r0)
        t2 = {k: np.ascontiguousarray(v[r0:r0 + nr]) for k, v in targets.items()}
        oracle.render(kf["gaussians"], cam2, st, t2)
        oracle.render_backward(kf["gaussians"], cam2, st, t2)

    t0 = time.perf_counter()
    ths = [threading.Thread(target=run, args=(b,)) for b in bands]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return time.perf_counter() - t0, len(bands)


def oracle_fits(fq, threads: int, nfits: int | None = None) -> tuple[float, int, int]:
    """FP64 oracle plain fits (Eq. 1 init + FIT_ITERS Adam steps) of the first nfits
    quadrics of the batch, split into `threads` contiguous chunks run concurrently (the
    oracle's calls release the interpreter lock).  Returns (seconds, fits, threads used)."""
    import numpy as np

    import oracle
    oracle.build()
    q_ptr = fq["q_ptr"]
    nq = q_ptr.shape[0] - 1 if nfits is None else min(nfits, q_ptr.shape[0] - 1)
    edges = np.linspace(0, nq, min(threads, nq) + 1).astype(int)
    chunks = [(a, b) for a, b in zip(edges[:-1], edges[1:]) if b > a]

    def run(ab):
        a, b = ab
        p0, p1 = int(q_ptr[a]), int(q_ptr[b])
        oracle.quadric_fit(fq["P"], q_ptr[a:b + 1] - p0, fq["pair_v"][p0:p1], fq["obs_bbox"][p0:p1], iters=FIT_ITERS)

    t0 = time.perf_counter()
    ths = [threading.Thread(target=run, args=(c,)) for c in chunks]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return time.perf_counter() - t0, nq, len(chunks)


def traffic_for(kernel: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it matches the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2503_02223_gb300", "csrc", KERNEL_SRC.get(kernel, ""))
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return rec.get("bytes_per_launch") if rec.get("src_sha") == h else None


# ----------------------------------------------------------------------------- arms

def image_slices(H: int, h: int, cores: int) -> list:
    """The image's rows as bands of h rows (the last one shorter), grouped `cores` bands to
    a slice: a slice is one reference step (its bands run concurrently)."""
    bands = [(r0, min(h, H - r0)) for r0 in range(0, H, h)]
    return [bands[i:i + cores] for i in range(0, len(bands), cores)]


def reference_band_rows(t1: float, t16: float, steps: int, warmup: int, budget_s: float) -> int:
    """The largest band height of 16, 8, 4, 2 whose step time, interpolated between the
    measured 1-row (t1) and 16-row (t16) steps, keeps steps + warmup steps within budget_s
    seconds; 1 when none does."""
    per_step = budget_s / max(1, steps + warmup)
    for cand in (16, 8, 4, 2):
        if t1 + (t16 - t1) * (cand - 1) / 15.0 <= per_step:
            return cand
    return 1


def run_reference(args, rank, world):
    """The FP64 CPU oracle on this host's cores (the reference arm of this workload): the
    whole keyframe per step, rows split into bands run concurrently on every core."""
    if rank != 0:
        return
    kf, targets = make_workload()
    H = kf["camera"]["height"]
    cores = os.cpu_count() or 1
    # A step is one slice of the image: `cores` bands of h rows each, run concurrently;
    # consecutive steps take consecutive slices.  Every band projects all Gaussians, so a
    # band's time is a fixed part plus a part per row: the first two warm-up steps measure
    # bands of 1 and 16 rows, and h (16, 8, 4, 2 or 1) is the largest that keeps the
    # K + W steps near REF_BUDGET_S seconds.
    t1, _ = oracle_full_parallel(kf, targets, cores, image_slices(H, 1, cores)[0])
    t16, _ = oracle_full_parallel(kf, targets, cores, image_slices(H, 16, cores)[0])
    h = reference_band_rows(t1, t16, args.steps, args.warmup, REF_BUDGET_S)
    slices = image_slices(H, h, cores)
    for w in range(max(0, args.warmup - 2)):
        oracle_full_parallel(kf, targets, cores, slices[w % len(slices)])
    times, rows_done = [], 0
    for k in range(args.steps):
        sl = slices[k % len(slices)]
        t, _ = oracle_full_parallel(kf, targets, cores, sl)
        times.append(t)
        rows_done += sum(nr for _, nr in sl)
    total = sum(times)
    val = (rows_done / H) / total if total > 0 else 0.0   # whole keyframes (forward + backward) per second
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": max(args.warmup, 2), "ms_per_step": 1e3 * total / max(1, len(times)),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(kf, None, args),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": min(cores, len(slices[0])), "kind": "oracle",
                             "sample": f"each step one slice of the {H}-row image: {len(slices[0])} bands of {h} "
                                       f"rows run concurrently (forward + backward, FP64, each band projecting all "
                                       f"300k Gaussians), slices in turn; value = image rows done / {H} per second "
                                       f"(the first 2 warm-up steps time 1- and 16-row bands to pick the band "
                                       f"height)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tile_evals(nc, W: int, H: int, tw: int, th: int) -> int:
    """E_tile: per tile, its pixel count times the longest walk of its pixels (the list
    positions the tile's CTA goes through until its last pixel stops), summed over tiles."""
    import torch
    ntx, nty = (W + tw - 1) // tw, (H + th - 1) // th
    img = torch.zeros(nty * th, ntx * tw, dtype=torch.int64, device=nc.device)
    img[:H, :W] = nc.view(H, W).to(torch.int64)
    per_tile = img.view(nty, th, ntx, tw).amax(dim=(1, 3))
    return int(per_tile.sum().item()) * tw * th


def workload_config(kf, m_pairs, args):
    cam = kf["camera"]
    return {"workload": "indoor keyframe: 300k Gaussians (30 ellipsoidal objects + room walls), "
                        "1200x680 RGB-D keyframe, 30 dual quadrics with up to 8 views",
            "gaussians": int(kf["gaussians"]["means"].shape[0]), "width": cam["width"], "height": cam["height"],
            "quadrics": int(kf["quadrics"]["params"].shape[0]),
            "quadric_pairs": int(kf["quadrics"]["pair_v"].shape[0]),
            "tile_gaussian_pairs": m_pairs, "tile": args.tile, "batch": args.batch,
            "l2": "flushed between steps (256 MiB write outside the timed events)",
            "parallelism": f"replicas x{args.gpus}"}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2503_02223_gb300 import dqo
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dqo.load(build_if_missing=True)
    kf, targets = make_workload()
    cam = kf["camera"]
    W, H = cam["width"], cam["height"]
    tw, th = (int(x) for x in args.tile.split("x"))
    ctx = dqo.Context(local_rank)
    # gradients overwritten by the adjoint (no separate clearing of the buffers per step)
    st = dqo.settings(tile_w=tw, tile_h=th, batch=args.batch, grads_zero=1)
    g = dqo.to_device(kf["gaussians"], dev)
    t = dqo.to_device(targets, dev)
    q = dqo.to_device({k: kf["quadrics"][k] for k in ("params", "P", "q_ptr", "pair_v", "obs_bbox")}, dev)
    n = g["means"].shape[0]
    nq = q["params"].shape[0]
    out = dqo.alloc_outputs(W, H, dev)
    grads = dqo.alloc_grads(n, dev)
    qloss = torch.zeros(nq, device=dev)
    qgrad = torch.zeros(nq, 9, device=dev)
    gs, cs, ts = dqo.gaussians(g, NUM_OBJECTS), dqo.camera(cam), dqo.targets(t)
    outs, gg = dqo.render_out(out), dqo.gaussian_grads(grads)
    stream = torch.cuda.current_stream()

    def step():
        dqo.dqo_render_forward(ctx, st, gs, cs, ts, outs, stream)
        dqo.dqo_render_backward(ctx, st, gs, cs, ts, None, gg, stream)
        dqo.dqo_quadric_bbox_loss(ctx, q["params"], q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"], qloss, qgrad,
                                  stream)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    m_pairs, n_vis, n_tiles = dqo.dqo_get_counts(ctx)
    nc = torch.empty(H * W, dtype=torch.int32, device=dev)
    dqo.dqo_get_buffer(ctx, dqo.DQO_BUF_N_CONTRIB, nc)
    torch.cuda.synchronize()
    evals = int(nc.to(torch.int64).sum().item())
    evals_tile = tile_evals(nc, W, H, tw, th)
    uuid = getattr(torch.cuda.get_device_properties(local_rank), "uuid", None)
    smi_id = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else \
        (str(uuid) if uuid is not None else None)

    # ---- the step as deployed: the batched path with this one keyframe and the quadric
    # loss, captured once in a CUDA graph (no host synchronisation, no launch gaps)
    bctx = dqo.Context(local_rank)
    kfb = dqo.keyframe(g, NUM_OBJECTS, cam, t, out, grads)

    bst = dqo.settings(tile_w=tw, tile_h=th, batch=args.batch, grads_zero=1)
    if args.no_tune:
        cps, sched, tune_ms = 0, dqo.SCHEDULE_PER_KEYFRAME, []
    else:
        cps, sched, tune_ms = dqo.dqo_batch_tune(bctx, bst, [kfb], None, reps=5)

    # the quadric loss does not depend on the keyframe: a concurrent branch of the graph
    qside = torch.cuda.Stream(dev)

    def graph_body():
        main = torch.cuda.current_stream()
        qside.wait_stream(main)
        with torch.cuda.stream(qside):
            dqo.dqo_quadric_bbox_loss(bctx, q["params"], q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"], qloss,
                                      qgrad)
        dqo.dqo_batch_step(bctx, bst, [kfb], None, cps, sched)
        main.wait_stream(qside)

    dqo.dqo_batch_step(bctx, bst, [kfb], None, cps, sched, stream)      # sizing call
    torch.cuda.synchronize()
    if (bst.tile_w, bst.tile_h) != (tw, th):
        # evaluations walked depend on the tile lists: count them with the tuned tiles
        ectx = dqo.Context(local_rank)
        dqo.dqo_render_forward(ectx, bst, gs, cs, ts, outs, stream)
        dqo.dqo_get_buffer(ectx, dqo.DQO_BUF_N_CONTRIB, nc)
        torch.cuda.synchronize()
        evals = int(nc.to(torch.int64).sum().item())
        evals_tile = tile_evals(nc, W, H, bst.tile_w, bst.tile_h)
        ectx.close()
    dqo.dqo_set_timing(bctx, True)
    graph = torch.cuda.CUDAGraph()
    cap_stream = torch.cuda.Stream(dev)
    cap_stream.wait_stream(torch.cuda.current_stream())
    l0 = dqo.dqo_launch_count(bctx)
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph, stream=cap_stream, capture_error_mode="thread_local"):
            graph_body()
    torch.cuda.current_stream().wait_stream(cap_stream)
    launches_per_step = dqo.dqo_launch_count(bctx) - l0
    for _ in range(max(args.warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()

    # ---- device-timed region
    phase_sum = {k: 0.0 for k in dqo.PHASES}
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(smi_id)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    graph_timing = True
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
        if graph_timing:
            try:
                ph = dqo.dqo_get_timings(bctx)
            except dqo.DqoError:
                graph_timing = False
                continue
            for k, v in ph.items():
                if v >= 0:
                    phase_sum[k] += v
    torch.cuda.synchronize()
    launches = launches_per_step * args.steps
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, args.steps, total_ms)
    phases = {k: v / args.steps for k, v in phase_sum.items() if v > 0}
    phase_source = "event-record nodes of the replayed graph"
    if not graph_timing:
        # the same kernels run eagerly (phase events recorded on the stream)
        dqo.dqo_set_timing(bctx, True)
        reps = max(20, args.steps // 5)
        phase_sum = {k: 0.0 for k in dqo.PHASES}
        for _ in range(reps):
            flush.zero_()
            graph_body()
            for k, v in dqo.dqo_get_timings(bctx).items():
                if v >= 0:
                    phase_sum[k] += v
        phases = {k: v / reps for k, v in phase_sum.items() if v > 0}
        phase_source = "eager calls of the same step (graph events could not be timed)"
    pairs_b, over_b = dqo.dqo_batch_check(bctx)

    # ---- the same step through the single-keyframe calls (host waits once per forward)
    dqo.dqo_set_timing(ctx, True)
    s_steps = max(20, args.steps // 3)
    s_phase = {k: 0.0 for k in dqo.PHASES}
    s_ms = 0.0
    for i in range(s_steps):
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        step()
        a1.record(stream)
        ph = dqo.dqo_get_timings(ctx)
        for k, v in ph.items():
            if v >= 0:
                s_phase[k] += v
        torch.cuda.synchronize()
        s_ms += a0.elapsed_time(a1)
    dqo.dqo_set_timing(ctx, False)
    single_call = {"value": world * s_steps / (s_ms / 1e3), "unit": UNIT, "ms_per_step": s_ms / s_steps,
                   "phases_ms": {k: round(v / s_steps, 4) for k, v in s_phase.items() if v > 0},
                   "form": "dqo_render_forward + dqo_render_backward + dqo_quadric_bbox_loss per step (the "
                           "forward waits on the host for the pair count)"}

    # ---- end to end through the C ABI with host buffers
    pin = {k: v.cpu().pin_memory() for k, v in g.items()}
    pin_t = {k: v.cpu().pin_memory() for k, v in t.items()}
    pin_q = {k: v.cpu().pin_memory() for k, v in q.items()}
    host_out = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in grads.items()}
    host_loss = torch.empty(4, pin_memory=True)
    host_q = (torch.empty(nq, pin_memory=True), torch.empty(nq, 9, pin_memory=True))
    h2d = sum(v.numel() * v.element_size() for d in (pin, pin_t, pin_q) for v in d.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out.values()) + 16 + nq * 40

    # two buffer sets, one captured graph each: step i+1's inputs go up on a copy stream
    # while step i computes, and step i's results come down while step i+1 computes
    g2 = {k: torch.empty_like(v) for k, v in g.items()}
    t2 = {k: torch.empty_like(v) for k, v in t.items()}
    q2 = {k: torch.empty_like(v) for k, v in q.items()}
    out2 = {k: torch.empty_like(v) for k, v in out.items()}
    grads2 = {k: torch.empty_like(v) for k, v in grads.items()}
    qloss2, qgrad2 = torch.empty_like(qloss), torch.empty_like(qgrad)
    kfb2 = dqo.keyframe(g2, NUM_OBJECTS, cam, t2, out2, grads2)
    for d, src in ((g2, g), (t2, t), (q2, q)):
        for k in d:
            d[k].copy_(src[k])

    def graph_body2():
        main = torch.cuda.current_stream()
        qside.wait_stream(main)
        with torch.cuda.stream(qside):
            dqo.dqo_quadric_bbox_loss(bctx, q2["params"], q2["P"], q2["q_ptr"], q2["pair_v"], q2["obs_bbox"],
                                      qloss2, qgrad2)
        dqo.dqo_batch_step(bctx, bst, [kfb2], None, cps, sched)
        main.wait_stream(qside)

    dqo.dqo_set_timing(bctx, False)
    graph2 = torch.cuda.CUDAGraph()
    cap_stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph2, stream=cap_stream, capture_error_mode="thread_local"):
            graph_body2()
    torch.cuda.current_stream().wait_stream(cap_stream)
    sets = [dict(g=g, t=t, q=q, grads=grads, out=out, ql=qloss, qg=qgrad, graph=graph),
            dict(g=g2, t=t2, q=q2, grads=grads2, out=out2, ql=qloss2, qg=qgrad2, graph=graph2)]
    copy_stream = torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]
    for e in ev_out:
        e.record(stream)

    def upload(k):
        sk = sets[k]
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_done[k])     # the set's previous step has finished with it
            for d, src in ((sk["g"], pin), (sk["t"], pin_t), (sk["q"], pin_q)):
                for name in d:
                    d[name].copy_(src[name], non_blocking=True)
            ev_in[k].record(copy_stream)

    def download(k):
        sk = sets[k]
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_done[k])
            for name in sk["grads"]:
                host_out[name].copy_(sk["grads"][name], non_blocking=True)
            host_loss.copy_(sk["out"]["loss"], non_blocking=True)
            host_q[0].copy_(sk["ql"], non_blocking=True)
            host_q[1].copy_(sk["qg"], non_blocking=True)
            ev_out[k].record(copy_stream)

    def run_e2e(steps_):
        for e in ev_done:
            e.record(stream)
        upload(0)
        for i in range(steps_):
            k = i % 2
            stream.wait_event(ev_in[k])
            stream.wait_event(ev_out[k])        # its previous results are on the host
            sets[k]["graph"].replay()
            ev_done[k].record(stream)
            if i + 1 < steps_:
                upload(1 - k)
            download(k)
        stream.wait_stream(copy_stream)

    run_e2e(3)
    torch.cuda.synchronize()
    e_steps = max(10, args.steps // 4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    run_e2e(e_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    e2e_val = job_throughput(world, e_steps, e_ms)

    # ---- measured FP32 FMA and ex2 peaks of this GPU (the library's probe kernels)
    alu = alu_peaks(dqo, dev, stream, smi_id)
    fp32_peak = alu["fp32_fma_tflops"]
    props = torch.cuda.get_device_properties(local_rank)
    sms = props.multi_processor_count
    sm_max = clk.get("sm_max_mhz") or alu["clocks"].get("sm_max_mhz")
    derived = sms * FP32_LANES * 2 * sm_max * 1e6 / 1e12 if sm_max else None

    # ---- roofline of the dominant kernels (FP32 pipe): the blend's forward + backward
    # (the phase also holds the per-keyframe loss sum, a few microseconds)
    dom = "blend_step"
    flops = FLOPS_PER_EVAL[dom] * evals
    achieved = flops / (phases[dom] * 1e-3) / 1e12
    kname = {dqo.SCHEDULE_FUSED: "k_blend_step", dqo.SCHEDULE_SPLIT: "k_blend_fwd_queue + k_blend_bwd_queue",
             dqo.SCHEDULE_PER_KEYFRAME: "k_blend_forward + k_blend_backward"}[sched]
    ex2_per_step = 2 * evals                 # one exponential per evaluation, forward and backward
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic_for(dom),
            "evals_per_launch": evals, "evals_tile_per_launch": evals_tile,
            "eval_share_of_tile_walk": evals / evals_tile if evals_tile else None,
            "flops_per_eval": FLOPS_PER_EVAL[dom],
            "frac_kernel_count": FLOPS_PER_EVAL_KERNEL[dom] * evals / (phases[dom] * 1e-3) / 1e12 / fp32_peak,
            "ex2_frac": ex2_per_step / (phases[dom] * 1e-3) / 1e12 / alu["ex2_tops"],
            "peak_basis": f"measured: FP32 FMA probe (dqo_alu_probe) on this GPU, best of 5 launches of ~5 ms "
                          f"filling all {sms} SMs, median SM clock {alu['clocks'].get('sm_mhz')} MHz (of measured)",
            "derived_peak_context": derived,
            "ex2_peak_tops": alu["ex2_tops"]}

    # ---- HBM rooflines of the projection, sort and gradient-scatter phases
    peaks, peak_src = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    hbm = {}
    for ph, (per_g, per_pair) in HBM_BYTES.items():
        if ph not in phases:
            continue
        nbytes = per_g * n + per_pair * pairs_b
        gbs = nbytes / (phases[ph] * 1e-3) / 1e9
        hbm[ph] = {"bytes": nbytes, "ms": round(phases[ph], 4), "achieved": round(gbs, 1),
                   "frac": round(gbs / hbm_peak, 4) if hbm_peak else None}
    if "depth_sort" in phases and "binning" in phases:
        t_sort = (phases["depth_sort"] + phases["binning"]) * 1e-3
        amin = SORT_MIN_BYTES[0] * n + SORT_MIN_BYTES[1] * pairs_b
        hbm["sort_algorithmic_minimum"] = {"bytes": amin, "achieved": round(amin / t_sort / 1e9, 1),
                                           "frac": round(amin / t_sort / 1e9 / hbm_peak, 4) if hbm_peak else None}
    hbm["peak_gbs"] = hbm_peak
    hbm["peak_basis"] = ("measured STREAM-style copy (MEASURED_PEAKS.json)" if peak_src == "measured"
                         else "fallback figure for a GB300 copy (no measured peaks file)")

    # ---- batched plain quadric fits: 512 quadrics, 3..40 views, Eq. 1 init + 100 Adam steps
    from paper_2503_02223_gb300 import synth
    fq = synth.batched_quadric_fits(SEED + 1)
    fd = dqo.to_device({k: fq[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")}, dev)
    nfit = fq["q_ptr"].shape[0] - 1
    f_par = torch.zeros(nfit, 9, device=dev)
    f_loss = torch.zeros(nfit, device=dev)
    f_ok = torch.zeros(nfit, dtype=torch.uint8, device=dev)

    def fit_call():
        dqo.dqo_quadric_fit(ctx, fd["P"], fd["q_ptr"], fd["pair_v"], fd["obs_bbox"], FIT_ITERS, 1e-2, None,
                            f_par, f_loss, f_ok, stream)

    for _ in range(3):
        fit_call()
    torch.cuda.synchronize()
    fit_reps = 20
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(fit_reps):
        fit_call()
    f1.record(stream)
    torch.cuda.synchronize()
    fit_ms = f0.elapsed_time(f1) / fit_reps
    npairs_fit = int(fq["pair_v"].shape[0])
    fit_flops = QUADRIC_FLOPS_PER_PAIR * npairs_fit * FIT_ITERS
    fit_tflops = fit_flops / (fit_ms * 1e-3) / 1e12
    fits = {"value": world * nfit / (fit_ms * 1e-3), "unit": "fits/s", "ms_per_batch": fit_ms,
            "batch": nfit, "views": f"{int(fq['counts'].min())}..{int(fq['counts'].max())}",
            "pairs": npairs_fit, "iters": FIT_ITERS, "form": "plain: Eq. 1 SVD init + 100 Adam steps, one launch",
            "ok_fraction": float(f_ok.float().mean().item()),
            "mean_bbox_loss": float(f_loss.mean().item()),
            "roofline": {"bound": "alu", "achieved": fit_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": fit_tflops / fp32_peak, "flops_per_pair_step": QUADRIC_FLOPS_PER_PAIR,
                         "flops_per_launch": fit_flops, "traffic": None,
                         "note": "refinement flops only (the Eq. 1 initialisation is not counted)",
                         "peak_basis": "measured FP32 FMA probe (of measured)"}}

    if not args.no_learned:
        fits["learned"] = learned_section(ctx, dev, stream, world, fd, nfit, fit_ms, fq)
    batched_section.no_tune = args.no_tune
    batched = None if args.no_batched else batched_section(dev, stream, world, fq, fd)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(kf, m_pairs, args), "clocks": clk,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "form": "each step's inputs copied from pinned host memory and its gradients, losses and "
                            "quadric gradient copied back, overlapped with the neighbouring steps' compute "
                            "(two buffer sets, a copy stream)"},
            "gpu_launches": launches, "roofline": roof, "hbm_phases": hbm,
            "phases_ms": {k: round(v, 4) for k, v in phases.items()}, "phases_from": phase_source,
            "step_form": "dqo_batch_step (1 keyframe) + dqo_quadric_bbox_loss (a concurrent branch) in one "
                         f"CUDA graph, {launches_per_step} kernels per step; tile pairs {pairs_b}, overflow {over_b}",
            "tuned": {"tile": f"{bst.tile_w}x{bst.tile_h}", "ctas_per_sm": cps, "schedule": sched,
                      "candidates_ms": tune_table(dqo, tune_ms)},
            "single_call": single_call,
            "quadric_fits": fits}
    if batched is not None:
        line["batched"] = batched
    if not args.no_adjoint_1m:
        line["adjoint_1m"] = adjoint_1m_section(dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        H_ = kf["camera"]["height"]
        cores = os.cpu_count() or 1
        model = cpu_model()
        t_full, nb = oracle_full_parallel(kf, targets, cores)
        # single thread: one 16-row band (its projection of all Gaussians included), scaled
        # to the whole image by rows -- an upper bound on the single-thread keyframe time
        t_band, _ = oracle_full_parallel(kf, targets, 1, [(320, 16)])
        line["cpu_baseline"] = {"value": 1.0 / t_full, "unit": UNIT, "cores": nb, "kind": "oracle",
                                "host_cores": cores, "cpu_model": model,
                                "sample": f"the whole {H_}-row image once (forward + backward, FP64), rows in {nb} "
                                          f"bands of whole tile rows run on {nb} threads, each band projecting all "
                                          f"300k Gaussians",
                                "single_thread": {"value": 1.0 / (t_band * H_ / 16), "unit": UNIT, "cores": 1,
                                                  "sample": "one 16-row band (rows 320..335, forward + backward, "
                                                            "projecting all 300k Gaussians) on one thread, scaled "
                                                            f"by {H_}/16 rows"}}
        t_fit, nf, nth = oracle_fits(fq, cores)
        t_fit1, nf1, _ = oracle_fits(fq, 1)
        fits["cpu_baseline"] = {"value": nf / t_fit, "unit": "fits/s", "cores": nth, "kind": "oracle",
                                "host_cores": cores, "cpu_model": model,
                                "sample": f"the same {nf} plain fits (FP64 Eq. 1 init + {FIT_ITERS} Adam steps), "
                                          f"split into {nth} chunks run on {nth} threads",
                                "single_thread": {"value": nf1 / t_fit1, "unit": "fits/s", "cores": 1,
                                                  "sample": f"the same {nf1} fits on one thread"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    bctx.close()


def learned_section(ctx, dev, stream, world, fd, nfit, plain_fit_ms, fq):
    """Learned quadric proposal: train the network on 1M samples with the library's tensor-core
    kernels (one CUDA graph per epoch), then fit the 512-quadric batch from its proposals, and
    the same quadrics from their first two views only (where the plain fit has no answer)."""
    import numpy as np
    import torch

    from paper_2503_02223_gb300 import dqo, proposal, synth
    t0 = time.perf_counter()
    s = synth.proposal_samples(SEED + 3, MLP_TRAIN_SAMPLES)
    gen_s = time.perf_counter() - t0
    d = dqo.to_device({k: s[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")}, dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    labels, ok = proposal.make_labels(ctx, d)
    e1.record(stream)
    torch.cuda.synchronize()
    label_ms = e0.elapsed_time(e1)
    st = dqo.MlpState(dev)
    dqo.dqo_mlp_set_params(st, torch.from_numpy(synth.mlp_init_params(SEED + 3)).to(dev))
    tr = proposal.Trainer(ctx, st, d, labels, batch=MLP_BATCH, epochs=MLP_EPOCHS, length_scale=s["length_scale"],
                          lr=2e-3, lr_final=1e-5)
    first = tr.epoch()                         # warm-up epoch (sizes the context's workspace)
    torch.cuda.synchronize()
    e0.record(stream)
    hist = [tr.epoch_async() for _ in range(MLP_EPOCHS - 1)]
    e1.record(stream)
    torch.cuda.synchronize()
    hist = [float(v) for v in hist]
    train_ms = e0.elapsed_time(e1) / (MLP_EPOCHS - 1)
    samples = tr.steps * MLP_BATCH
    flops = MLP_FLOPS_PER_SAMPLE * samples
    peaks, peak_src = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained")
    achieved = flops / (train_ms * 1e-3) / 1e12
    # the 512-fit batch: proposal from the first <= 8 views + the same 100 refinement steps
    reps = 20

    def learned_call():
        prop = proposal.propose(ctx, st, fd, length_scale=s["length_scale"])
        return proposal.fit(ctx, fd, start=prop)

    for _ in range(3):
        learned_call()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        out = learned_call()
    e1.record(stream)
    torch.cuda.synchronize()
    learned_ms = e0.elapsed_time(e1) / reps
    plain = proposal.fit(ctx, fd)
    # the first two views of every quadric: the Eq. 1 system is underdetermined there
    q_ptr = fq["q_ptr"]
    sel = np.stack([q_ptr[:-1], q_ptr[:-1] + 1], 1).reshape(-1)
    two = dqo.to_device({"P": np.ascontiguousarray(fq["P"][fq["pair_v"][sel]]),
                         "q_ptr": (np.arange(nfit + 1) * 2).astype(np.int32),
                         "pair_v": np.arange(2 * nfit, dtype=np.int32),
                         "obs_bbox": np.ascontiguousarray(fq["obs_bbox"][sel])}, dev)
    plain2 = proposal.fit(ctx, two)
    e0.record(stream)
    for _ in range(reps):
        out2 = proposal.fit(ctx, two, start=proposal.propose(ctx, st, two, length_scale=s["length_scale"]))
    e1.record(stream)
    torch.cuda.synchronize()
    two_ms = e0.elapsed_time(e1) / reps
    all_loss = torch.zeros(nfit, device=dev)
    dqo.dqo_quadric_bbox_loss(ctx, out2["params"], fd["P"], fd["q_ptr"], fd["pair_v"], fd["obs_bbox"], all_loss)
    torch.cuda.synchronize()
    return {"value": world * nfit / (learned_ms * 1e-3), "unit": "fits/s", "ms_per_batch": learned_ms,
            "vs_plain_speed": plain_fit_ms / learned_ms,
            "mean_bbox_loss": float(out["loss"].mean().item()),
            "plain_mean_bbox_loss": float(plain["loss"].mean().item()),
            "two_views": {"plain_ok_fraction": float(plain2["ok"].float().mean().item()),
                          "learned_fits_per_s": world * nfit / (two_ms * 1e-3),
                          "learned_mean_bbox_loss_all_views": float(all_loss.mean().item()),
                          "note": "each quadric fitted from its first 2 views (the Eq. 1 system is "
                                  "underdetermined: the plain fit returns none); the loss is then evaluated "
                                  "on all of its views, against plain_mean_bbox_loss fitted on all views"},
            "form": "features + BF16 MLP proposal (tcgen05) + 100 Adam steps from it, 4 launches",
            "training": {"samples": samples, "epochs": MLP_EPOCHS, "batch": MLP_BATCH,
                         "ms_per_epoch": train_ms, "samples_per_s": samples / (train_ms * 1e-3),
                         "loss_first_epoch": first, "loss_last_epoch": hist[-1],
                         "label_fits_ms": label_ms, "label_fits_ok": float(ok.float().mean().item()),
                         "generation_s_host": gen_s,
                         "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                      "frac": achieved / peak if peak else None,
                                      "peak_basis": ("measured bf16 cuBLAS sustained (MEASURED_PEAKS.json)"
                                                     if peak_src == "measured"
                                                     else "fallback bf16 sustained figure (no measured peaks file)"),
                                      "flops_per_sample": MLP_FLOPS_PER_SAMPLE,
                                      "traffic": None}}}


def adjoint_1m_section(dev, stream) -> dict:
    """1M Gaussians at 1200x680 (the indoor recipe with 3.33x the Gaussians): forward with
    the fused losses + backward through the library, the blend state recomputed in the
    backward (the forward keeps only T_final and the blended count per pixel).  Reports the
    device memory it takes and its time."""
    import torch

    from paper_2503_02223_gb300 import dqo, synth
    kf = synth.indoor_keyframe(SEED + 4, n_total=1_000_000, object_total=783_000)
    cam = kf["camera"]
    g = dqo.to_device(kf["gaussians"], dev)
    t = dqo.to_device(synth.raycast_targets(kf), dev)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    free0, _ = torch.cuda.mem_get_info(dev)
    base = torch.cuda.memory_allocated(dev)
    ctx = dqo.Context(dev.index)
    st = dqo.settings()
    out = dqo.alloc_outputs(cam["width"], cam["height"], dev)
    grads = dqo.alloc_grads(g["means"].shape[0], dev)
    gs, cs, ts = dqo.gaussians(g, NUM_OBJECTS), dqo.camera(cam), dqo.targets(t)

    def step():
        dqo.dqo_render_forward(ctx, st, gs, cs, ts, dqo.render_out(out), stream)
        dqo.dqo_render_backward(ctx, st, gs, cs, ts, None, dqo.gaussian_grads(grads), stream)

    step()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    torch_peak = torch.cuda.max_memory_allocated(dev) - base
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    m, nvis, _ = dqo.dqo_get_counts(ctx)
    ctx.close()
    return {"gaussians": int(kf["gaussians"]["means"].shape[0]), "visible": int(nvis), "tile_gaussian_pairs": int(m),
            "ms_per_iter": ms, "iters_per_s": 1e3 / ms,
            "peak_memory_mib": {"device_in_use": (free0 - free1) / 2 ** 20, "torch_max_allocated": torch_peak / 2 ** 20},
            "form": "dqo_render_forward (fused losses) + dqo_render_backward per iteration, the backward re-walking "
                    "each pixel's list (no per-(pixel, Gaussian) state kept)"}


def tune_table(dqo, ms) -> dict:
    names = {0: "fused", 1: "split", 2: "per-keyframe"}
    out = {}
    for i, m in enumerate(ms):
        w, h, c, sc = dqo.tune_candidate(i)
        out[f"{w}x{h}/{names[sc]}" + (f"/{c}" if sc != 2 else "")] = round(m, 4)
    return out


BATCH_KEYFRAMES = 8
BATCH_REPS = 20


def batched_section(dev, stream, world, fq, fd):
    """8 keyframes of uneven resolution (four 640x480 f=525, four 1200x680 f=600) over 8
    indoor scenes of 200k..500k Gaussians and 20..60 objects, plus the 512 plain fits:
    the single-launch form (each keyframe's forward + backward calls in turn, then the fit
    launch) against the batched step (tuned, replayed from a CUDA graph)."""
    import numpy as np
    import torch

    from paper_2503_02223_gb300 import dqo, synth
    Ns = np.linspace(200_000, 500_000, BATCH_KEYFRAMES).astype(int)
    objs = np.linspace(20, 60, BATCH_KEYFRAMES).astype(int)
    cases = []
    for k in range(BATCH_KEYFRAMES):
        small = k % 2 == 0
        kf = synth.indoor_keyframe(SEED + 10 + k, n_total=int(Ns[k]), n_obj=int(objs[k]),
                                   width=640 if small else 1200, height=480 if small else 680,
                                   f=525.0 if small else 600.0, object_total=int(0.783 * Ns[k]))
        cases.append((kf, synth.raycast_targets(kf), int(objs[k]) + 1))
    gd = [dqo.to_device(kf["gaussians"], dev) for kf, _, _ in cases]
    td = [dqo.to_device(t, dev) for _, t, _ in cases]
    outs = [dqo.alloc_outputs(kf["camera"]["width"], kf["camera"]["height"], dev) for kf, _, _ in cases]
    grads = [dqo.alloc_grads(kf["gaussians"]["means"].shape[0], dev) for kf, _, _ in cases]
    nfit = fd["q_ptr"].shape[0] - 1
    f_par = torch.zeros(nfit, 9, device=dev)
    f_loss = torch.zeros(nfit, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # ---- single-launch form
    ctx = dqo.Context(dev.index)
    st = dqo.settings()
    per = [(dqo.gaussians(gd[k], cases[k][2]), dqo.camera(cases[k][0]["camera"]), dqo.targets(td[k]),
            dqo.render_out(outs[k]), dqo.gaussian_grads(grads[k])) for k in range(BATCH_KEYFRAMES)]

    def single():
        for gs, cs, ts, os_, gg in per:
            dqo.dqo_render_forward(ctx, st, gs, cs, ts, os_, stream)
            dqo.dqo_render_backward(ctx, st, gs, cs, ts, None, gg, stream)
        dqo.dqo_quadric_fit(ctx, fd["P"], fd["q_ptr"], fd["pair_v"], fd["obs_bbox"], FIT_ITERS, 1e-2, None, f_par,
                            f_loss, None, stream)

    for _ in range(3):
        single()
    torch.cuda.synchronize()
    loss_single = [o["loss"].clone() for o in outs]
    e0.record(stream)
    for _ in range(BATCH_REPS):
        single()
    e1.record(stream)
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1) / BATCH_REPS

    # ---- batched form: tuned, captured, replayed
    bctx = dqo.Context(dev.index)
    bst = dqo.settings()
    kfs = [dqo.keyframe(gd[k], cases[k][2], cases[k][0]["camera"], td[k], outs[k], grads[k])
           for k in range(BATCH_KEYFRAMES)]
    fb = dqo.fit_batch(fd["P"], fd["q_ptr"], fd["pair_v"], fd["obs_bbox"], FIT_ITERS, 1e-2, None, None, f_par,
                       f_loss, None)
    dqo.dqo_batch_step(bctx, bst, kfs, fb)             # same 16x16 tiles as the single form
    torch.cuda.synchronize()
    same_loss = all(torch.equal(a, o["loss"]) for a, o in zip(loss_single, outs))
    if getattr(batched_section, "no_tune", False):
        cps, sched, tune_ms = 0, dqo.SCHEDULE_SPLIT, []
    else:
        cps, sched, tune_ms = dqo.dqo_batch_tune(bctx, bst, kfs, fb, reps=3)
    dqo.dqo_batch_step(bctx, bst, kfs, fb, cps, sched)        # sizing call for the chosen configuration
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    cs_ = torch.cuda.Stream(dev)
    cs_.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs_):
        with torch.cuda.graph(graph, stream=cs_, capture_error_mode="thread_local"):
            dqo.dqo_batch_step(bctx, bst, kfs, fb, cps, sched)
    torch.cuda.current_stream().wait_stream(cs_)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(BATCH_REPS):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / BATCH_REPS
    pairs, over = dqo.dqo_batch_check(bctx)
    res = {"workload": "8 keyframes (4x 640x480, 4x 1200x680) over 8 indoor scenes of 200k..500k Gaussians, "
                       "20..60 objects, + 512 plain fits (3..40 views, 100 Adam steps)",
           "gaussians": int(Ns.sum()), "tile_gaussian_pairs": pairs, "overflow": over,
           "single_launch_ms": single_ms, "batched_graph_ms": batched_ms, "speedup": single_ms / batched_ms,
           "keyframe_iters_per_s": world * BATCH_KEYFRAMES / (batched_ms * 1e-3),
           "single_keyframe_iters_per_s": world * BATCH_KEYFRAMES / (single_ms * 1e-3),
           "losses_match_single": same_loss,
           "tuned": {"tile": f"{bst.tile_w}x{bst.tile_h}", "ctas_per_sm": cps, "schedule": sched,
                     "candidates_ms": tune_table(dqo, tune_ms)},
           "form": "one launch per phase over all keyframes; blend: "
                   + {0: "one persistent forward+backward kernel on a work queue",
                      1: "persistent forward and backward kernels on work queues",
                      2: "forward and backward kernels per keyframe"}[sched]
                   + " (tiles heaviest first); fits on a concurrent graph branch; one CUDA graph"}
    ctx.close()
    bctx.close()
    return res


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
