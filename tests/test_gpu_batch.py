"""The batched optimisation step (several keyframes of different resolutions and scenes,
plus a batch of quadric fits, every phase one launch over the batch, the blend one
persistent kernel on a work queue): it must give each keyframe what the single-keyframe
calls give it (images bitwise, gradients up to the order of additions), capture in a CUDA
graph, report a pair-capacity overflow instead of faulting, and its autotuner must pick a
working configuration."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_IMG, oracle_settings, tiny_case
from paper_2503_02223_gb300 import dqo, synth

pytestmark = pytest.mark.gpu

NUM_OBJECTS = 4
IMG_KEYS = ("rgb", "depth", "alpha", "ins", "id_map", "update_mask", "loss")
GRAD_KEYS = ("means", "log_scales", "quats", "opacity_logit", "rgb")


def _camera(width, height, f, eye, target=(0.0, 0.0, 0.0)):
    return synth.make_camera(f, f, width / 2.0, height / 2.0, width, height, synth.look_at(eye, target))


def _scenes():
    """Three keyframes: two share a scene (and its gradient buffers), image sizes with
    ragged tiles."""
    gA, camA, tA = tiny_case(seed=1201)
    gB, camB, tB = tiny_case(seed=1203, n=3000, width=200, height=150, f=220.0)
    camC = _camera(96, 80, 90.0, (0.5, -0.4, -2.6))
    tgt = oracle.render(synth.tiny_gaussians(1202, n=2000, n_objects=NUM_OBJECTS), camC,
                        oracle.settings(num_objects=NUM_OBJECTS))
    tC = dict(rgb=tgt["rgb"].astype(np.float32), depth=tgt["depth"].astype(np.float32),
              gt_id=tgt["id_map"].astype(np.int32))
    return [(gA, camA, tA), (gB, camB, tB), (gA, camC, tC)]


class Batch:
    def __init__(self, cases, share=(0, 1, 0), **st):
        self.ctx = dqo.Context()
        self.st = dqo.settings(**st)
        self.scenes = {}
        self.kfs, self.outs, self.grads, self.tgts = [], [], [], []
        for k, (g, cam, t) in enumerate(cases):
            key = share[k] if share else k
            if key not in self.scenes:
                gd = dqo.to_device(g)
                self.scenes[key] = (gd, dqo.alloc_grads(g["means"].shape[0]))
            gd, gr = self.scenes[key]
            td = dqo.to_device(t)
            out = dqo.alloc_outputs(cam["width"], cam["height"], mask=True)
            self.tgts.append(td)
            self.outs.append(out)
            self.grads.append(gr)
            self.kfs.append(dqo.keyframe(gd, NUM_OBJECTS, cam, td, out, gr))

    def step(self, fits=None, ctas_per_sm=0, schedule=dqo.SCHEDULE_FUSED):
        dqo.dqo_batch_step(self.ctx, self.st, self.kfs, fits, ctas_per_sm, schedule)

    def zero_grads(self):
        for gd, gr in self.scenes.values():
            for v in gr.values():
                v.zero_()


def _single(g, cam, t, **st):
    ctx = dqo.Context()
    gd, td = dqo.to_device(g), dqo.to_device(t)
    out = dqo.alloc_outputs(cam["width"], cam["height"], mask=True)
    grads = dqo.alloc_grads(g["means"].shape[0])
    s = dqo.settings(**st)
    dqo.dqo_render_forward(ctx, s, dqo.gaussians(gd, NUM_OBJECTS), dqo.camera(cam), dqo.targets(td),
                           dqo.render_out(out))
    dqo.dqo_render_backward(ctx, s, dqo.gaussians(gd, NUM_OBJECTS), dqo.camera(cam), dqo.targets(td), None,
                            dqo.gaussian_grads(grads))
    torch.cuda.synchronize()
    ctx.close()
    return {k: v.cpu().numpy() for k, v in out.items()}, {k: v.cpu().numpy() for k, v in grads.items()}


def _close(a, b, rel=1e-5):
    scale = max(np.abs(b).max(), 1e-30)
    return np.abs(a - b).max() <= rel * scale


def _check_against_singles(bt, cases, **st):
    singles = [_single(g, cam, t, **st) for g, cam, t in cases]
    for k, (o_ref, _) in enumerate(singles):
        for name in IMG_KEYS:
            got = bt.outs[k][name].cpu().numpy()
            assert np.array_equal(got, o_ref[name]), (k, name)
    # keyframes 0 and 2 share a scene: its gradient is the sum of theirs
    want = {0: [0, 2], 1: [1]}
    for key, members in want.items():
        gr = {n: v.cpu().numpy() for n, v in bt.scenes[key][1].items()}
        for name in GRAD_KEYS:
            ref = sum(singles[m][1][name].astype(np.float64) for m in members)
            assert _close(gr[name], ref), (key, name, np.abs(gr[name] - ref).max(), np.abs(ref).max())


@pytest.mark.parametrize("schedule", [dqo.SCHEDULE_FUSED, dqo.SCHEDULE_SPLIT, dqo.SCHEDULE_PER_KEYFRAME])
@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_batch_step_matches_single_keyframe_calls(tile, schedule):
    cases = _scenes()
    st = dict(tile_w=tile[0], tile_h=tile[1])
    bt = Batch(cases, **st)
    bt.step(schedule=schedule)
    torch.cuda.synchronize()
    _check_against_singles(bt, cases, **st)
    pairs, over = dqo.dqo_batch_check(bt.ctx)
    assert pairs > 0 and not over
    bt.ctx.close()


@pytest.mark.parametrize("share", [(0, 1, 0), (0, 1, 2)])
def test_batch_step_overwrites_gradients_with_grads_zero(share):
    # grads_zero = 1: buffers filled with NaN beforehand hold exactly the step's gradients
    # afterwards -- overwritten where a keyframe uses its buffers alone, cleared and added
    # to where keyframes share them -- equal to a zeroed accumulating step
    cases = _scenes()
    ref = Batch(cases, share=share)
    ref.zero_grads()
    ref.step(schedule=dqo.SCHEDULE_SPLIT)
    bt = Batch(cases, share=share, grads_zero=1)
    for gd, gr in bt.scenes.values():
        for v in gr.values():
            v.fill_(float("nan"))
    for _ in range(2):          # a second step overwrites the first step's gradients
        bt.step(schedule=dqo.SCHEDULE_SPLIT)
    torch.cuda.synchronize()
    for key in ref.scenes:
        for name in GRAD_KEYS:
            a = bt.scenes[key][1][name].cpu().numpy()
            b = ref.scenes[key][1][name].cpu().numpy()
            assert np.isfinite(a).all(), (key, name)
            assert _close(a, b), (key, name)
    ref.ctx.close()
    bt.ctx.close()


def test_single_call_backward_overwrites_gradients_with_grads_zero():
    g, cam, t = tiny_case(seed=1205)
    g = dict(g)
    g["means"] = g["means"].copy()
    g["means"][::5, 2] -= 6.0                # culled Gaussians: their gradient is zero
    _, ref = _single(g, cam, t)
    ctx = dqo.Context()
    gd, td = dqo.to_device(g), dqo.to_device(t)
    out = dqo.alloc_outputs(cam["width"], cam["height"])
    grads = {k: torch.full_like(v, float("nan")) for k, v in dqo.alloc_grads(g["means"].shape[0]).items()}
    st = dqo.settings(grads_zero=1)
    gs, cs, ts = dqo.gaussians(gd, NUM_OBJECTS), dqo.camera(cam), dqo.targets(td)
    dqo.dqo_render_forward(ctx, st, gs, cs, ts, dqo.render_out(out))
    for _ in range(2):
        dqo.dqo_render_backward(ctx, st, gs, cs, ts, None, dqo.gaussian_grads(grads))
    torch.cuda.synchronize()
    for name in GRAD_KEYS:
        # the blend backward adds in a run-dependent order: equal to rounding, and culled
        # Gaussians exactly zero
        a = grads[name].cpu().numpy()
        assert np.isfinite(a).all() and _close(a, ref[name]), name
        assert not a.reshape(a.shape[0], -1)[::5].any(), name
    with pytest.raises(dqo.DqoError):
        dqo.dqo_render_backward(ctx, dqo.settings(grads_zero=2), gs, cs, ts, None, dqo.gaussian_grads(grads))
    ctx.close()


def test_batch_step_against_oracle():
    cases = _scenes()
    bt = Batch(cases)
    bt.step()
    torch.cuda.synchronize()
    g, cam, t = cases[1]
    ref = oracle.render(g, cam, oracle_settings(NUM_OBJECTS), t)
    ok = ref["amb"] == 0
    assert ok.mean() >= 0.99
    got = bt.outs[1]["rgb"].cpu().numpy()
    assert np.abs(got - ref["rgb"]).max(-1)[ok].max() < TOL_IMG
    assert np.abs(bt.outs[1]["depth"].cpu().numpy() - ref["depth"])[ok].max() < TOL_IMG
    np.testing.assert_allclose(bt.outs[1]["loss"].cpu().numpy(), ref["loss"], rtol=1e-4, atol=1e-6)
    bt.ctx.close()


def test_batch_step_in_a_cuda_graph():
    cases = _scenes()
    bt = Batch(cases)
    bt.step()                       # sizing call
    torch.cuda.synchronize()
    first = [{k: v.clone() for k, v in o.items()} for o in bt.outs]
    bt.zero_grads()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
            bt.step()
    torch.cuda.current_stream().wait_stream(s)
    bt.zero_grads()
    for o in bt.outs:
        for v in o.values():
            v.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for k, o in enumerate(bt.outs):
        for name in IMG_KEYS:
            assert torch.equal(o[name], first[k][name]), (k, name)
    # two replays accumulate two steps' gradients
    single = _single(*cases[1])[1]
    got = {n: v.cpu().numpy() for n, v in bt.scenes[1][1].items()}
    for name in GRAD_KEYS:
        assert _close(got[name], 2 * single[name].astype(np.float64)), name
    bt.ctx.close()


def test_batch_fits_run_beside_the_keyframes():
    cases = _scenes()
    q = synth.batched_quadric_fits(1204, nq=64, min_views=3, max_views=12)
    d = dqo.to_device({k: q[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")})
    outs = {k: torch.zeros(64, 9, device="cuda") for k in ("init", "params")}
    loss = torch.zeros(64, device="cuda")
    ok = torch.zeros(64, dtype=torch.uint8, device="cuda")
    fb = dqo.fit_batch(d["P"], d["q_ptr"], d["pair_v"], d["obs_bbox"], 50, 1e-2, None, outs["init"], outs["params"],
                       loss, ok)
    bt = Batch(cases)
    bt.step(fits=fb)
    torch.cuda.synchronize()
    ctx = dqo.Context()
    ref_p = torch.zeros(64, 9, device="cuda")
    ref_l = torch.zeros(64, device="cuda")
    dqo.dqo_quadric_fit(ctx, d["P"], d["q_ptr"], d["pair_v"], d["obs_bbox"], 50, 1e-2, None, ref_p, ref_l)
    torch.cuda.synchronize()
    assert torch.equal(outs["params"], ref_p) and torch.equal(loss, ref_l)
    _check_against_singles(bt, cases)
    ctx.close()
    bt.ctx.close()


def test_batch_capacity_overflow_is_reported_then_resized():
    cases = _scenes()
    bt = Batch(cases)
    bt.step()                       # sizes the pair buffers for these scenes
    torch.cuda.synchronize()
    pairs0, over = dqo.dqo_batch_check(bt.ctx)
    assert not over
    # same layout, much larger footprints: more pairs than the capacity
    for gd, _ in bt.scenes.values():
        gd["log_scales"] += 1.5
    bt.step()
    torch.cuda.synchronize()
    pairs1, over = dqo.dqo_batch_check(bt.ctx)
    assert over and pairs1 > pairs0
    # the next step sizes again and is right
    bt.zero_grads()
    bt.step()
    torch.cuda.synchronize()
    pairs2, over = dqo.dqo_batch_check(bt.ctx)
    assert not over and pairs2 == pairs1
    big = [({**g, "log_scales": g["log_scales"] + np.float32(1.5)}, cam, t) for g, cam, t in cases]
    _check_against_singles(bt, big)
    bt.ctx.close()


def test_batch_autotuner_picks_a_working_configuration():
    cases = _scenes()
    bt = Batch(cases)
    cps, sched, ms = dqo.dqo_batch_tune(bt.ctx, bt.st, bt.kfs, None, reps=2)
    assert len(ms) == dqo.TUNE_CANDIDATES and all(m > 0 for m in ms)
    best = int(np.argmin(ms))
    assert dqo.tune_candidate(best) == (bt.st.tile_w, bt.st.tile_h, cps, sched)
    bt.zero_grads()
    bt.step(ctas_per_sm=cps, schedule=sched)
    torch.cuda.synchronize()
    _check_against_singles(bt, cases, tile_w=bt.st.tile_w, tile_h=bt.st.tile_h)
    bt.ctx.close()


def test_batch_invalid_arguments():
    cases = _scenes()
    bt = Batch(cases)
    with pytest.raises(dqo.DqoError):
        dqo.dqo_batch_step(bt.ctx, bt.st, [])
    with pytest.raises(dqo.DqoError):
        dqo.dqo_batch_step(bt.ctx, bt.st, bt.kfs * 6)          # 18 > 16 keyframes
    k = bt.kfs[0]
    k2 = dqo.dqo_keyframe()
    k2.gaussians, k2.camera, k2.out, k2.grads = k.gaussians, k.camera, k.out, k.grads
    with pytest.raises(dqo.DqoError):                          # no targets
        dqo.dqo_batch_step(bt.ctx, bt.st, [k2])
    bt.ctx.close()


def test_indoor_keyframe_batch_step_full_size_parity():
    # The bench's timed configuration (dqo_batch_step on the 300k-Gaussian indoor keyframe,
    # per-keyframe blend schedule, 16x16 tiles): images bitwise those of the single-keyframe
    # calls (whose full-size image parity with the oracle the rasterizer tests check), and
    # every Gaussian gradient against the FP64 oracle with the rasterizer tests' criterion
    # (relative 1e-3 plus the oracle's per-element decision and rounding bound).
    from gpu_util import assert_grads_close, condition_targets
    kf = synth.indoor_keyframe(1002)
    g, cam = kf["gaussians"], kf["camera"]
    st_o = oracle_settings(31)
    t = condition_targets(g, cam, synth.raycast_targets(kf), st_o)
    outs_ref, _ = _single_n(g, cam, t, 31)
    ctx = dqo.Context()
    gd, td = dqo.to_device(g), dqo.to_device(t)
    out = dqo.alloc_outputs(cam["width"], cam["height"], mask=True)
    gr = dqo.alloc_grads(g["means"].shape[0])
    kf_b = dqo.keyframe(gd, 31, cam, td, out, gr)
    # the first call sizes the buffers (pair offsets by a scan of their own); the second is
    # the steady-state step the bench times (the scan inside the pair emission): check it
    dqo.dqo_batch_step(ctx, dqo.settings(), [kf_b], None, 0, dqo.SCHEDULE_PER_KEYFRAME)
    torch.cuda.synchronize()
    for v in list(out.values()) + list(gr.values()):
        v.zero_()
    dqo.dqo_batch_step(ctx, dqo.settings(), [kf_b], None, 0, dqo.SCHEDULE_PER_KEYFRAME)
    torch.cuda.synchronize()
    pairs, over = dqo.dqo_batch_check(ctx)
    assert pairs > 1_000_000 and not over
    for name in IMG_KEYS:
        assert np.array_equal(out[name].cpu().numpy(), outs_ref[name]), name
    refb = oracle.render_backward(g, cam, st_o, t)
    report = {}
    assert_grads_close({k: v.cpu().numpy() for k, v in gr.items()}, refb, report=report)
    print("gradients", report)
    ctx.close()


def _single_n(g, cam, t, nobj, **st):
    ctx = dqo.Context()
    gd, td = dqo.to_device(g), dqo.to_device(t)
    out = dqo.alloc_outputs(cam["width"], cam["height"], mask=True)
    grads = dqo.alloc_grads(g["means"].shape[0])
    s = dqo.settings(**st)
    dqo.dqo_render_forward(ctx, s, dqo.gaussians(gd, nobj), dqo.camera(cam), dqo.targets(td), dqo.render_out(out))
    dqo.dqo_render_backward(ctx, s, dqo.gaussians(gd, nobj), dqo.camera(cam), dqo.targets(td), None,
                            dqo.gaussian_grads(grads))
    torch.cuda.synchronize()
    ctx.close()
    return {k: v.cpu().numpy() for k, v in out.items()}, {k: v.cpu().numpy() for k, v in grads.items()}
