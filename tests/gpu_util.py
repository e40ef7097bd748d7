"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and
compare it with the FP64 oracle under the tolerances the tests state."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2503_02223_gb300 import dqo, synth

# Parity tolerances (float32 GPU vs float64 oracle)
TOL_IMG = 1e-4          # absolute, rendered colour / depth / alpha / ins
TOL_GRAD_REL = 1e-3     # relative, gradients
TOL_GRAD_FLOOR = 1e-2   # per-element floor as a fraction of the tensor's largest |g|


class Render:
    """Forward (+ optional backward) of the CUDA path on numpy inputs."""

    def __init__(self, g_np: dict, cam: dict, num_objects: int, targets_np: dict | None = None, id_map=True,
                 **st):
        self.ctx = dqo.Context()
        self.g = dqo.to_device(g_np)
        self.n = g_np["means"].shape[0]
        self.cam = cam
        self.num_objects = num_objects
        self.t = dqo.to_device(targets_np) if targets_np is not None else None
        self.st = dqo.settings(**st)
        self.gs = dqo.gaussians(self.g, num_objects)
        self.cs = dqo.camera(cam)
        self.ts = dqo.targets(self.t)
        W, H = cam["width"], cam["height"]
        self.out = dqo.alloc_outputs(W, H, loss=targets_np is not None, id_map=id_map)

    def forward(self):
        dqo.dqo_render_forward(self.ctx, self.st, self.gs, self.cs, self.ts, dqo.render_out(self.out))
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in self.out.items()}

    def backward(self, pixel_grads: dict | None = None):
        grads = dqo.alloc_grads(self.n)
        pg = None
        if pixel_grads is not None:
            self._pg = dqo.to_device(pixel_grads)
            pg = dqo.pixel_grads(self._pg)
        dqo.dqo_render_backward(self.ctx, self.st, self.gs, self.cs, self.ts, pg, dqo.gaussian_grads(grads))
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in grads.items()}

    def buffer(self, which, dtype):
        nbytes = dqo.dqo_get_buffer(self.ctx, which)
        dst = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
        dqo.dqo_get_buffer(self.ctx, which, dst)
        torch.cuda.synchronize()
        return dst[:nbytes].cpu().numpy().view(dtype)

    def proj(self):
        a = self.buffer(dqo.DQO_BUF_PROJ, np.float32).reshape(3, self.n, 4)
        return a

    def close(self):
        self.ctx.close()


def oracle_settings(num_objects, **st):
    return oracle.settings(num_objects=num_objects, **st)


def tiny_case(seed=1001, n=2000, width=320, height=240, f=300.0, og_fraction=1.0, n_objects=4):
    g = synth.tiny_gaussians(seed, n=n, n_objects=n_objects, og_fraction=og_fraction)
    cam = synth.tiny_camera(width=width, height=height, f=f)
    tgt = oracle.render(synth.tiny_gaussians(seed + 1, n=n, n_objects=n_objects), cam,
                        oracle.settings(num_objects=n_objects))
    t = dict(rgb=tgt["rgb"].astype(np.float32), depth=tgt["depth"].astype(np.float32),
             gt_id=tgt["id_map"].astype(np.int32))
    return g, cam, t


KINK_MARGIN = 1e-4   # ten times the largest colour / depth difference measured at full size


def condition_targets(g, cam, t, st_o):
    """Moves targets off the L1 kinks (|render - target| < KINK_MARGIN in the oracle's
    render), so both sides differentiate |.| on the same side.  Uses oracle outputs only."""
    r = oracle.render(g, cam, st_o, t)
    t = {k: v.copy() for k, v in t.items()}
    e = r["rgb"] - t["rgb"]
    near = (np.abs(e) < KINK_MARGIN) & (e != 0)
    t["rgb"][near] += np.where(e[near] > 0, -1e-3, 1e-3)
    ed = r["depth"] - t["depth"]
    nd = (np.abs(ed) < KINK_MARGIN) & (ed != 0) & (t["depth"] > 0)
    t["depth"][nd] += np.where(ed[nd] > 0, -1e-3, 1e-3)
    return t


def assert_grads_close(got: dict, ref: dict, keys=("means", "log_scales", "quats", "opacity_logit", "rgb"),
                       rel=TOL_GRAD_REL, floor=TOL_GRAD_FLOOR, report=None):
    """Per Gaussian, each parameter's gradient vector (means 3, log-scales 3, quaternion 4,
    opacity 1, colour 3) within rel * max(|ref_i|, floor * max_j |ref_j|) in norm, plus the
    oracle's bound |unc_i| on the change a near-threshold decision taken the other way can
    cause; each whole tensor within rel in norm with the same allowance.  Gaussians feeding
    a pixel at an L1 kink (ref["amb"] bit 3; the targets are conditioned so there are none)
    are left out."""
    keep = (ref["amb"] & 8) == 0
    for k in keys:
        g = got[k].reshape(got[k].shape[0], -1)[keep].astype(np.float64)
        r = ref[k].reshape(ref[k].shape[0], -1)[keep]
        u = ref["unc"][k].reshape(ref[k].shape[0], -1)[keep]
        rn = np.linalg.norm(r, axis=1)
        scale = rn.max() if rn.size else 0.0
        if scale == 0:
            assert np.abs(g).max(initial=0) == 0, k
            continue
        base = rel * np.maximum(rn, floor * scale)
        un = np.linalg.norm(u, axis=1)
        err = np.linalg.norm(g - r, axis=1)
        bad = err > base + un
        nrm = np.linalg.norm(g - r) / np.linalg.norm(r)
        unrm = np.linalg.norm(u) / np.linalg.norm(r)
        if report is not None:
            report[k] = dict(bad=int(bad.sum()), norm=float(nrm), unc_norm=float(unrm),
                             worst=float((err / (base + un)).max()), widened=float((un > base).mean()))
        assert nrm <= rel + unrm, (k, nrm, unrm)
        worst = int(np.argmax(err / (base + un)))
        assert not bad.any(), (k, int(bad.sum()), float((err / (base + un)).max()),
                               int(np.nonzero(keep)[0][worst]), r[worst].tolist(), g[worst].tolist())
