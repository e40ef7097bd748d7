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
TOL_GRAD_FLOOR = 1e-3   # per-element floor as a fraction of the tensor's largest |g|
ID_MARGIN = 1e-5        # the id map is certain where the FP64 top-2 weight margin exceeds this


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

    def last_blended(self):
        """[H, W] index of each pixel's last blended Gaussian (-1: none), read off the GPU's
        own tile list at position n_contrib - 1 (list positions shift when an unrelated
        Gaussian's tile membership differs; the Gaussian itself does not)."""
        W, H = self.cam["width"], self.cam["height"]
        tw, th = self.st.tile_w, self.st.tile_h
        nc = self.buffer(dqo.DQO_BUF_N_CONTRIB, np.uint32).reshape(H, W).astype(np.int64)
        if not nc.any():
            return np.full((H, W), -1, np.int64)
        ranges = self.buffer(dqo.DQO_BUF_TILE_RANGES, np.uint32).reshape(-1, 2).astype(np.int64)
        lst = self.buffer(dqo.DQO_BUF_TILE_LIST, np.uint32).astype(np.int64)
        yy, xx = np.mgrid[0:H, 0:W]
        tile = (yy // th) * (-(-W // tw)) + xx // tw
        pos = np.clip(ranges[tile, 0] + nc - 1, 0, lst.size - 1)
        return np.where(nc > 0, lst[pos], -1)

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
                       rel=TOL_GRAD_REL, floor=TOL_GRAD_FLOOR, report=None, sel=None, max_over=1e-3):
    """Per element: |g - g_ref| <= rel * max(|g_ref|, floor * max |g_ref| over the tensor).  At
    most a fraction `max_over` of the compared Gaussians (or 5) may exceed that per-element
    tolerance, and each of them must be one the oracle flags -- one of its decisions (alpha
    skip / clamp / stop, tile membership) lies within rounding distance of its threshold at
    a pixel with a gradient (ref["amb"] bits 0, 2), or the oracle's bound on single-
    precision rounding (of its gradient sums, and of the projection adjoint's chain)
    exceeds the tolerance -- and lie within the tolerance plus the oracle's bound
    ref["unc"] on how far a correct single-precision evaluation may differ.  Per tensor,
    over the Gaussians within the per-element tolerance, ||g - g_ref|| <= rel ||g_ref||.
    Gaussians feeding a pixel at an L1 kink (bit 3; the targets are conditioned so there
    are none) are left out.  sel: optional index subset compared.  Returns the number of
    Gaussians over the plain tolerance."""
    keep = (ref["amb"] & 8) == 0
    if sel is not None:
        m = np.zeros_like(keep)
        m[sel] = True
        keep &= m
    n = int(keep.sum())
    flagged = (ref["amb"][keep] & 5) != 0
    over = np.zeros(n, bool)
    rows = {}
    for k in keys:
        g = got[k].reshape(got[k].shape[0], -1)[keep].astype(np.float64)
        r = ref[k].reshape(ref[k].shape[0], -1)[keep]
        u = ref["unc"][k].reshape(ref[k].shape[0], -1)[keep]
        scale = np.abs(r).max(initial=0.0)
        if scale == 0:
            assert np.abs(g).max(initial=0) == 0, k
            continue
        tol = rel * np.maximum(np.abs(r), floor * scale)
        err = np.abs(g - r)
        flagged |= (u > tol).any(1)
        over |= (err > tol).any(1)
        rows[k] = (g, r, u, tol, err)
    for k, (g, r, u, tol, err) in rows.items():
        allow = tol + np.where(flagged[:, None], u, 0.0)
        bad = err > allow
        nrm_all = np.linalg.norm(g - r) / np.linalg.norm(r)
        rin = np.linalg.norm(r[~over])
        nrm = np.linalg.norm((g - r)[~over]) / rin if rin > 0 else 0.0
        if report is not None:
            report[k] = dict(bad=int(bad.sum()), norm=float(nrm), norm_all=float(nrm_all),
                             worst=float((err / allow).max()), over=int(((err > tol).any(1)).sum()))
        assert nrm <= rel, (k, nrm)
        worst = np.unravel_index(int(np.argmax(err / allow)), err.shape)
        assert not bad.any(), (k, int(bad.sum()), float((err / allow).max()),
                               int(np.nonzero(keep)[0][worst[0]]), r[worst[0]].tolist(), g[worst[0]].tolist())
    if report is not None:
        report["summary"] = dict(compared=n, flagged=int(flagged.sum()), over_plain_tolerance=int(over.sum()))
    # every Gaussian over the plain tolerance is flagged, and they are few
    assert not (over & ~flagged).any()
    assert over.sum() <= max(max_over * n, 5), (int(over.sum()), n)
    return int(over.sum())


def check_flagged_pixels(g, cam, st_o, t, ref, out, T_final, last, report=None, max_alt=64):
    """Every pixel the oracle flags (ref["amb"] != 0: a decision within rounding distance
    of its threshold or an uncertain tile membership) must match one of the outcomes the
    oracle gives with those decisions taken the other way: colour, depth, alpha, ins and
    T_final within TOL_IMG, the same last blended Gaussian (`last`, from
    Render.last_blended), and the id where that outcome's top-2 margin exceeds ID_MARGIN.
    Returns the number of flagged pixels."""
    yx = np.argwhere(ref["amb"] != 0)
    if yx.size == 0:
        return 0
    alt = oracle.render_alternatives(g, cam, yx[:, ::-1], st_o, None if t is None else t["gt_id"], max_alt=max_alt)
    y, x = yx[:, 0], yx[:, 1]
    v = np.concatenate([out["rgb"][y, x], np.stack([out["depth"][y, x], out["alpha"][y, x], out["ins"][y, x],
                                                    T_final[y, x]], 1)], 1).astype(np.float64)
    close = np.abs(alt["vals"] - v[:, None, :]).max(-1) < TOL_IMG
    close &= alt["last"] == last[y, x].astype(np.int64)[:, None]
    if "id_map" in out:
        gid = out["id_map"][y, x][:, None]
        id_ok = (alt["id_map"] == gid) | ((alt["id_margin"] <= ID_MARGIN) & (alt["id_map"] != -1))
        close &= id_ok
    close &= np.arange(max_alt)[None, :] < alt["count"][:, None]
    matched = close.any(1)
    if report is not None:
        report["flagged"] = int(len(yx))
        report["matched_base"] = int(close[:, 0].sum())
        report["unmatched"] = int((~matched).sum())
    bad = np.nonzero(~matched)[0]
    assert bad.size == 0, (int(bad.size), len(yx), [(int(y[b]), int(x[b]), int(alt["count"][b])) for b in bad[:8]])
    return int(len(yx))
