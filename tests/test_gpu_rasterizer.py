"""Parity of the CUDA rasterizer (through the C ABI) with the FP64 oracle.

Tolerances: rendered colour / depth / alpha / ins within 1e-4 absolute; tile lists and
the depth order bit-exact given the GPU's own FP32 projections; the object-id map exact
on pixels whose FP64 top-2 weight margin exceeds 1e-5 (pixels under that margin at most
0.01% of the image); gradients within 1e-3 relative per element (floor 1e-3 of the
tensor's largest |g|) and per tensor.  A pixel the oracle flags as within rounding
distance of a discrete decision (alpha skip / clamp / stop thresholds, tile-membership
edges) must match one of the outcomes the oracle gives with those decisions taken the
other way; flagged pixels must be rare.  For gradients the oracle bounds the change such
a decision (or FP32 rounding of the gradient sums) can cause, and only the Gaussians it
flags have their per-element tolerance widened by that bound.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import (ID_MARGIN, TOL_IMG, Render, assert_grads_close, check_flagged_pixels, condition_targets,
                      oracle_settings, tiny_case)
from paper_2503_02223_gb300 import dqo, synth

pytestmark = pytest.mark.gpu

LOG2E = 1.4426950408889634


def _img_compare(out, ref, ok, keys=("rgb", "depth", "alpha", "ins")):
    for k in keys:
        d = np.abs(out[k] - ref[k])
        if d.ndim == 3:
            d = d.max(-1)
        assert d[ok].max(initial=0) < TOL_IMG, (k, float(d[ok].max(initial=0)))


def test_projection_parity_config1():
    g, cam, t = tiny_case()
    r = Render(g, cam, 4, t)
    r.forward()
    P = r.proj()
    ref = oracle.preprocess(g, cam, oracle_settings(4))
    vis = ref["visible"] > 0
    sc = -0.5 * LOG2E
    np.testing.assert_allclose(P[0, vis, 0], ref["xy"][vis, 0], atol=2e-4 * 320)
    np.testing.assert_allclose(P[0, vis, 1], ref["xy"][vis, 1], atol=2e-4 * 240)
    np.testing.assert_allclose(P[0, vis, 2] / sc, ref["conic"][vis, 0], rtol=1e-4)
    np.testing.assert_allclose(P[0, vis, 3] / (2 * sc), ref["conic"][vis, 1],
                               rtol=1e-4, atol=1e-4 * np.abs(ref["conic"][vis]).max())
    np.testing.assert_allclose(P[1, vis, 0] / sc, ref["conic"][vis, 2], rtol=1e-4)
    np.testing.assert_allclose(P[1, vis, 1], ref["opac"][vis], rtol=1e-6)
    np.testing.assert_allclose(P[1, vis, 2], ref["z"][vis], rtol=1e-6)
    rect = r.buffer(dqo.DQO_BUF_RECT, np.uint16).reshape(-1, 4).astype(np.int32)
    sure = ref["ambiguous"] == 0
    assert np.array_equal(rect[sure], ref["rect"][sure])
    r.close()


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_tile_lists_bit_exact(tile):
    g, cam, t = tiny_case(width=333, height=251)
    r = Render(g, cam, 4, t, tile_w=tile[0], tile_h=tile[1])
    r.forward()
    _check_tile_lists(r, 333, 251, tile)
    r.close()


def test_tile_lists_bit_exact_wide_keys():
    """Depth-rank bits + tile bits above 32 (140k Gaussians, 49152 tiles): the pair keys are
    64-bit and the pair sort still covers only the tile bits."""
    g = synth.tiny_gaussians(1101, n=140000)
    cam = synth.tiny_camera(width=4096, height=3072, f=3000.0)
    r = Render(g, cam, 4, None)
    r.forward()
    m, nvis, ntiles = dqo.dqo_get_counts(r.ctx)
    assert ntiles == 256 * 192 and int(nvis).bit_length() + int(ntiles - 1).bit_length() > 32
    _check_tile_lists(r, 4096, 3072, (16, 16))
    r.close()


def _check_tile_lists(r, W, H, tile):
    P = r.proj()
    rect = r.buffer(dqo.DQO_BUF_RECT, np.uint16).reshape(-1, 4).astype(np.int32)
    vis = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
    zbits = P[1, :, 2].copy().view(np.uint32)
    ntx, nty = -(-W // tile[0]), -(-H // tile[1])
    ranges_ref, list_ref = oracle.bin_tiles(rect, zbits, vis.astype(np.uint8), ntx, nty)
    ranges = r.buffer(dqo.DQO_BUF_TILE_RANGES, np.uint32).reshape(-1, 2).astype(np.int64)
    lst = r.buffer(dqo.DQO_BUF_TILE_LIST, np.uint32).astype(np.int64)
    m, nvis, ntiles = dqo.dqo_get_counts(r.ctx)
    assert ntiles == ntx * nty and nvis == vis.sum() and m == list_ref.size
    empty = ranges_ref[:, 0] == ranges_ref[:, 1]
    assert np.array_equal(ranges[~empty], ranges_ref[~empty])
    assert np.all(ranges[empty, 0] == ranges[empty, 1])
    assert np.array_equal(lst, list_ref)
    # depth order: visible Gaussians by (z bits, index), culled ones after
    order = r.buffer(dqo.DQO_BUF_DEPTH_ORDER, np.uint32).astype(np.int64)
    key = np.where(vis, zbits, np.uint32(0xFFFFFFFF))
    assert np.array_equal(order, np.lexsort((np.arange(len(key)), key)))


def _near_ties(ref):
    """Non-empty pixels whose FP64 top-2 object weight margin is within ID_MARGIN."""
    return int(((ref["id_margin"] <= ID_MARGIN) & (ref["id_map"] != -1)).sum())


def _forward_parity(g, cam, t, nobj, st_kw=None, id_check=True, max_flagged=0.01, max_ties=1e-4, report=None):
    st_kw = st_kw or {}
    r = Render(g, cam, nobj, t, **st_kw)
    out = r.forward()
    st_o = oracle_settings(nobj, **{k: v for k, v in st_kw.items() if k not in ("batch",)})
    ref = oracle.render(g, cam, st_o, t)
    ok = ref["amb"] == 0
    assert 1 - ok.mean() <= max_flagged, 1 - ok.mean()
    _img_compare(out, ref, ok)
    H, W = cam["height"], cam["width"]
    Tf = r.buffer(dqo.DQO_BUF_T_FINAL, np.float32).reshape(H, W)
    last = r.last_blended()
    assert np.abs(Tf - ref["T_final"])[ok].max(initial=0) < TOL_IMG
    assert np.array_equal(last[ok], ref["last"][ok])
    if id_check:
        # an empty pixel (id -1) is certain; otherwise the top-2 weight margin must exceed 1e-5
        sure = ok & ((ref["id_margin"] > ID_MARGIN) | (ref["id_map"] == -1))
        assert np.array_equal(out["id_map"][sure], ref["id_map"][sure])
        ties = _near_ties(ref)
        assert ties <= max(max_ties * H * W, 2), (ties, H * W)
        if report is not None:
            report["near_ties"] = ties
    else:
        out = {k: v for k, v in out.items() if k != "id_map"}
    # every flagged pixel is one of the outcomes of its uncertain decisions
    check_flagged_pixels(g, cam, st_o, t, ref, out, Tf, last, report=report)
    if t is not None:
        np.testing.assert_allclose(out["loss"], ref["loss"], rtol=2e-5, atol=1e-6)
    return r, out, ref


def test_forward_parity_config1():
    g, cam, t = tiny_case()
    r, out, ref = _forward_parity(g, cam, t, 4)
    assert out["alpha"].max() > 0.9 and (out["id_map"] >= 0).mean() > 0.3
    r.close()


@pytest.mark.parametrize("tile,batch", [((8, 32), 64), ((32, 8), 128), ((16, 16), 32)])
def test_forward_parity_tile_shapes_ragged(tile, batch):
    g, cam, t = tiny_case(seed=1011, width=333, height=251)
    r, _, _ = _forward_parity(g, cam, t, 4, dict(tile_w=tile[0], tile_h=tile[1], batch=batch))
    r.close()


def test_forward_parity_many_objects_per_tile_and_og_filter():
    # 40 objects, half the Gaussians transparent: the id map needs several slot rounds
    g, cam, t = tiny_case(seed=1021, n=3000, n_objects=40, og_fraction=0.5, width=160, height=120, f=150.0)
    r, out, ref = _forward_parity(g, cam, t, 40)
    r.close()
    r, out, ref = _forward_parity(g, cam, t, 40, dict(og_filter=0, bg=(0.2, 0.4, 0.1), lambda_ins=0.3))
    r.close()


def test_forward_without_targets_and_empty_scenes():
    g, cam, _ = tiny_case()
    r, out, ref = _forward_parity(g, cam, None, 4)
    assert np.all(out["ins"] == 0)
    r.close()
    # no Gaussians at all: background, zero alpha, id -1, loss of the empty render
    e = synth.empty_gaussians()
    t = dict(rgb=np.full((48, 64, 3), 0.5, np.float32), depth=np.ones((48, 64), np.float32),
             gt_id=np.zeros((48, 64), np.int32))
    cam2 = synth.tiny_camera(width=64, height=48)
    r, out, ref = _forward_parity(e, cam2, t, 4, dict(bg=(0.1, 0.2, 0.3)))
    assert np.allclose(out["rgb"], [0.1, 0.2, 0.3]) and np.all(out["alpha"] == 0) and np.all(out["id_map"] == -1)
    grads = r.backward()
    assert all(v.size == 0 for v in grads.values())
    r.close()
    # every Gaussian behind the camera
    g2 = dict(g)
    g2["means"] = g["means"] - np.array([0, 0, 10.0], np.float32)
    r, out, ref = _forward_parity(g2, cam, None, 4)
    assert np.all(out["alpha"] == 0)
    assert dqo.dqo_get_counts(r.ctx)[:2] == (0, 0)
    grads = r.backward(dict(rgb=np.ones((240, 320, 3), np.float32)))
    assert all(np.all(v == 0) for v in grads.values())
    r.close()


def test_backward_parity_fused_loss_config1():
    g, cam, t = tiny_case()
    st_o = oracle_settings(4)
    t = condition_targets(g, cam, t, st_o)
    r = Render(g, cam, 4, t)
    r.forward()
    got = r.backward()
    ref = oracle.render_backward(g, cam, st_o, t)
    report = {}
    assert_grads_close(got, ref, report=report)
    r.close()


def test_backward_parity_pixel_grads_linear_functional():
    # upstream gradients for every output channel (alpha and ins included), OG filter on,
    # non-black background
    g, cam, t = tiny_case(seed=1031, og_fraction=0.6)
    rng = synth.rng_for(77)
    H, W = cam["height"], cam["width"]
    dl = rng.standard_normal((H, W, 6)).astype(np.float32)
    st_kw = dict(bg=(0.3, 0.2, 0.5))
    st_o = oracle_settings(4, **st_kw)
    r = Render(g, cam, 4, t, **st_kw)
    r.forward()
    got = r.backward(dict(rgb=np.ascontiguousarray(dl[..., :3]), depth=np.ascontiguousarray(dl[..., 3]),
                          alpha=np.ascontiguousarray(dl[..., 4]), ins=np.ascontiguousarray(dl[..., 5])))
    ref = oracle.render_backward(g, cam, st_o, t, dl=dl.astype(np.float64))
    assert_grads_close(got, ref)
    # the 2D moment record agrees with the oracle's 2D gradients for opacity, colour, depth
    G2 = r.buffer(dqo.DQO_BUF_GRAD2D, np.float32).reshape(-1, 12)
    keep = ref["amb"] == 0
    for gi, ri in ((5, 5), (6, 6), (7, 7), (8, 8), (9, 9)):
        a, b = G2[keep, gi], ref["g2"][keep, ri]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)
    r.close()


def test_backward_accumulates_and_errors():
    g, cam, t = tiny_case(n=500)
    r = Render(g, cam, 4, t)
    # backward before any forward
    with pytest.raises(dqo.DqoError) as e:
        r.backward()
    assert e.value.status == dqo.DQO_ESTATE
    r.forward()
    grads = dqo.alloc_grads(r.n)
    for _ in range(2):
        dqo.dqo_render_backward(r.ctx, r.st, r.gs, r.cs, r.ts, None, dqo.gaussian_grads(grads))
    once = r.backward()
    torch.cuda.synchronize()
    # float atomics add in a run-dependent order: agree to rounding, scaled per tensor
    for k in once:
        acc = grads[k].cpu().numpy().astype(np.float64)
        ref = 2 * once[k].astype(np.float64)
        assert np.abs(acc - ref).max() <= 1e-5 * np.abs(ref).max(), k
    r.close()


def test_invalid_arguments_are_rejected():
    g, cam, t = tiny_case(n=100)
    r = Render(g, cam, 4, t)
    for bad in (dict(tile_w=10, tile_h=10), dict(tile_w=16, tile_h=8), dict(batch=48), dict(batch=512),
                dict(znear=0.0)):
        st = dqo.settings(**bad)
        with pytest.raises(dqo.DqoError) as e:
            dqo.dqo_render_forward(r.ctx, st, r.gs, r.cs, r.ts, dqo.render_out(r.out))
        assert e.value.status == dqo.DQO_EINVAL
    with pytest.raises(dqo.DqoError):
        dqo.dqo_render_forward(r.ctx, r.st, dqo.gaussians(r.g, 0), r.cs, r.ts, dqo.render_out(r.out))
    cam_bad = dqo.camera(dict(cam, width=0))
    with pytest.raises(dqo.DqoError):
        dqo.dqo_render_forward(r.ctx, r.st, r.gs, cam_bad, r.ts, dqo.render_out(r.out))
    r.close()


def test_indoor_keyframe_full_size_parity():
    # The bench workload itself (300k Gaussians, 1200x680, 31 object ids, default settings
    # and launch configuration): every pixel and every Gaussian gradient against the oracle.
    kf = synth.indoor_keyframe(1002)
    g, cam = kf["gaussians"], kf["camera"]
    st_o = oracle_settings(31)
    t = condition_targets(g, cam, synth.raycast_targets(kf), st_o)
    r = Render(g, cam, 31, t)
    out = r.forward()
    m, nvis, _ = dqo.dqo_get_counts(r.ctx)
    assert m > 1_000_000 and nvis > 200_000
    got = r.backward()
    ref = oracle.render(g, cam, st_o, t)
    ok = ref["amb"] == 0
    # flagged pixels (decisions within rounding distance of a threshold) are at most 1%
    assert ok.mean() >= 0.99, ok.mean()
    _img_compare(out, ref, ok)
    H, W = cam["height"], cam["width"]
    Tf = r.buffer(dqo.DQO_BUF_T_FINAL, np.float32).reshape(H, W)
    last = r.last_blended()
    assert np.abs(Tf - ref["T_final"])[ok].max(initial=0) < TOL_IMG
    assert np.array_equal(last[ok], ref["last"][ok])
    sure = ok & ((ref["id_margin"] > ID_MARGIN) | (ref["id_map"] == -1))
    assert np.array_equal(out["id_map"][sure], ref["id_map"][sure])
    # id-map near ties are at most 0.01% of the pixels
    assert _near_ties(ref) <= 1e-4 * H * W, _near_ties(ref)
    # every flagged pixel matches one of the outcomes of its uncertain decisions
    rep_px = {}
    check_flagged_pixels(g, cam, st_o, t, ref, out, Tf, last, report=rep_px)
    np.testing.assert_allclose(out["loss"], ref["loss"], rtol=2e-5, atol=1e-6)
    refb = oracle.render_backward(g, cam, st_o, t)
    report = {}
    assert_grads_close(got, refb, report=report)
    print("flagged pixels", rep_px, "near ties", _near_ties(ref), "gradients", report)
    r.close()


def test_update_masks_eq11():
    # Mask_geo / Mask_rgb of Eq. 11 fused into the blend epilogue, against the oracle
    # (pixels within 1e-4 of a mask threshold or flagged for the render are left out)
    g, cam, t = tiny_case(seed=1041)
    st_kw = dict(theta_alpha=0.6, theta_d=0.1, theta_c=0.1)
    r = Render(g, cam, 4, t, **st_kw)
    r.out["update_mask"] = torch.empty(cam["height"], cam["width"], dtype=torch.uint8, device="cuda")
    out = r.forward()
    ref = oracle.render(g, cam, oracle_settings(4, **st_kw), t)
    ok = (ref["amb"] == 0) & (ref["mask_amb"] == 0)
    assert ok.mean() > 0.97
    assert np.array_equal(out["update_mask"][ok], ref["update_mask"][ok])
    assert (ref["update_mask"] & 1).any() and (ref["update_mask"] & 2).any() and (ref["update_mask"] == 0).any()
    assert np.all(out["update_mask"][t["gt_id"] < 0] == 0)
    r.close()


def test_update_masks_golden_cases():
    # the CUDA path on the cases of tests/golden/eq11_update_masks.txt (Eq. 11, thresholds
    # as printed after it), against the fixture's expected bits
    from golden_cases import eq11_case, read_fixture
    consts, rows = read_fixture("eq11_update_masks.txt")
    st_kw = dict(theta_alpha=consts["theta_alpha"], theta_d=consts["theta_d"], theta_c=consts["theta_c"])
    default = dqo.settings()
    assert abs(default.theta_d - consts["theta_d"]) < 1e-7 and abs(default.theta_c - consts["theta_c"]) < 1e-7
    for a, dd, dc, geo, rgb in rows:
        g, cam, t, (y, x) = eq11_case(a, dd, dc)
        g = {k: v.astype(np.float32) if v.dtype == np.float64 else v for k, v in g.items()}
        r = Render(g, cam, 4, t, **st_kw)
        r.out["update_mask"] = torch.empty(cam["height"], cam["width"], dtype=torch.uint8, device="cuda")
        out = r.forward()
        assert abs(out["ins"][y, x] - a) < 1e-6
        assert out["update_mask"][y, x] == int(geo) | (int(rgb) << 1), (a, dd, dc)
        assert np.all(out["update_mask"][t["gt_id"] < 0] == 0)
        r.close()
