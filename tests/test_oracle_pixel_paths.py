"""Pins of the oracle's per-pixel entry points against its full render, and of the
re-rendering with decisions taken the other way against renders whose settings take
that decision the other way by themselves.

* oracle_render_pixels restates the render at chosen pixels: it must give the full
  render's values bit for bit (ragged tiny image, every pixel; indoor keyframe, sampled
  pixels of three row bands).
* oracle_render's row window renders those rows exactly as the full image does.
* oracle_render_alternatives: alternative 0 is the render; a pixel whose alpha skip,
  clamp or stop decision lies within rounding distance of its threshold gets the outcome
  of the other decision, which equals the render with the threshold moved past the
  value (Sec. IV's 3DGS constants as configurable settings).
* oracle_render_backward skips pixels with a zero upstream gradient: the gradient stays
  linear in the upstream gradient over disjoint pixel sets and over channels, and the
  fused-loss gradient with unlabelled pixels equals that of its own per-pixel dl.
"""
import numpy as np

import oracle
from paper_2503_02223_gb300 import synth

KEYS = ("rgb", "depth", "alpha", "ins", "id_map", "T_final", "n_contrib", "id_margin")


def _tiny_targets(g_seed, cam, st, n=2000):
    tgt = oracle.render(synth.tiny_gaussians(g_seed, n=n), cam, st)
    return dict(rgb=tgt["rgb"], depth=tgt["depth"], gt_id=tgt["id_map"])


def test_render_pixels_equals_render_on_every_pixel_of_a_ragged_image():
    g = synth.tiny_gaussians(1011)
    cam = synth.tiny_camera(width=333, height=251)
    st = oracle.settings(num_objects=4)
    t = _tiny_targets(1012, cam, st)
    full = oracle.render(g, cam, st, t)
    yy, xx = np.mgrid[0:251, 0:333]
    pxy = np.stack([xx.ravel(), yy.ravel()], 1)
    px = oracle.render_pixels(g, cam, pxy, st, t["gt_id"])
    for k in KEYS:
        a = full[k].reshape((251 * 333,) + full[k].shape[2:])
        assert np.array_equal(px[k], a), k
    # render_pixels has no colour / depth targets, so only the decision flags compare
    assert np.array_equal(px["amb"], full["amb"].ravel() & 5)
    assert (px["amb"] != 0).any() and (px["alpha"] > 0.5).mean() > 0.2


def test_render_pixels_equals_render_on_sampled_pixels_of_the_indoor_keyframe():
    kf = synth.indoor_keyframe(1002)
    g, cam = kf["gaussians"], kf["camera"]
    st = oracle.settings(num_objects=31)
    gt = synth.raycast_targets(kf)["gt_id"]
    rng = np.random.default_rng(3)
    pxy, ref = [], {k: [] for k in KEYS}
    for y0, y1 in ((0, 16), (336, 352), (672, 680)):      # first, middle and the ragged last tile row
        r = oracle.render(g, cam, st, dict(rgb=np.zeros((680, 1200, 3)), depth=None, gt_id=gt), rows=(y0, y1))
        p = np.stack([rng.integers(0, 1200, 40), rng.integers(y0, y1, 40)], 1)
        pxy.append(p)
        for k in KEYS:
            ref[k].append(r[k][p[:, 1], p[:, 0]])
    pxy = np.concatenate(pxy)
    px = oracle.render_pixels(g, cam, pxy, st, gt)
    for k in KEYS:
        assert np.array_equal(px[k], np.concatenate(ref[k])), k
    assert (px["n_contrib"] > 20).mean() > 0.5


def test_render_row_window_renders_those_rows_as_the_full_image_does():
    g = synth.tiny_gaussians(1021)
    cam = synth.tiny_camera()
    st = oracle.settings(num_objects=4)
    t = _tiny_targets(1022, cam, st)
    full = oracle.render(g, cam, st, t)
    y0, y1 = 37, 101                                        # not tile aligned
    part = oracle.render(g, cam, st, t, rows=(y0, y1))
    for k in KEYS + ("amb", "dl", "update_mask"):
        assert np.array_equal(part[k][y0:y1], full[k][y0:y1]), k
        assert not part[k][:y0].any() and not part[k][y1:].any(), k
    # the losses are the window's share of the full image's per-pixel L1 terms
    HW = cam["width"] * cam["height"]
    lab = t["gt_id"][y0:y1] >= 0
    l_rgb = np.abs(full["rgb"][y0:y1] - t["rgb"][y0:y1]).sum(-1)[lab].sum() / HW
    assert abs(part["loss"][0] - l_rgb) < 1e-12 * max(l_rgb, 1)


def _single_pixel_scene(opacities, depths, W=32, H=32):
    n = len(opacities)
    o = np.asarray(opacities, np.float64)
    return dict(means=np.stack([np.zeros(n), np.zeros(n), np.asarray(depths, np.float64)], 1),
                log_scales=np.full((n, 3), np.log(0.05)), quats=np.tile([1.0, 0, 0, 0], (n, 1)),
                opacity_logit=np.log(o / (1 - o)), rgb=synth.rng_for(4).uniform(0, 1, (n, 3)),
                obj_id=np.arange(n, dtype=np.int32) % 4, flags=np.ones(n, np.uint8)), \
        synth.make_camera(100.0, 100.0, W / 2, H / 2, W, H, np.concatenate([np.eye(3), np.zeros((3, 1))], 1))


def _alt_matches(alt, r, k=0):
    v = np.concatenate([r["rgb"][16, 16], [r["depth"][16, 16], r["alpha"][16, 16], r["ins"][16, 16],
                                           r["T_final"][16, 16]]])
    for a in range(alt["count"][k]):
        if np.array_equal(alt["vals"][k, a], v) and alt["n_contrib"][k, a] == r["n_contrib"][16, 16] \
                and alt["id_map"][k, a] == r["id_map"][16, 16]:
            return a
    return -1


def test_alternatives_take_each_near_threshold_decision_the_other_way():
    # Every Gaussian is centred on pixel (16, 16) (G = 1 there), so alpha = opacity.
    amin = 1.0 / 255.0
    cases = [
        # alpha within 1e-6 of alpha_min: blended; skipped with alpha_min just above it
        ([amin * (1 + 1e-6)], [2.0], dict(alpha_min=amin * (1 + 1e-3))),
        # opacity within 1e-6 above the clamp: clamped; unclamped with the clamp just above it
        ([0.99 * (1 + 1e-6)], [2.0], dict(alpha_clamp=0.99 * (1 + 1e-3))),
        # T (1 - alpha) within 1e-6 of t_stop = 0.05 before the second Gaussian: it blends;
        # the walk stops there with t_stop just above
        ([0.8, 0.75 - 2.5e-7], [2.0, 2.5], dict(t_stop=0.05 * (1 + 1e-3))),
    ]
    for ops, zs, moved in cases:
        g, cam = _single_pixel_scene(ops, zs)
        base_st = dict(num_objects=4, t_stop=0.05 if "t_stop" in moved else 1e-4)
        st = oracle.settings(**base_st)
        r0 = oracle.render(g, cam, st)
        assert r0["amb"][16, 16] & 1, ops
        r1 = oracle.render(g, cam, oracle.settings(**dict(base_st, **moved)))
        assert not np.array_equal(r0["alpha"][16, 16], r1["alpha"][16, 16])
        alt = oracle.render_alternatives(g, cam, [[16, 16]], st)
        assert alt["count"][0] >= 2
        assert _alt_matches(alt, r0) == 0, ops               # alternative 0: the render itself
        assert _alt_matches(alt, r1) > 0, ops                 # the other decision's outcome


def test_alternatives_zero_is_the_render_and_flagged_pixels_get_more():
    g = synth.tiny_gaussians(1031)
    cam = synth.tiny_camera(width=160, height=120, f=150.0)
    st = oracle.settings(num_objects=4)
    full = oracle.render(g, cam, st)
    flagged = np.argwhere(full["amb"] != 0)[:40]
    plain = np.argwhere(full["amb"] == 0)[::997][:20]
    yx = np.concatenate([flagged, plain])
    alt = oracle.render_alternatives(g, cam, yx[:, ::-1], st)
    y, x = yx[:, 0], yx[:, 1]
    v0 = np.concatenate([full["rgb"][y, x], np.stack([full[k][y, x] for k in ("depth", "alpha", "ins", "T_final")],
                                                     1)], 1)
    assert np.array_equal(alt["vals"][:, 0], v0)
    assert np.array_equal(alt["n_contrib"][:, 0], full["n_contrib"][y, x])
    assert np.all(alt["count"][:len(flagged)] >= 2) and np.all(alt["count"][len(flagged):] == 1)


def test_backward_skip_of_zero_gradient_pixels_keeps_it_linear():
    g = synth.tiny_gaussians(1041, n=800)
    cam = synth.tiny_camera(width=96, height=80, f=100.0)
    st = oracle.settings(num_objects=4)
    rng = synth.rng_for(21)
    dl = rng.standard_normal((80, 96, 6))
    win = np.zeros((80, 96, 1))
    win[20:53, 17:70] = 1                                   # not tile aligned
    full = oracle.render_backward(g, cam, st, dl=dl)
    a = oracle.render_backward(g, cam, st, dl=dl * win)
    b = oracle.render_backward(g, cam, st, dl=dl * (1 - win))
    chans = [oracle.render_backward(g, cam, st, dl=dl * (np.arange(6) == c)) for c in range(6)]
    for k in ("means", "log_scales", "quats", "opacity_logit", "rgb", "g2"):
        scale = np.abs(full[k]).max()
        assert np.abs(a[k] + b[k] - full[k]).max() <= 1e-12 * scale, k
        assert np.abs(sum(c[k] for c in chans) - full[k]).max() <= 1e-12 * scale, k
        assert np.abs(a[k]).max() > 0.05 * scale and np.abs(b[k]).max() > 0.05 * scale, k
    # fused losses: unlabelled pixels carry no gradient; the result equals the backward of
    # the render's own per-pixel loss gradient
    t = _tiny_targets(1042, cam, st, n=800)
    t["gt_id"] = np.where(win[..., 0] > 0, t["gt_id"], -1).astype(np.int32)
    fused = oracle.render_backward(g, cam, st, t)
    dl_f = oracle.render(g, cam, st, t)["dl"]
    assert not dl_f[win[..., 0] == 0].any()
    lin = oracle.render_backward(g, cam, st, t, dl=dl_f)
    for k in ("means", "log_scales", "quats", "opacity_logit", "rgb"):
        assert np.abs(fused[k] - lin[k]).max() <= 1e-12 * np.abs(lin[k]).max(), k


def test_last_blended_is_the_tile_list_entry_at_n_contrib():
    # the render's `last` output is the Gaussian at list position n_contrib - 1 of the
    # pixel's tile list, rebuilt here from the projections by the tile-list builder
    g = synth.tiny_gaussians(1051)
    W, H = 333, 251
    cam = synth.tiny_camera(width=W, height=H)
    st = oracle.settings(num_objects=4)
    r = oracle.render(g, cam, st)
    pp = oracle.preprocess(g, cam, st)
    ntx, nty = -(-W // 16), -(-H // 16)
    zbits = pp["z"].astype(np.float32).view(np.uint32)
    ranges, lst = oracle.bin_tiles(pp["rect"], zbits, pp["visible"], ntx, nty)
    yy, xx = np.mgrid[0:H, 0:W]
    tile = (yy // 16) * ntx + xx // 16
    nc = r["n_contrib"]
    expect = np.where(nc > 0, lst[np.clip(ranges[tile, 0] + nc - 1, 0, lst.size - 1)], -1)
    assert np.array_equal(r["last"], expect)
    assert (r["last"] >= 0).mean() > 0.5
