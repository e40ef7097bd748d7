"""Pins of the FP64 rasterizer oracle against facts fixed outside the oracle itself:
closed-form Gaussian integrals and moments, a numerically differentiated pinhole map,
scipy's quaternion rotation, invariants of alpha compositing, brute force, and
central finite differences of every gradient; each test states the fact it checks.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2503_02223_gb300 import synth


def one_gaussian(mean, log_scales, quat_wxyz, logit, rgb=(0.2, 0.5, 0.9), obj=0, og=1):
    return dict(means=np.array([mean], np.float64), log_scales=np.array([log_scales], np.float64),
                quats=np.array([quat_wxyz], np.float64), opacity_logit=np.array([logit], np.float64),
                rgb=np.array([rgb], np.float64), obj_id=np.array([obj], np.int32),
                flags=np.array([og], np.uint8))


def cam64(W=64, H=64, f=300.0, cx=None, cy=None, vm=None):
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) if vm is None else vm
    return synth.make_camera(f, f, W / 2 if cx is None else cx, H / 2 if cy is None else cy, W, H, vm)


SMOOTH = oracle.settings(num_objects=4, **oracle.SMOOTH)


def test_isotropic_gaussian_integral_and_centre_values():
    # A 3D isotropic Gaussian of std s on the optical axis at depth z projects to an
    # isotropic 2D Gaussian of variance (f s / z)^2 + lowpass; sum over the pixel grid of
    # its opacity o * exp(-r^2 / 2 var) equals o * 2 pi var (Poisson summation error
    # ~exp(-2 pi^2 var) is negligible for var > 9).
    s, z, f = 0.05, 3.0, 300.0
    o_logit = -0.4
    o = 1 / (1 + np.exp(-o_logit))
    g = one_gaussian([0, 0, z], [np.log(s)] * 3, [1, 0, 0, 0], o_logit)
    cam = cam64(96, 96, f)
    r = oracle.render(g, cam, SMOOTH)
    var = (f * s / z) ** 2 + 0.3
    assert var > 9
    assert abs(r["alpha"].sum() - o * 2 * np.pi * var) < 1e-7 * o * 2 * np.pi * var
    # mean projects onto pixel (48, 48): G = 1 there, so C = o rgb, D = o z
    np.testing.assert_allclose(r["rgb"][48, 48], o * np.array([0.2, 0.5, 0.9]), rtol=1e-13)
    np.testing.assert_allclose(r["depth"][48, 48], o * z, rtol=1e-13)
    # single Gaussian: T_final = 1 - alpha
    np.testing.assert_allclose(r["T_final"], 1 - r["alpha"], atol=1e-15)


def test_anisotropic_projection_moments_match_numerical_jacobian():
    # Off-axis rotated anisotropic Gaussian.  The rendered opacity map is o*exp(-q/2) with
    # covariance Sigma' = Jn Sigma Jn^T + 0.3 I; its zeroth moment is o 2 pi sqrt(det Sigma'),
    # its centroid the projected mean and its second moment Sigma' itself.  Jn is obtained
    # by central differences of the pinhole map and Sigma from scipy's rotation.
    f, W, H = 400.0, 200, 180
    cam = cam64(W, H, f, cx=97.0, cy=83.0)
    mean = np.array([0.11, -0.07, 2.2])
    ls = np.log([0.06, 0.025, 0.04])
    q = np.array([0.8, 0.3, -0.4, 0.2])
    g = one_gaussian(mean, ls, q, 0.3)
    r = oracle.render(g, cam, SMOOTH)
    a = r["alpha"]

    def proj(X):
        return np.array([f * X[0] / X[2] + 97.0, f * X[1] / X[2] + 83.0])

    h = 1e-6
    Jn = np.stack([(proj(mean + h * e) - proj(mean - h * e)) / (2 * h) for e in np.eye(3)], 1)
    Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = Rm @ np.diag(np.exp(2 * ls)) @ Rm.T
    S2 = Jn @ Sig @ Jn.T + 0.3 * np.eye(2)
    o = 1 / (1 + np.exp(-0.3))
    assert abs(a.sum() - o * 2 * np.pi * np.sqrt(np.linalg.det(S2))) < 1e-6 * a.sum()
    v, u = np.mgrid[0:H, 0:W]
    cu, cv = (a * u).sum() / a.sum(), (a * v).sum() / a.sum()
    np.testing.assert_allclose([cu, cv], proj(mean), atol=1e-6)
    du, dv = u - cu, v - cv
    M2 = np.array([[(a * du * du).sum(), (a * du * dv).sum()], [(a * du * dv).sum(), (a * dv * dv).sum()]]) / a.sum()
    np.testing.assert_allclose(M2, S2, rtol=1e-5, atol=1e-6)
    pp = oracle.preprocess(g, cam, SMOOTH)
    np.testing.assert_allclose(pp["conic"][0], [np.linalg.inv(S2)[0, 0], np.linalg.inv(S2)[0, 1],
                                               np.linalg.inv(S2)[1, 1]], rtol=1e-7)
    # 3 sigma radius from the largest eigenvalue
    assert pp["radius"][0] == int(np.ceil(9.0 * np.sqrt(np.linalg.eigvalsh(S2).max())))


def test_culling_and_tile_rect():
    cam = cam64(64, 48, 100.0)
    st = oracle.settings(num_objects=4)
    # behind the near plane
    g = one_gaussian([0, 0, 0.1], [np.log(0.01)] * 3, [1, 0, 0, 0], 0.0)
    assert oracle.preprocess(g, cam, st)["visible"][0] == 0
    # far off-screen to the right: its 3 sigma box holds no pixel centre
    g = one_gaussian([5.0, 0, 1.0], [np.log(0.01)] * 3, [1, 0, 0, 0], 0.0)
    assert oracle.preprocess(g, cam, st)["visible"][0] == 0
    # a Gaussian centred at pixel (20.5, 17.25) with radius r covers the tiles holding the
    # pixel centres in [20.5 - r, 20.5 + r] x [17.25 - r, 17.25 + r]
    z = 2.0
    g = one_gaussian([(20.5 - 32) * z / 100, (17.25 - 24) * z / 100, z], [np.log(0.08)] * 3, [1, 0, 0, 0], 0.0)
    pp = oracle.preprocess(g, cam, st)
    r = pp["radius"][0]
    ulo, uhi = int(np.ceil(20.5 - r)), int(np.floor(20.5 + r))
    vlo, vhi = int(np.ceil(17.25 - r)), int(np.floor(17.25 + r))
    ulo, vlo, uhi, vhi = max(ulo, 0), max(vlo, 0), min(uhi, 63), min(vhi, 47)
    assert list(pp["rect"][0]) == [ulo // 16, vlo // 16, uhi // 16 + 1, vhi // 16 + 1]


def _square_tiles(x, y, h, W, H, tw, th):
    """Tile range [tx0, ty0, tx1, ty1) of the pixel centres in [x-h, x+h] x [y-h, y+h]
    (h a scalar or a pair of half-widths); all zeros if it holds none."""
    hx, hy = (h, h) if np.isscalar(h) else h
    ulo, uhi = max(int(np.ceil(x - hx)), 0), min(int(np.floor(x + hx)), W - 1)
    vlo, vhi = max(int(np.ceil(y - hy)), 0), min(int(np.floor(y + hy)), H - 1)
    if ulo > uhi or vlo > vhi:
        return [0, 0, 0, 0]
    return [ulo // tw, vlo // th, uhi // tw + 1, vhi // th + 1]


def _narrowing_scene(seed, n):
    g = synth.tiny_gaussians(seed, n=n)
    g["opacity_logit"] = 2.0 * g["opacity_logit"] - 1.5     # opacities from 0.1% to 90%
    return g


def test_tile_rect_holds_every_blending_pixel_and_is_narrowed_to_the_alpha_min_ellipse():
    """Brute force over the pixel centres of each Gaussian's 3 sigma square: every pixel
    where the FP64 alpha o exp(-q/2) reaches alpha_min lies in a tile of the Gaussian's
    rect, and the rect holds no tile beyond the bounding box of the ellipse
    q <= 2 ln(o / alpha_min) (Sigma' from the conic by numpy's inverse) widened by 0.05 px;
    a Gaussian with o < alpha_min has no tiles.  Low-opacity Gaussians get rects strictly
    inside their 3 sigma squares."""
    W, H = 96, 80
    cam = synth.tiny_camera(width=W, height=H, f=120.0)
    g = _narrowing_scene(1021, 600)
    for tw, th in ((16, 16), (8, 4)):
        st = oracle.settings(num_objects=4, tile_w=tw, tile_h=th)
        pp = oracle.preprocess(g, cam, st)
        narrowed = checked = 0
        for i in range(len(pp["opac"])):
            if pp["conic"][i].any() == 0:
                continue                                          # behind the camera
            x, y = pp["xy"][i]
            a, b, c = pp["conic"][i]
            o, r = pp["opac"][i], int(pp["radius"][i])
            rect = list(pp["rect"][i]) if pp["visible"][i] else [0, 0, 0, 0]
            u = np.arange(max(int(np.ceil(x - r)), 0), min(int(np.floor(x + r)), W - 1) + 1)
            v = np.arange(max(int(np.ceil(y - r)), 0), min(int(np.floor(y + r)), H - 1) + 1)
            if u.size and v.size:
                du, dv = np.meshgrid(u - x, v - y)
                q = a * du * du + 2 * b * du * dv + c * dv * dv
                hit = np.minimum(st.alpha_clamp, o * np.exp(-0.5 * q)) >= st.alpha_min
                for uu, vv in zip(*np.nonzero(hit.T)):
                    tx, ty = u[uu] // tw, v[vv] // th
                    assert rect[0] <= tx < rect[2] and rect[1] <= ty < rect[3], (i, u[uu], v[vv], rect)
                    checked += 1
            T = 2 * np.log(o / st.alpha_min)
            if T < -0.01:
                assert rect == [0, 0, 0, 0], i
                continue
            S = np.linalg.inv(np.array([[a, b], [b, c]]))
            hx, hy = np.sqrt(max(T, 0) * S[0, 0]) + 0.05, np.sqrt(max(T, 0) * S[1, 1]) + 0.05
            box = _square_tiles(x, y, (min(r, hx), min(r, hy)), W, H, tw, th)
            if rect != [0, 0, 0, 0]:
                assert box[0] <= rect[0] and box[1] <= rect[1] and rect[2] <= box[2] and rect[3] <= box[3], \
                    (i, rect, box)
            sq = _square_tiles(x, y, r, W, H, tw, th)
            area = lambda t: max(t[2] - t[0], 0) * max(t[3] - t[1], 0)
            narrowed += area(rect) < area(sq)
        assert checked > 1000 and narrowed > 50, (checked, narrowed)


def test_narrowed_rects_change_no_pixel():
    """A per-pixel brute force in numpy over all Gaussians in (float z bits, index) order,
    with tile membership by the plain 3 sigma square (no narrowing): alpha = min(clamp,
    o exp(-q/2)), skipped below alpha_min, stopping before T (1 - alpha) < t_stop.  The
    oracle's render with its narrowed rects gives the same colour, alpha and T_final."""
    W, H = 48, 40
    cam = synth.tiny_camera(width=W, height=H, f=60.0)
    g = _narrowing_scene(1022, 120)
    st = oracle.settings(num_objects=4)
    pp = oracle.preprocess(g, cam, st)
    ref = oracle.render(g, cam, st)
    zb = pp["z"].astype(np.float32).view(np.uint32)
    order = np.lexsort((np.arange(len(zb)), zb))
    live = [i for i in order if pp["conic"][i].any()]
    sq = {i: _square_tiles(*pp["xy"][i], int(pp["radius"][i]), W, H, st.tile_w, st.tile_h) for i in live}
    assert sum(pp["visible"]) < len(live) or any(
        list(pp["rect"][i]) != sq[i] for i in live if pp["visible"][i])    # the narrowing acts here
    for py in range(H):
        for px in range(W):
            tx, ty = px // st.tile_w, py // st.tile_h
            T, C = 1.0, np.zeros(3)
            for i in live:
                t4 = sq[i]
                if not (t4[0] <= tx < t4[2] and t4[1] <= ty < t4[3]):
                    continue
                a, b, c = pp["conic"][i]
                du, dv = px - pp["xy"][i][0], py - pp["xy"][i][1]
                al = min(st.alpha_clamp, pp["opac"][i] * np.exp(-0.5 * (a * du * du + 2 * b * du * dv + c * dv * dv)))
                if al < st.alpha_min:
                    continue
                if T * (1 - al) < st.t_stop:
                    break
                C += al * T * g["rgb"][i]
                T *= 1 - al
            np.testing.assert_allclose(ref["rgb"][py, px], C + T * np.array(st.bg[:]), atol=1e-12)
            assert abs(ref["T_final"][py, px] - T) < 1e-12
            assert abs(ref["alpha"][py, px] - (1 - T)) < 1e-12


def _two_layer_scene():
    # two overlapping Gaussians at different depths, plus one in another tile
    g = dict(means=np.array([[0.0, 0.0, 2.0], [0.0, 0.0, 3.0], [0.3, 0.2, 2.5]]),
             log_scales=np.log(np.array([[0.03] * 3, [0.05] * 3, [0.02] * 3])),
             quats=np.array([[1.0, 0, 0, 0]] * 3), opacity_logit=np.array([1.0, 2.0, 0.0]),
             rgb=np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]), obj_id=np.array([1, 2, 3], np.int32),
             flags=np.array([1, 1, 1], np.uint8))
    return g


def test_front_to_back_compositing_hand_case():
    # At the common centre pixel: front alpha a1 = o1 G1, back alpha a2 = o2 G2;
    # C = a1 c1 + (1 - a1) a2 c2, D = a1 z1 + (1 - a1) a2 z2.
    g = _two_layer_scene()
    f = 200.0
    cam = cam64(64, 64, f)
    st = oracle.settings(num_objects=4)
    r = oracle.render(g, cam, st)
    o1, o2 = 1 / (1 + np.exp(-1.0)), 1 / (1 + np.exp(-2.0))
    # both on the optical axis: isotropic footprints of variance (f s / z)^2 + 0.3
    var1 = (f * 0.03 / 2.0) ** 2 + 0.3
    var2 = (f * 0.05 / 3.0) ** 2 + 0.3
    for du in (0, 2, 5):
        a1 = min(0.99, o1 * np.exp(-0.5 * du * du / var1))
        a2 = min(0.99, o2 * np.exp(-0.5 * du * du / var2))
        np.testing.assert_allclose(r["rgb"][32, 32 + du], [a1, (1 - a1) * a2, 0.0], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(r["depth"][32, 32 + du], a1 * 2.0 + (1 - a1) * a2 * 3.0, rtol=1e-12)
        np.testing.assert_allclose(r["T_final"][32, 32 + du], (1 - a1) * (1 - a2), rtol=1e-12)
        # id argmax: object 1 weight a1 vs object 2 weight (1 - a1) a2
        assert r["id_map"][32, 32 + du] == (1 if a1 >= (1 - a1) * a2 else 2)


def test_invariants_and_brute_force_config1():
    g = synth.tiny_gaussians(1001)
    cam = synth.tiny_camera()
    st = oracle.settings(num_objects=4, og_filter=0)
    gt = np.zeros((cam["height"], cam["width"]), np.int32)
    tg = dict(rgb=np.zeros((cam["height"], cam["width"], 3)), depth=None, gt_id=gt)
    r = oracle.render(g, cam, st, tg)
    # sum of weights telescopes: A = 1 - T_final; 0 <= A <= 1
    np.testing.assert_allclose(r["alpha"], 1 - r["T_final"], atol=1e-12)
    assert r["alpha"].min() >= 0 and r["alpha"].max() <= 1
    assert r["T_final"].min() >= 1e-4 * (1 - 1e-12)   # stopping keeps T above t_stop
    # per-object weights W_k (ins with og_filter off and gt = k) sum to A; argmax = id map
    Wk = []
    for k in range(4):
        tg["gt_id"] = np.full_like(gt, k)
        Wk.append(oracle.render(g, cam, st, tg)["ins"])
    Wk = np.stack(Wk, 0)
    np.testing.assert_allclose(Wk.sum(0), r["alpha"], atol=1e-12)
    am = np.where(Wk.max(0) > 0, Wk.argmax(0), -1)
    assert np.array_equal(am, r["id_map"])
    assert np.all(r["ins"] <= r["alpha"] + 1e-15)
    # tiled lists and the per-pixel brute force over all Gaussians in (z, index) order agree
    b = oracle.render(g, cam, st, tg, mode=1)
    t = oracle.render(g, cam, st, tg, mode=0)
    for k in ("rgb", "depth", "alpha", "ins", "id_map", "T_final", "n_contrib"):
        assert np.array_equal(b[k], t[k]), k


def test_ragged_image_brute_force_and_opaque_filter():
    g = synth.tiny_gaussians(1003, n=300, og_fraction=0.5)
    cam = synth.tiny_camera(width=70, height=50, f=80.0)
    st = oracle.settings(num_objects=4, og_filter=1)
    gt = synth.rng_for(5).integers(-1, 4, (50, 70)).astype(np.int32)
    tg = dict(rgb=np.zeros((50, 70, 3)), depth=None, gt_id=gt)
    b = oracle.render(g, cam, st, tg, mode=1)
    t = oracle.render(g, cam, st, tg, mode=0)
    for k in ("rgb", "depth", "alpha", "ins", "id_map", "T_final", "n_contrib"):
        assert np.array_equal(b[k], t[k]), k
    # with the filter on, only opaque Gaussians count: ins <= ins without the filter
    t2 = oracle.render(g, cam, oracle.settings(num_objects=4, og_filter=0), tg)
    assert np.all(t["ins"] <= t2["ins"] + 1e-15)
    assert np.any(t["ins"] < t2["ins"] - 1e-6)
    assert np.all(t["ins"][gt < 0] == 0)


def test_losses_are_means_over_labelled_pixels():
    g = synth.tiny_gaussians(1001)
    cam = synth.tiny_camera()
    st = oracle.settings(num_objects=4, lambda_ins=0.7)
    tgt = oracle.render(synth.tiny_gaussians(1002), cam, st)
    tg = dict(rgb=tgt["rgb"], depth=tgt["depth"], gt_id=tgt["id_map"])
    r = oracle.render(g, cam, st, tg)
    lab = tg["gt_id"] >= 0
    HW = cam["width"] * cam["height"]
    l_rgb = np.abs(r["rgb"] - tg["rgb"]).sum(-1)[lab].sum() / HW
    dm = lab & (tg["depth"] > 0)
    l_d = np.abs(r["depth"] - tg["depth"])[dm].sum() / HW
    l_i = np.abs(r["ins"] - 1)[lab].sum() / HW
    np.testing.assert_allclose(r["loss"], [l_rgb, l_d, l_i, l_rgb + l_d + 0.7 * l_i], rtol=1e-12)
    assert l_rgb > 0 and l_d > 0 and l_i > 0


# ----------------------------------------------------------------------------- finite differences

def fd_scene(seed=7, n=64):
    rng = synth.rng_for(seed)
    return dict(means=np.stack([rng.uniform(-0.35, 0.35, n), rng.uniform(-0.35, 0.35, n),
                                rng.uniform(1.6, 2.4, n)], 1),
                log_scales=rng.normal(np.log(0.03), 0.25, (n, 3)),
                quats=rng.standard_normal((n, 4)),
                opacity_logit=rng.normal(-0.5, 0.5, n),
                rgb=rng.uniform(0, 1, (n, 3)),
                obj_id=rng.integers(0, 3, n).astype(np.int32),
                flags=(rng.uniform(0, 1, n) < 0.7).astype(np.uint8))


PARAMS = ("means", "log_scales", "quats", "opacity_logit", "rgb")


def _fd_check(g, cam, st, value_fn, grads, rel=1e-5):
    worst = 0.0
    for key in PARAMS:
        base = np.asarray(g[key], np.float64)
        flat = base.reshape(-1)
        an = np.asarray(grads[key]).reshape(-1)
        scale = np.abs(an).max()
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            gp = dict(g); xp = flat.copy(); xp[i] += h; gp[key] = xp.reshape(base.shape)
            gm = dict(g); xm = flat.copy(); xm[i] -= h; gm[key] = xm.reshape(base.shape)
            fd = (value_fn(gp) - value_fn(gm)) / (2 * h)
            err = abs(fd - an[i]) / max(abs(an[i]), 1e-3 * scale, 1e-12)
            worst = max(worst, err)
            assert err < rel or abs(fd - an[i]) < 5e-8, (key, i, fd, an[i])
    return worst


def test_render_backward_finite_differences_linear_functional():
    # L = sum over pixels of dl . (C, D, A, ins): its gradient from the oracle's adjoint
    # matches central differences of the forward in every parameter.
    g = fd_scene()
    cam = cam64(64, 64, 300.0)
    st = SMOOTH
    rng = synth.rng_for(11)
    gt = rng.integers(-1, 3, (64, 64)).astype(np.int32)
    dl = rng.standard_normal((64, 64, 6))
    tg = dict(rgb=np.zeros((64, 64, 3)), depth=None, gt_id=gt)

    def value(gg):
        r = oracle.render(gg, cam, st, tg)
        return float((dl[..., :3] * r["rgb"]).sum() + (dl[..., 3] * r["depth"]).sum() +
                     (dl[..., 4] * r["alpha"]).sum() + (dl[..., 5] * r["ins"]).sum())

    b = oracle.render_backward(g, cam, st, tg, dl=dl)
    _fd_check(g, cam, st, value, b)


def test_render_backward_finite_differences_fused_loss_with_background():
    # The fused L1 losses (targets kept away from the kinks) with a non-black background.
    g = fd_scene(seed=9)
    cam = cam64(64, 64, 300.0)
    st = oracle.settings(num_objects=4, lambda_ins=0.5, bg=(0.3, 0.1, 0.6), **oracle.SMOOTH)
    rng = synth.rng_for(12)
    tg = dict(rgb=rng.uniform(1.5, 2.0, (64, 64, 3)) * np.where(rng.uniform(0, 1, (64, 64, 1)) < 0.5, 1, -1),
              depth=rng.uniform(5.0, 6.0, (64, 64)) * (rng.uniform(0, 1, (64, 64)) < 0.8),
              gt_id=rng.integers(-1, 3, (64, 64)).astype(np.int32))

    def value(gg):
        return float(oracle.render(gg, cam, st, tg)["loss"][3])

    b = oracle.render_backward(g, cam, st, tg)
    _fd_check(g, cam, st, value, b)


def test_eq11_update_masks_golden_cases():
    # Eq. 11's masks at one labelled pixel for the cases of tests/golden/eq11_update_masks.txt
    # (thresholds theta_d = theta_c = 0.1 as printed after Eq. 11), and the oracle's default
    # thresholds are the printed ones
    from golden_cases import eq11_case, read_fixture
    consts, rows = read_fixture("eq11_update_masks.txt")
    assert oracle.DEFAULTS["theta_d"] == consts["theta_d"] and oracle.DEFAULTS["theta_c"] == consts["theta_c"]
    st = oracle.settings(num_objects=4, theta_d=consts["theta_d"], theta_c=consts["theta_c"],
                         theta_alpha=consts["theta_alpha"])
    for a, dd, dc, geo, rgb in rows:
        g, cam, t, (y, x) = eq11_case(a, dd, dc)
        r = oracle.render(g, cam, st, t)
        assert abs(r["ins"][y, x] - a) < 1e-12            # the case's premise: ins = alpha
        assert r["update_mask"][y, x] == int(geo) | (int(rgb) << 1), (a, dd, dc)
        assert np.all(r["update_mask"][t["gt_id"] < 0] == 0)
