"""Pins of the FP64 dual-quadric oracle (Eq. 1-4, 12 readings) against geometry fixed
outside it: the projected radius of a sphere, the exact silhouette box found by
maximising over the ellipsoid surface, tangent-plane incidence, hand IoU cases,
validity cases, and central finite differences of the loss gradient."""
import numpy as np
from scipy.optimize import minimize

import oracle
from paper_2503_02223_gb300 import synth


def K(f=500.0, cx=320.0, cy=240.0):
    return synth.intrinsics(f, f, cx, cy)


def P_of(K_, vm):
    return (K_ @ vm).reshape(1, 3, 4)


def test_sphere_on_axis_projects_to_closed_form_circle():
    # A sphere of radius r at distance D on the optical axis subtends a cone of half-angle
    # asin(r/D); its image is a circle of radius f r / sqrt(D^2 - r^2) about (cx, cy).
    f, r, D = 500.0, 0.4, 3.0
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    params = np.array([[0.0, 0.0, D, np.log(r), np.log(r), np.log(r), 0.3, -0.2, 0.1]])
    out = oracle.quadric_project(params, P_of(K(f), vm), [0, 1], [0])
    rho = f * r / np.sqrt(D * D - r * r)
    assert out["valid"][0] == 1
    np.testing.assert_allclose(out["bbox"][0], [320 - rho, 240 - rho, 320 + rho, 240 + rho], rtol=1e-13)


def _exact_silhouette_box(centre, axes, R, P):
    # u and v extremes over the ellipsoid surface x = c + R diag(axes) d(theta, phi),
    # refined from the best of many samples by a local optimiser.
    def proj(th_ph):
        th, ph = th_ph
        d = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        x = centre + R @ (axes * d)
        h = P[:, :3] @ x + P[:, 3]
        return h[:2] / h[2]

    th, ph = np.meshgrid(np.linspace(0.01, np.pi - 0.01, 181), np.linspace(0, 2 * np.pi, 361))
    pts = np.stack([th.ravel(), ph.ravel()], 1)
    uv = np.array([proj(p) for p in pts])
    box = []
    for k, sgn in ((0, 1), (1, 1), (0, -1), (1, -1)):
        i0 = np.argmin(sgn * uv[:, k])
        res = minimize(lambda p: sgn * proj(p)[k], pts[i0], method="Nelder-Mead",
                       options=dict(xatol=1e-12, fatol=1e-13, maxiter=4000))
        box.append(sgn * res.fun)
    return np.array(box)


def test_off_axis_ellipsoid_box_equals_silhouette_extremes():
    rng = synth.rng_for(21)
    for trial in range(3):
        params, centres, axes, Rs = synth.random_quadrics(rng, 1)
        vm = synth.sphere_views(rng, 1)[0]
        P = K() @ vm
        out = oracle.quadric_project(params, P.reshape(1, 3, 4), [0, 1], [0])
        assert out["valid"][0] == 1
        ref = _exact_silhouette_box(centres[0], axes[0], Rs[0], P)
        np.testing.assert_allclose(out["bbox"][0], ref, atol=1e-6)


def test_dual_quadric_tangent_planes_and_points():
    # Eq. 1: every plane tangent to the ellipsoid satisfies pi^T Q* pi = 0; the point quadric
    # Q = adj(Q*) vanishes on surface points; Q*_44 = -1 in this parameterisation.
    rng = synth.rng_for(22)
    params, centres, axes, Rs = synth.random_quadrics(rng, 4)
    Q = oracle.quadric_matrix(params)
    for k in range(4):
        np.testing.assert_allclose(Q[k], Q[k].T, atol=1e-15)
        assert abs(Q[k, 3, 3] + 1) < 1e-12
        Qi = np.linalg.inv(Q[k])
        for d in rng.standard_normal((10, 3)):
            d /= np.linalg.norm(d)
            x = centres[k] + Rs[k] @ (axes[k] * d)
            # outward normal of |diag(1/axes) R^T (x - c)| = 1
            nrm = Rs[k] @ ((Rs[k].T @ (x - centres[k])) / axes[k] ** 2)
            pi = np.concatenate([nrm, [-nrm @ x]])
            assert abs(pi @ Q[k] @ pi) < 1e-12 * (pi @ pi)
            xh = np.concatenate([x, [1.0]])
            assert abs(xh @ Qi @ xh) < 1e-10


def test_validity_cases():
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    P = P_of(K(), vm)
    mk = lambda c, a: np.array([[c[0], c[1], c[2], np.log(a), np.log(a), np.log(a), 0, 0, 0]])
    # camera inside the sphere
    assert oracle.quadric_project(mk([0, 0, 0.2], 0.5), P, [0, 1], [0])["valid"][0] == 0
    # behind the camera
    assert oracle.quadric_project(mk([0, 0, -3.0], 0.5), P, [0, 1], [0])["valid"][0] == 0
    # straddling the principal plane (centre in front, surface behind)
    assert oracle.quadric_project(mk([0.8, 0, 0.3], 0.5), P, [0, 1], [0])["valid"][0] == 0
    # well in front
    assert oracle.quadric_project(mk([0.2, 0.1, 3.0], 0.5), P, [0, 1], [0])["valid"][0] == 1
    # invalid pairs are left out of the loss
    l = oracle.quadric_bbox_loss(mk([0, 0, -3.0], 0.5), P, [0, 1], [0], np.array([[0, 0, 10, 10.0]]))
    assert l["loss"][0] == 0 and np.all(l["dparams"] == 0)


def test_iou_hand_cases():
    # obs = predicted box: IoU 1, loss 0.  obs = predicted box shifted by half its width:
    # intersection w h / 2, union 3 w h / 2, IoU 1/3.  Disjoint: loss 1.
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    P = P_of(K(), vm)
    params = np.array([[0.1, -0.2, 3.0, np.log(0.3), np.log(0.2), np.log(0.25), 0.2, 0.4, -0.1]])
    b = oracle.quadric_project(params, P, [0, 1], [0])["bbox"][0]
    w = b[2] - b[0]
    obs = np.stack([b, b + np.array([w / 2, 0, w / 2, 0]), b + np.array([2 * w, 0, 2 * w, 0])])
    q_ptr = [0, 3]
    loss = [oracle.quadric_bbox_loss(params, P, [0, 1], [0], obs[i:i + 1])["loss"][0] for i in range(3)]
    np.testing.assert_allclose(loss, [0.0, 2.0 / 3.0, 1.0], atol=1e-12)
    tot = oracle.quadric_bbox_loss(params, np.repeat(P, 3, 0), q_ptr, [0, 1, 2], obs)["loss"][0]
    np.testing.assert_allclose(tot, 5.0 / 3.0, atol=1e-12)


def test_bbox_loss_gradient_finite_differences():
    q = synth.tiny_quadrics(1001)
    params = q["params"].astype(np.float64)
    out = oracle.quadric_bbox_loss(params, q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"])
    assert np.all(out["loss"] > 0)
    for k in range(params.shape[0]):
        for i in range(9):
            h = 1e-6 * max(1.0, abs(params[k, i]))
            pp = params.copy(); pp[k, i] += h
            pm = params.copy(); pm[k, i] -= h
            lp = oracle.quadric_bbox_loss(pp, q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"])["loss"][k]
            lm = oracle.quadric_bbox_loss(pm, q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"])["loss"][k]
            fd = (lp - lm) / (2 * h)
            an = out["dparams"][k, i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k, i, fd, an)


def test_rotation_vector_small_angle_branch_is_continuous():
    # The series branch (|r|^2 < 1e-8) and the closed form agree at the switch.
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    P = P_of(K(), vm)
    base = np.array([0.1, -0.2, 3.0, np.log(0.3), np.log(0.2), np.log(0.25), 0.0, 0.0, 0.0])
    qs = []
    for t in (0.9e-4, 1.1e-4):
        p = base.copy(); p[6:] = t * np.array([0.6, 0.0, 0.8])
        qs.append(oracle.quadric_matrix(p[None])[0])
    assert np.abs(qs[0] - qs[1]).max() < 1e-4 * 0.3
    obs = np.array([[280.0, 200, 360, 290]])
    for t in (0.5e-4, 2e-4):
        p = base.copy(); p[6:] = t * np.array([0.6, 0.0, 0.8])
        out = oracle.quadric_bbox_loss(p[None], P, [0, 1], [0], obs)
        for i in range(6, 9):
            h = 1e-7
            pp = p.copy(); pp[i] += h
            pm = p.copy(); pm[i] -= h
            fd = (oracle.quadric_bbox_loss(pp[None], P, [0, 1], [0], obs)["loss"][0] -
                  oracle.quadric_bbox_loss(pm[None], P, [0, 1], [0], obs)["loss"][0]) / (2 * h)
            assert abs(fd - out["dparams"][0, i]) < 1e-5 * max(1, abs(fd))
