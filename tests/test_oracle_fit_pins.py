"""Pins of the oracle's plain multi-view quadric fit (Eq. 1 initialisation + Eq. 12
refinement): exact recovery from exact boxes, the eigen solver against numpy, the
rotation log map against scipy, and the Adam refinement against torch.optim.Adam driving
the oracle's own loss gradient."""
import numpy as np
import torch
from scipy.spatial.transform import Rotation

import oracle
from paper_2503_02223_gb300 import synth


def test_jacobi_eigen_matches_numpy():
    rng = synth.rng_for(41)
    for n in (3, 10):
        M = rng.standard_normal((n, n))
        A = M @ M.T
        w, V = oracle.jacobi_eigen(A)
        order = np.argsort(w)
        np.testing.assert_allclose(w[order], np.linalg.eigvalsh(A), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(A @ V, V * w[None, :], atol=1e-10)
        np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-12)


def test_rotation_log_map_matches_scipy_including_near_pi():
    rng = synth.rng_for(42)
    axes = rng.standard_normal((20, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    angles = np.concatenate([rng.uniform(0, np.pi, 14), [1e-10, 1e-6, np.pi - 1e-3, np.pi - 1e-6, np.pi, 0.0]])
    for a, t in zip(axes, angles):
        R = Rotation.from_rotvec(a * t).as_matrix()
        r = oracle.rot_to_rotvec(R)
        np.testing.assert_allclose(Rotation.from_rotvec(r).as_matrix(), R, atol=1e-9)
        assert np.linalg.norm(r) <= np.pi + 1e-9


def _exact_case(seed, nq=6, nview=5):
    rng = synth.rng_for(seed)
    params, centres, axes, Rs = synth.random_quadrics(rng, nq)
    K = synth.intrinsics(500.0, 500.0, 320.0, 240.0)
    P = np.einsum("ij,njk->nik", K, synth.sphere_views(rng, nq * nview, radius=3.5))
    q_ptr = np.arange(0, nq * nview + 1, nview).astype(np.int32)
    pair_v = np.arange(nq * nview, dtype=np.int32)
    box = oracle.quadric_project(params, P, q_ptr, pair_v)
    assert np.all(box["valid"])
    return params, P, q_ptr, pair_v, box["bbox"]


def test_init_recovers_the_generating_quadric_from_exact_boxes():
    # every edge plane of an exact box is tangent to the quadric, so the 4V x 10 system has
    # the generating Q* as its exact null vector (Eq. 1)
    params, P, q_ptr, pair_v, bbox = _exact_case(43)
    out = oracle.quadric_fit(P, q_ptr, pair_v, bbox, iters=0)
    assert np.all(out["ok"])
    Q = oracle.quadric_matrix(params)
    np.testing.assert_allclose(out["init_Q"], Q, atol=1e-9 * np.abs(Q).max())
    # the decomposed parameters describe the same quadric (up to axis order / sign)
    np.testing.assert_allclose(oracle.quadric_matrix(out["init"]), Q, atol=1e-8 * np.abs(Q).max())
    # and reproduce the boxes: zero loss
    np.testing.assert_allclose(out["loss"], 0.0, atol=1e-9)


def test_refinement_is_adam_on_the_bbox_loss():
    q = synth.tiny_quadrics(1001)
    out = oracle.quadric_fit(q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"], iters=100, lr=1e-2)
    assert np.all(out["ok"])
    for k in range(q["params"].shape[0]):
        views = q["pair_v"][q["q_ptr"][k]:q["q_ptr"][k + 1]]
        obs = q["obs_bbox"][q["q_ptr"][k]:q["q_ptr"][k + 1]]
        p = torch.tensor(out["init"][k], dtype=torch.float64, requires_grad=True)
        opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
        for _ in range(100):
            r = oracle.quadric_bbox_loss(p.detach().numpy()[None], q["P"], [0, len(views)], views, obs)
            opt.zero_grad()
            p.grad = torch.tensor(r["dparams"][0])
            opt.step()
        np.testing.assert_allclose(p.detach().numpy(), out["params"][k], rtol=1e-10, atol=1e-12)
        l0 = oracle.quadric_bbox_loss(out["init"][k][None], q["P"], [0, len(views)], views, obs)["loss"][0]
        assert out["loss"][k] < l0


def test_fit_recovers_truth_from_noisy_boxes():
    # 2 px box noise, 8 views: the refined quadric's boxes sit close to the exact boxes
    params, P, q_ptr, pair_v, bbox = _exact_case(44, nq=4, nview=8)
    noisy = bbox + synth.rng_for(45).normal(0.0, 2.0, bbox.shape)
    out = oracle.quadric_fit(P, q_ptr, pair_v, noisy, iters=100, lr=1e-2)
    assert np.all(out["ok"])
    fit_box = oracle.quadric_project(out["params"], P, q_ptr, pair_v)["bbox"]
    assert np.abs(fit_box - bbox).mean() < 4.0
