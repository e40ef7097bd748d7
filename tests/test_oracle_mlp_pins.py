"""Pins of the oracle's learned-proposal functions against what fixes them independently:
torch's bfloat16 conversion, camera matrices built from known intrinsics and poses,
projection of the feature ray, FP64 finite differences, torch's Adam, and the quadric
matrix (canonical parameters describe the same ellipsoid)."""
import numpy as np
import torch

import oracle
from paper_2503_02223_gb300 import synth


def test_round_bf16_matches_torch_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000),
                        # exact ties between two bfloat16 neighbours, both parities
                        (256 + np.arange(64) + 0.5) / 256.0 * 2.0 ** rng.integers(-20, 20, 64),
                        np.array([0.0, -0.0, 1e-39, -3e-40, 2 ** -133, 3 * 2 ** -134])]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_bf16(x.astype(np.float64)), ref)


def _camera(rng, skew=True):
    R = synth.random_rotations(rng, 1)[0]
    K = np.array([[rng.uniform(300, 900), rng.uniform(-5, 5) if skew else 0.0, rng.uniform(200, 400)],
                  [0.0, rng.uniform(300, 900), rng.uniform(150, 300)], [0.0, 0.0, 1.0]])
    C = rng.normal(0, 3, 3)
    t = -R @ C
    lam = rng.uniform(0.2, 5.0) * rng.choice([-1.0, 1.0])
    P = lam * K @ np.concatenate([R, t[:, None]], 1)
    return P, K, R, C


def test_features_recover_known_camera_and_ray():
    rng = np.random.default_rng(1)
    nq, nv = 5, 6
    cams = [_camera(rng) for _ in range(nv)]
    P = np.stack([c[0] for c in cams]).reshape(nv, 12)
    q_ptr = np.array([0, 6, 9, 11, 12, 12], np.int32)
    pair_v = np.array([0, 1, 2, 3, 4, 5, 5, 4, 3, 2, 1, 0], np.int32)
    obs = np.stack([np.sort(rng.uniform(0, 600, 2)) for _ in range(24)]).reshape(12, 2, 2)
    obs = np.stack([obs[:, 0, 0], obs[:, 1, 0], obs[:, 0, 1], obs[:, 1, 1]], 1)   # u0 v0 u1 v1
    counts = np.array([8, 2, 8, 8, 8], np.int32)
    scale = 2.5
    F = oracle.mlp_features(P, q_ptr, pair_v, obs, counts, scale).reshape(nq, 8, 16)
    for q in range(nq):
        use = min(q_ptr[q + 1] - q_ptr[q], 8, counts[q])
        assert np.all(F[q, use:] == 0)
        for j in range(use):
            k = q_ptr[q] + j
            Pv, K, R, C = cams[pair_v[k]]
            f = F[q, j]
            np.testing.assert_allclose(f[4:7], R[0], atol=1e-12)
            np.testing.assert_allclose(f[7:10], R[1], atol=1e-12)
            np.testing.assert_allclose(f[13:16] * scale, C, atol=1e-10)
            b = obs[k]
            uc, vc = 0.5 * (b[0] + b[2]), 0.5 * (b[1] + b[3])
            np.testing.assert_allclose(K @ np.array([f[0], f[1], 1.0]), [uc, vc, 1.0], atol=1e-9)
            np.testing.assert_allclose(f[2:4], [(b[2] - b[0]) / (2 * K[0, 0]), (b[3] - b[1]) / (2 * K[1, 1])],
                                       rtol=1e-12)
            # the ray C + s d projects onto the box centre, in front of the camera
            assert abs(np.linalg.norm(f[10:13]) - 1) < 1e-12
            X = np.append(C + 1.7 * f[10:13], 1.0)
            h = Pv @ X
            np.testing.assert_allclose(h[:2] / h[2], [uc, vc], atol=1e-8)
            assert (R @ f[10:13])[2] > 0


def _params(rng, scale=0.1):
    p = rng.normal(0, scale, oracle.MLP_PARAMS)
    p[33024 + 9 * 128:35072] = 0.0   # W3 rows 9..15
    p[35072 + 9:] = 0.0              # b3 9..15
    return p


def test_mlp_forward_matches_torch_linear_layers():
    rng = np.random.default_rng(2)
    p = _params(rng)
    X = rng.standard_normal((7, 128))
    out = oracle.mlp_forward(X, p, round_bf16_points=False)
    L = oracle.MLP_LAYOUT

    def blk(k):
        o, sh = L[k]
        return torch.from_numpy(p[o:o + int(np.prod(sh))].reshape(sh))
    x = torch.from_numpy(X)
    h1 = torch.relu(torch.nn.functional.linear(x, blk("W1"), blk("b1")))
    h2 = torch.relu(torch.nn.functional.linear(h1, blk("W2"), blk("b2")))
    y = torch.nn.functional.linear(h2, blk("W3")[:9], blk("b3")[:9])
    np.testing.assert_allclose(out["y"], y.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out["h2"], h2.numpy(), rtol=1e-12, atol=1e-12)
    # with rounding, weights and activations are bfloat16 values
    r = oracle.mlp_forward(X, p, round_bf16_points=True)
    assert np.array_equal(oracle.round_bf16(r["h1"]), r["h1"])
    assert np.array_equal(oracle.round_bf16(r["h2"]), r["h2"])
    assert np.abs(r["y"] - out["y"]).max() < 0.05 * np.abs(out["y"]).max()


def test_mlp_backward_against_central_differences():
    rng = np.random.default_rng(3)
    p = _params(rng, 0.15)
    X = rng.standard_normal((5, 128))
    lab = rng.standard_normal((5, 9))
    w = np.array([1, 1, 1, 1, 1, 1, 0.3, 0.3, 0.3])
    g, L = oracle.mlp_backward(X, lab, w, p, round_bf16_points=False)
    y = oracle.mlp_forward(X, p, round_bf16_points=False)["y"]
    assert abs(L - float((w * (y - lab) ** 2).sum() / 5)) < 1e-12
    # every block, sampled, and all of b3
    idx = np.concatenate([rng.choice(16384, 40, replace=False), 16384 + rng.choice(128, 10, replace=False),
                          16512 + rng.choice(16384, 40, replace=False), 32896 + rng.choice(128, 10, replace=False),
                          33024 + rng.choice(9 * 128, 40, replace=False), 35072 + np.arange(9)])
    for i in idx:
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (oracle.mlp_backward(X, lab, w, pp, False)[1] - oracle.mlp_backward(X, lab, w, pm, False)[1]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # padding rows of W3 / b3 get no gradient
    assert np.all(g[33024 + 9 * 128:35072] == 0) and np.all(g[35072 + 9:] == 0)


def test_adam_matches_torch_and_cosine_schedule():
    rng = np.random.default_rng(4)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(4)]
    t = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads):
        t.grad = torch.tensor(g)
        opt.step()
        p, m, v = oracle.mlp_adam(p, g, m, v, k + 1, 1e-2)
        np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-14)
    # constant gradient: every step moves by the scheduled learning rate
    lr0, lr1, T = 1e-2, 1e-4, 10
    p, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    for s in range(1, T + 3):
        prev = p.copy()
        p, m, v = oracle.mlp_adam(p, np.ones(1), m, v, s, lr0, lr1, T)
        want = lr1 + 0.5 * (lr0 - lr1) * (1 + np.cos(np.pi * min((s - 1) / T, 1.0)))
        assert abs((prev - p)[0] - want) < 1e-7 * want   # step = lr / (1 + eps)


def test_canonical_parameters_describe_the_same_ellipsoid():
    rng = np.random.default_rng(5)
    params, _, _, _ = synth.random_quadrics(rng, 200)
    params[:, 6:] *= rng.uniform(0.2, 1.7, (200, 1))    # rotation angles across (0, pi)
    can = oracle.quadric_canonical(params)
    np.testing.assert_allclose(oracle.quadric_matrix(can), oracle.quadric_matrix(params), atol=1e-12)
    assert np.all(np.diff(can[:, 3:6], axis=1) <= 0)
    np.testing.assert_allclose(np.sort(can[:, 3:6], 1), np.sort(params[:, 3:6], 1), atol=0)
    ang = np.linalg.norm(can[:, 6:], axis=1)
    assert np.all(ang <= 2 * np.pi / 3 + 1e-9)   # the largest trace of the four is >= 0
    # brute force: no other rotation describing the same ellipsoid has a larger trace
    for k in range(20):
        R = synth.rotvec_to_mat(params[k, 6:][None])[0]
        o = np.argsort(-params[k, 3:6], kind="stable")
        Rs = R[:, o]
        best = max(np.trace(Rs * np.array(s)) for s in
                   ([1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1], [-1, -1, -1], [-1, 1, 1], [1, -1, 1],
                    [1, 1, -1]) if np.linalg.det(Rs * np.array(s)) > 0)
        Rc = synth.rotvec_to_mat(can[k, 6:][None])[0]
        assert abs(np.trace(Rc) - best) < 1e-9
    # idempotent
    np.testing.assert_allclose(oracle.quadric_canonical(can), can, atol=1e-9)
