"""Parity of the CUDA dual-quadric kernels (through the C ABI) with the FP64 oracle:
conic and bbox within 1e-3 relative, validity exact, the Eq. 12 loss and its gradient
within 1e-3 relative per quadric."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_02223_gb300 import dqo, synth

pytestmark = pytest.mark.gpu


def _run(q, ctx=None):
    ctx = ctx or dqo.Context()
    d = dqo.to_device({k: q[k] for k in ("params", "P", "q_ptr", "pair_v", "obs_bbox")})
    npairs = q["pair_v"].shape[0]
    nq = q["params"].shape[0]
    conic = torch.zeros(npairs, 6, device="cuda")
    bbox = torch.zeros(npairs, 4, device="cuda")
    valid = torch.zeros(npairs, dtype=torch.uint8, device="cuda")
    loss = torch.zeros(nq, device="cuda")
    dpar = torch.zeros(nq, 9, device="cuda")
    dqo.dqo_quadric_project(ctx, d["params"], d["P"], d["q_ptr"], d["pair_v"], conic, bbox, valid)
    dqo.dqo_quadric_bbox_loss(ctx, d["params"], d["P"], d["q_ptr"], d["pair_v"], d["obs_bbox"], loss, dpar)
    torch.cuda.synchronize()
    return dict(conic=conic.cpu().numpy(), bbox=bbox.cpu().numpy(), valid=valid.cpu().numpy(),
                loss=loss.cpu().numpy(), dparams=dpar.cpu().numpy())


def _check(q, got):
    ref_p = oracle.quadric_project(q["params"], q["P"], q["q_ptr"], q["pair_v"])
    ref_l = oracle.quadric_bbox_loss(q["params"], q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"])
    assert np.array_equal(got["valid"], ref_p["valid"])
    v = ref_p["valid"] > 0
    # conic up to its scale: compare each pair normalised by its largest entry
    sc = np.abs(ref_p["conic"]).max(1, keepdims=True)
    np.testing.assert_allclose(got["conic"] / sc, ref_p["conic"] / sc, atol=1e-5)
    w = (ref_p["bbox"][v, 2:] - ref_p["bbox"][v, :2]).max(1, keepdims=True)
    assert np.all(np.abs(got["bbox"][v] - ref_p["bbox"][v]) <= 1e-3 * np.maximum(w, 1.0))
    np.testing.assert_allclose(got["loss"], ref_l["loss"], rtol=1e-3, atol=1e-5)
    for k in range(q["params"].shape[0]):
        r = ref_l["dparams"][k]
        g = got["dparams"][k]
        assert np.linalg.norm(g - r) <= 1e-3 * max(np.linalg.norm(r), 1e-6), (k, g, r)


def test_quadric_parity_config1():
    q = synth.tiny_quadrics(1001)
    _check(q, _run(q))


def test_quadric_parity_indoor_keyframe():
    kf = synth.indoor_keyframe(1002)
    q = kf["quadrics"]
    _check(q, _run(q))


def test_quadric_parity_many_fits_uneven_views():
    # 512 quadrics with 3..40 views each (batched-fit sizes), small and large rotations
    rng = synth.rng_for(1003)
    nq = 512
    params, centres, axes, Rs = synth.random_quadrics(rng, nq)
    counts = rng.integers(3, 41, nq)
    K = synth.intrinsics(525.0, 525.0, 320.0, 240.0)
    views = synth.sphere_views(rng, int(counts.sum()), radius=3.5)
    P = np.einsum("ij,njk->nik", K, views)
    q_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    pair_v = np.arange(int(counts.sum()), dtype=np.int32)
    obs = np.zeros((pair_v.size, 4))
    ref = oracle.quadric_project(params, P, q_ptr, pair_v)
    obs = ref["bbox"] + rng.normal(0, 2.0, (pair_v.size, 4))
    init = params + np.concatenate([rng.normal(0, 0.05, (nq, 3)), rng.normal(0, 0.1, (nq, 3)),
                                    rng.normal(0, 0.1, (nq, 3))], 1)
    init[:8, 6:] = rng.normal(0, 1e-3, (8, 3))   # near-identity rotations: series branch
    q = dict(params=init.astype(np.float32), P=P.astype(np.float32), q_ptr=q_ptr, pair_v=pair_v,
             obs_bbox=obs.astype(np.float32))
    _check(q, _run(q))


def test_quadric_edge_cases():
    ctx = dqo.Context()
    # no quadrics, no pairs
    q = dict(params=np.zeros((0, 9), np.float32), P=np.zeros((1, 12), np.float32), q_ptr=np.zeros(1, np.int32),
             pair_v=np.zeros(0, np.int32), obs_bbox=np.zeros((0, 4), np.float32))
    got = _run(q, ctx)
    assert got["loss"].size == 0
    # a quadric without views, a camera inside, one behind, one straddling
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    P = (synth.intrinsics(500, 500, 320, 240) @ vm).reshape(1, 12)
    mk = lambda c, a: [c[0], c[1], c[2], np.log(a), np.log(a), np.log(a), 0.1, 0.2, 0.3]
    params = np.array([mk([0, 0, 3], 0.3), mk([0, 0, 0.2], 0.5), mk([0, 0, -3], 0.5), mk([0.8, 0, 0.3], 0.5)],
                      np.float32)
    q = dict(params=params, P=P.astype(np.float32), q_ptr=np.array([0, 0, 1, 2, 3], np.int32),
             pair_v=np.zeros(3, np.int32), obs_bbox=np.tile(np.array([[300, 220, 340, 260]], np.float32), (3, 1)))
    got = _run(q, ctx)
    assert list(got["valid"]) == [0, 0, 0]
    assert np.all(got["loss"] == 0) and np.all(got["dparams"] == 0)
    # invalid arguments
    with pytest.raises(dqo.DqoError):
        d = dqo.to_device(q)
        dqo.dqo_quadric_bbox_loss(ctx, d["params"], d["P"], None, d["pair_v"], d["obs_bbox"])


def _batched_fits(seed=1003, nq=512, lo=3, hi=41, noise=2.0):
    """nq ellipsoids (axes U[0.1,0.5], centres U[-1,1]^3) with U{lo..hi-1} views each on a
    3.5 m sphere, observed boxes = exact boxes + N(0, noise^2)."""
    rng = synth.rng_for(seed)
    params, centres, axes, Rs = synth.random_quadrics(rng, nq)
    counts = rng.integers(lo, hi, nq)
    K = synth.intrinsics(525.0, 525.0, 320.0, 240.0)
    P = np.einsum("ij,njk->nik", K, synth.sphere_views(rng, int(counts.sum()), radius=3.5))
    q_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    pair_v = np.arange(int(counts.sum()), dtype=np.int32)
    box = oracle.quadric_project(params, P, q_ptr, pair_v)["bbox"]
    obs = box + rng.normal(0, noise, box.shape)
    return dict(P=P.astype(np.float32), q_ptr=q_ptr, pair_v=pair_v, obs_bbox=obs.astype(np.float32),
                counts=counts, params_true=params)


def _gpu_fit(q, iters, lr=1e-2):
    ctx = dqo.Context()
    d = dqo.to_device({k: q[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")})
    nq = q["q_ptr"].shape[0] - 1
    init = torch.zeros(nq, 9, device="cuda")
    par = torch.zeros(nq, 9, device="cuda")
    loss = torch.zeros(nq, device="cuda")
    ok = torch.zeros(nq, dtype=torch.uint8, device="cuda")
    dqo.dqo_quadric_fit(ctx, d["P"], d["q_ptr"], d["pair_v"], d["obs_bbox"], iters, lr, init, par, loss, ok)
    torch.cuda.synchronize()
    return dict(init=init.cpu().numpy(), params=par.cpu().numpy(), loss=loss.cpu().numpy(), ok=ok.cpu().numpy())


def _qnorm(params):
    Q = oracle.quadric_matrix(params)
    return Q / -Q[:, 3:4, 3:4]


def _rel_q(pa, pb):
    Qa, Qb = _qnorm(pa), _qnorm(pb)
    return np.linalg.norm((Qa - Qb).reshape(-1, 16), axis=1) / np.linalg.norm(Qb.reshape(-1, 16), axis=1)


def test_quadric_fit_init_parity_512_fits():
    # The Eq. 1 initialisation, single precision on the GPU against the FP64 oracle.  In the
    # normalised frame the null vector of the single-precision normal matrix is within
    # about eps_32 * lambda_max / (lambda_9 - lambda_10) of the FP64 one (measured on this
    # set: median 6e-7, at most 2e-5); the decomposition adds the cancellation of t t^T
    # against the axes (about |t|^2 / a^2 < 100).  Stated tolerance on the normalised Q*:
    # median 1e-5, every quadric 1e-3.
    q = _batched_fits()
    got = _gpu_fit(q, iters=0)
    ref = oracle.quadric_fit(q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"], iters=0)
    assert np.array_equal(got["ok"], ref["ok"]) and ref["ok"].mean() > 0.99
    ok = ref["ok"] > 0
    rel = _rel_q(got["init"][ok].astype(np.float64), ref["init"][ok])
    print("init rel Q*: median %.2e p90 %.2e max %.2e" % (np.median(rel), np.percentile(rel, 90), rel.max()))
    assert np.all(rel < 1e-3), (rel.max(), np.argmax(rel))
    assert np.median(rel) < 1e-5
    # the loss the kernel reports at its own starting point (a view whose box is nearly
    # degenerate moves the loss by more than 1e-3 under the init's rounding)
    idx = np.nonzero(ok)[0]
    sel_v = np.concatenate([np.arange(q["q_ptr"][i], q["q_ptr"][i + 1]) for i in idx])
    at = oracle.quadric_bbox_loss(got["init"][ok].astype(np.float64), q["P"],
                                  np.concatenate([[0], np.cumsum(np.diff(q["q_ptr"])[idx])]).astype(np.int32),
                                  q["pair_v"][sel_v], q["obs_bbox"][sel_v])
    np.testing.assert_allclose(got["loss"][ok], at["loss"], rtol=1e-3, atol=1e-4)


def test_quadric_fit_refinement_parity():
    # 100 Adam steps from the same start, fp32 (GPU) vs fp64 (oracle).  Adam's normalised
    # steps make the end state sensitive: the oracle's own end state moves by ~1e-3
    # (normalised Q*) when its start moves by 1e-7 relative, so the GPU end state must lie
    # within that spread, and the final losses must agree on average within 1%.
    q = _batched_fits(seed=1004, nq=256, lo=4, hi=41)
    got = _gpu_fit(q, iters=100)
    ok = got["ok"] > 0
    assert ok.mean() > 0.99
    start = got["init"].astype(np.float64)
    ref = oracle.quadric_fit(q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"], iters=100, start=start)
    pert = start * (1 + 1e-7 * synth.rng_for(7).standard_normal(start.shape))
    ref_p = oracle.quadric_fit(q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"], iters=100, start=pert)
    rel_gpu = _rel_q(got["params"][ok].astype(np.float64), ref["params"][ok])
    rel_self = _rel_q(ref_p["params"][ok], ref["params"][ok])
    for pct in (50, 90):
        assert np.percentile(rel_gpu, pct) <= 2 * np.percentile(rel_self, pct) + 1e-4, \
            (pct, np.percentile(rel_gpu, pct), np.percentile(rel_self, pct))
    assert abs(got["loss"][ok].mean() - ref["loss"][ok].mean()) <= 1e-2 * ref["loss"][ok].mean()
    # the refinement lowers the loss of the initialisation
    init = _gpu_fit(q, iters=0)
    assert np.mean(got["loss"][ok]) < np.mean(init["loss"][ok])


def test_quadric_fit_edge_cases():
    q = _batched_fits(seed=1005, nq=8, lo=3, hi=5)
    q["q_ptr"][3] = q["q_ptr"][2] + 1        # quadric 2 keeps 1 view (too few), quadric 3 absorbs the rest
    got = _gpu_fit(q, iters=5)
    assert got["ok"][2] == 0 and np.all(got["params"][2] == 0)
    ref = oracle.quadric_fit(q["P"], q["q_ptr"], q["pair_v"], q["obs_bbox"], iters=5)
    assert np.array_equal(got["ok"], ref["ok"])
    ctx = dqo.Context()
    d = dqo.to_device({k: q[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")})
    with pytest.raises(dqo.DqoError):
        dqo.dqo_quadric_fit(ctx, d["P"], d["q_ptr"], d["pair_v"], d["obs_bbox"], -1, 1e-2)
