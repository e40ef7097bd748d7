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
