"""The learned quadric proposal on the tensor cores against the FP64 oracle: features,
canonical labels, the network's forward, its gradients and the Adam step; then a network
trained by the library's own kernels, and what it adds to the plain fit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_02223_gb300 import dqo, proposal, synth

pytestmark = pytest.mark.gpu

LOSS_W = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 0.3, 0.3, 0.3)


FEATURE_FP32_ERR = 1e-6   # FP32 evaluation error of the unit-scale features, before rounding


def _bf16_of_nearby(got, ref):
    """got is the bfloat16 rounding of a value within FEATURE_FP32_ERR of ref (rounding is
    monotone, so that is the interval between the roundings of ref -+ the error)."""
    lo = oracle.round_bf16(ref - FEATURE_FP32_ERR)
    hi = oracle.round_bf16(ref + FEATURE_FP32_ERR)
    return (got >= lo) & (got <= hi)


def _features_case(seed, n, counts=None):
    s = synth.proposal_samples(seed, n)
    d = dqo.to_device({k: s[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")})
    return s, d


def test_features_parity_and_transpose():
    s, d = _features_case(1101, 700)
    rng = np.random.default_rng(0)
    counts = rng.integers(0, 10, 700).astype(np.int32)          # 0 views, fewer, more than 8
    ldt = 704
    X = torch.empty(700, 128, dtype=torch.bfloat16, device="cuda")
    XT = torch.full((128, ldt), 7.0, dtype=torch.bfloat16, device="cuda")
    dqo.dqo_mlp_features(d["P"], d["q_ptr"], d["pair_v"], d["obs_bbox"], torch.from_numpy(counts).cuda(),
                         s["length_scale"], X, XT)
    got = X.float().cpu().numpy().astype(np.float64)
    ref = oracle.mlp_features(s["P"], s["q_ptr"], s["pair_v"], s["obs_bbox"], counts, s["length_scale"])
    ok = _bf16_of_nearby(got, ref)
    assert np.all(ok), np.argwhere(~ok)[:5]
    big = np.abs(ref) > 1e-3
    assert (got == oracle.round_bf16(ref))[big].mean() > 0.99
    assert np.array_equal(XT[:, :700].float().cpu().numpy(), X.float().cpu().numpy().T)
    assert torch.all(XT[:, 700:] == 7.0)      # padding columns untouched
    # empty slots are exactly zero
    for q in range(700):
        assert np.all(got[q, 16 * min(counts[q], 8):] == 0)


def test_canonical_parity():
    rng = synth.rng_for(1102)
    params, _, _, _ = synth.random_quadrics(rng, 1000)
    params[:, 6:] *= rng.uniform(0.1, 1.8, (1000, 1))
    params = params.astype(np.float32)
    got = dqo.dqo_quadric_canonical(torch.from_numpy(params).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.quadric_canonical(params)
    # the same ellipsoid on both sides, always
    Qg, Qr = oracle.quadric_matrix(got), oracle.quadric_matrix(ref)
    assert np.abs(Qg - Qr).max() < 1e-5
    # the parameters themselves wherever the choice of representative is clear
    close = np.abs(got - ref).max(1) < 2e-5
    assert close.mean() > 0.99


def _net_case(seed, n):
    s = synth.proposal_samples(seed, n)
    F = oracle.round_bf16(oracle.mlp_features(s["P"], s["q_ptr"], s["pair_v"], s["obs_bbox"], None,
                                               s["length_scale"]))
    params = synth.mlp_init_params(seed)
    params[16384:16512] = synth.rng_for(seed + 1).normal(0, 0.1, 128)    # non-zero biases
    params[32896:33024] = synth.rng_for(seed + 2).normal(0, 0.1, 128)
    params[35072:35081] = synth.rng_for(seed + 3).normal(0, 0.1, 9)
    labels = oracle.quadric_canonical(s["params_true"]).astype(np.float32)
    return s, F, params, labels


def _state(params):
    st = dqo.MlpState()
    dqo.dqo_mlp_set_params(st, torch.from_numpy(params).cuda())
    return st


def test_forward_parity_with_ragged_tail():
    s, F, params, _ = _net_case(1103, 1000)            # 7 full tiles of 128 + 104 rows
    ctx = dqo.Context()
    st = _state(params)
    X = torch.from_numpy(F.astype(np.float32)).cuda().to(torch.bfloat16)
    assert np.array_equal(X.float().cpu().numpy(), F)  # bf16 values carried exactly
    y = dqo.dqo_mlp_forward(ctx, st, X).cpu().numpy().astype(np.float64)
    ref = oracle.mlp_forward(F, params.astype(np.float64))["y"]
    err = np.abs(y - ref)
    assert err.max() < 2e-3, err.max()                  # a hidden activation rounded the other way
    assert np.median(err) < 1e-5
    assert not dqo.dqo_mlp_check(ctx)
    # parameters round-trip
    assert np.array_equal(dqo.dqo_mlp_get_params(st).cpu().numpy(), params)
    ctx.close()


def _block_rel(g, r):
    out = {}
    for k, (o, sh) in oracle.MLP_LAYOUT.items():
        m = int(np.prod(sh))
        out[k] = np.linalg.norm(g[o:o + m] - r[o:o + m]) / max(np.linalg.norm(r[o:o + m]), 1e-30)
    return out


def test_gradients_parity():
    s, F, params, labels = _net_case(1104, 512)
    ctx = dqo.Context()
    st = _state(params)
    X = torch.from_numpy(F.astype(np.float32)).cuda().to(torch.bfloat16)
    g, loss = dqo.dqo_mlp_gradients(ctx, st, X, torch.from_numpy(labels).cuda(), LOSS_W)
    g = g.cpu().numpy().astype(np.float64)
    ref, ref_loss = oracle.mlp_backward(F, labels, np.array(LOSS_W), params.astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 1e-4 * ref_loss
    rel = _block_rel(g, ref)
    assert all(v < 2e-3 for v in rel.values()), rel
    # rows of every weight block (per output unit)
    for k in ("W1", "W2"):
        o, sh = oracle.MLP_LAYOUT[k]
        G = g[o:o + sh[0] * sh[1]].reshape(sh)
        R = ref[o:o + sh[0] * sh[1]].reshape(sh)
        rn = np.linalg.norm(R, axis=1)
        e = np.linalg.norm(G - R, axis=1)
        assert np.all(e <= 5e-3 * np.maximum(rn, 1e-2 * rn.max())), (k, float((e / np.maximum(rn, 1e-2 * rn.max())).max()))
    assert np.all(g[33024 + 9 * 128:35072] == 0) and np.all(g[35072 + 9:] == 0)
    # a second call gives the same result bit for bit (the tiles are summed in tile order)
    g2, _ = dqo.dqo_mlp_gradients(ctx, st, X, torch.from_numpy(labels).cuda(), LOSS_W)
    assert np.array_equal(g2.cpu().numpy().astype(np.float64), g)
    ctx.close()


def test_train_step_parity():
    s, F, params, labels = _net_case(1105, 256)
    ctx = dqo.Context()
    st = _state(params)
    X = torch.from_numpy(F.astype(np.float32)).cuda().to(torch.bfloat16)
    lab = torch.from_numpy(labels).cuda()
    lr = 1e-3
    hp = dqo.mlp_hparams(lr=lr, lr_final=lr, total_steps=0, loss_w=LOSS_W)
    loss = torch.zeros(1, device="cuda")
    dqo.dqo_mlp_train_step(ctx, st, hp, X, lab, loss)
    p1 = dqo.dqo_mlp_get_params(st).cpu().numpy().astype(np.float64)
    g, ref_loss = oracle.mlp_backward(F, labels, np.array(LOSS_W), params.astype(np.float64))
    r1, m, v = oracle.mlp_adam(params.astype(np.float64), g, 0, 0, 1, lr)
    assert abs(loss.item() - ref_loss) <= 1e-4 * ref_loss
    # first Adam step = lr * g / (|g| + eps): compare where the gradient is clear of zero
    clear = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.abs(p1 - r1)[clear].max() <= 1e-6 + 1e-3 * lr
    assert np.abs(p1 - r1).max() <= 2.0 * lr + 1e-6
    # the second step uses the updated BF16 copies and the advanced step count
    dqo.dqo_mlp_train_step(ctx, st, hp, X, lab, loss)
    g2, loss2 = oracle.mlp_backward(F, labels, np.array(LOSS_W), r1)
    assert abs(loss.item() - loss2) <= 2e-3 * loss2
    assert loss2 < ref_loss
    ctx.close()


def test_train_steps_equal_single_steps():
    """One launch of k steps = k single-step calls on the same batches: the parameters
    bitwise (every sum is in a fixed order), the per-step losses up to the order of the
    loss sum's atomic additions."""
    s, F, params, labels = _net_case(1107, 3 * 512)
    ctx = dqo.Context()
    X = torch.from_numpy(F.astype(np.float32)).cuda().to(torch.bfloat16)
    lab = torch.from_numpy(labels).cuda()
    hp = dqo.mlp_hparams(lr=1e-3, lr_final=1e-4, total_steps=5, loss_w=LOSS_W)
    st1 = _state(params)
    loss1 = torch.zeros(3, device="cuda")
    for k in range(3):
        dqo.dqo_mlp_train_step(ctx, st1, hp, X[k * 512:(k + 1) * 512], lab[k * 512:(k + 1) * 512], loss1[k:k + 1])
    st3 = _state(params)
    loss3 = torch.zeros(3, device="cuda")
    dqo.dqo_mlp_train_steps(ctx, st3, hp, X, lab, 512, loss3)
    p1, p3 = dqo.dqo_mlp_get_params(st1).cpu().numpy(), dqo.dqo_mlp_get_params(st3).cpu().numpy()
    assert np.array_equal(p1, p3)
    assert torch.allclose(loss1, loss3, rtol=1e-6, atol=0)
    # the steps continue the schedule: a fourth step from either state agrees too
    dqo.dqo_mlp_train_step(ctx, st1, hp, X[:512], lab[:512])
    dqo.dqo_mlp_train_steps(ctx, st3, hp, X[:512], lab[:512], 512)
    assert np.array_equal(dqo.dqo_mlp_get_params(st1).cpu().numpy(), dqo.dqo_mlp_get_params(st3).cpu().numpy())
    assert not dqo.dqo_mlp_check(ctx)
    ctx.close()


def test_gradients_parity_more_tiles_than_sms():
    """160 tiles of 128 samples: more tiles than the GPU has SMs, so CTAs take several tiles
    of the step (and the gradient still sums the tiles in tile order)."""
    n = 160 * 128
    s, F, params, labels = _net_case(1108, n)
    ctx = dqo.Context()
    st = _state(params)
    X = torch.from_numpy(F.astype(np.float32)).cuda().to(torch.bfloat16)
    g, loss = dqo.dqo_mlp_gradients(ctx, st, X, torch.from_numpy(labels).cuda(), LOSS_W)
    g = g.cpu().numpy().astype(np.float64)
    ref, ref_loss = oracle.mlp_backward(F, labels, np.array(LOSS_W), params.astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 1e-4 * ref_loss
    rel = _block_rel(g, ref)
    assert all(v < 2e-3 for v in rel.values()), rel
    g2, _ = dqo.dqo_mlp_gradients(ctx, st, X, torch.from_numpy(labels).cuda(), LOSS_W)
    assert np.array_equal(g2.cpu().numpy().astype(np.float64), g)      # same sums in the same order
    assert not dqo.dqo_mlp_check(ctx)
    ctx.close()


def test_invalid_arguments():
    ctx = dqo.Context()
    st = dqo.MlpState()
    X = torch.zeros(100, 128, dtype=torch.bfloat16, device="cuda")       # not a multiple of 128
    with pytest.raises(dqo.DqoError):
        dqo.dqo_mlp_gradients(ctx, st, X, torch.zeros(100, 9, device="cuda"), LOSS_W)
    hp = dqo.mlp_hparams(lr=1e-3, lr_final=1e-3, total_steps=0, loss_w=LOSS_W)
    with pytest.raises(dqo.DqoError):                                      # batch not a multiple of 128
        dqo.dqo_mlp_train_steps(ctx, st, hp, torch.zeros(200, 128, dtype=torch.bfloat16, device="cuda"),
                                torch.zeros(200, 9, device="cuda"), 100)
    with pytest.raises(ValueError):                                        # not a whole number of batches
        dqo.dqo_mlp_train_steps(ctx, st, hp, torch.zeros(300, 128, dtype=torch.bfloat16, device="cuda"),
                                torch.zeros(300, 9, device="cuda"), 128)
    with pytest.raises(dqo.DqoError):
        dqo.dqo_mlp_features(torch.zeros(1, 12, device="cuda"), torch.zeros(2, dtype=torch.int32, device="cuda"),
                             torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, 4, device="cuda"),
                             None, 0.0)
    ctx.close()


# ----------------------------------------------------------------------------- trained network

N_TRAIN = 1 << 18
N_EVAL = 4096


@pytest.fixture(scope="module")
def trained():
    ctx = dqo.Context()
    s = synth.proposal_samples(1106, N_TRAIN)
    d = dqo.to_device({k: s[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")})
    labels, ok = proposal.make_labels(ctx, d)
    assert ok.float().mean().item() > 0.999
    st = dqo.MlpState()
    dqo.dqo_mlp_set_params(st, torch.from_numpy(synth.mlp_init_params(1106)).cuda())
    tr = proposal.Trainer(ctx, st, d, labels, epochs=40, length_scale=s["length_scale"], lr=2e-3, lr_final=1e-5,
                          loss_w=LOSS_W)
    hist = [tr.epoch() for _ in range(40)]
    torch.cuda.synchronize()
    assert not dqo.dqo_mlp_check(ctx)
    yield ctx, st, hist, s["length_scale"]
    ctx.close()


def _centre_err(p, ref):
    return np.linalg.norm(p[:, :3] - ref[:, :3], axis=1)


def test_training_lowers_the_loss(trained):
    # the floor is set by the rotation term: where two semi-axes are close the canonical
    # rotation vector jumps, which no smooth proposal can follow
    _, _, hist, _ = trained
    assert hist[-1] < 0.5 * hist[0], hist[::8]
    assert hist[-1] <= min(hist[:-1]) * 1.01


def test_learned_proposal_gains_two_view_fits(trained):
    """With 2 views the Eq. 1 system (8 tangent planes, 9 unknowns) has no solution, so the
    plain fit returns nothing; the network's proposal refined on the same 2 views gives
    each quadric an estimate.  Errors against the FP64 oracle's plain fit on all 8 views."""
    ctx, st, _, scale = trained
    ev = synth.proposal_samples(1107, N_EVAL)
    ref = oracle.quadric_fit(ev["P"], ev["q_ptr"], ev["pair_v"], ev["obs_bbox"], iters=100)
    assert ref["ok"].mean() > 0.999
    two = synth.subset_views(ev, 2)
    d2 = dqo.to_device({k: two[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")})
    plain = proposal.fit(ctx, d2)
    assert plain["ok"].sum().item() == 0
    prop = proposal.propose(ctx, st, d2, length_scale=scale)
    refined = proposal.fit(ctx, d2, start=prop)
    p = refined["params"].cpu().numpy().astype(np.float64)
    e_prop = _centre_err(prop.cpu().numpy().astype(np.float64), ref["params"])
    e = _centre_err(p, ref["params"])
    print(f"2 views: proposal centre error median {np.median(e_prop):.3f} m, after refinement "
          f"{np.median(e):.3f} m (p90 {np.percentile(e, 90):.3f})")
    assert np.median(e) < 0.05 and np.median(e) < 0.5 * np.median(e_prop)
    # the refined quadrics explain the 6 views they never saw better than the bare proposal
    held = oracle.quadric_bbox_loss(p, ev["P"], ev["q_ptr"], ev["pair_v"], ev["obs_bbox"])["loss"]
    held_p = oracle.quadric_bbox_loss(prop.cpu().numpy().astype(np.float64), ev["P"], ev["q_ptr"], ev["pair_v"],
                                      ev["obs_bbox"])["loss"]
    assert np.mean(held) < np.mean(held_p)


def test_learned_proposal_against_plain_fit_at_three_views(trained):
    """With 3 views both methods run.  With boxes of 2 px noise the Eq. 1 initialisation is
    close to the optimum and the plain fit is the more accurate one (it is the fallback and
    the judge); the refined proposal stays within a factor of it.  The test pins that
    order, so a change of either side shows here."""
    ctx, st, _, scale = trained
    ev = synth.proposal_samples(1108, N_EVAL)
    ref = oracle.quadric_fit(ev["P"], ev["q_ptr"], ev["pair_v"], ev["obs_bbox"], iters=100)
    three = synth.subset_views(ev, 3)
    d3 = dqo.to_device({k: three[k] for k in ("P", "q_ptr", "pair_v", "obs_bbox")})
    plain = proposal.fit(ctx, d3)
    prop = proposal.propose(ctx, st, d3, length_scale=scale)
    refined = proposal.fit(ctx, d3, start=prop)
    ok = plain["ok"].cpu().numpy() > 0
    e_plain = _centre_err(plain["params"].cpu().numpy().astype(np.float64), ref["params"])[ok]
    e_learn = _centre_err(refined["params"].cpu().numpy().astype(np.float64), ref["params"])[ok]
    print(f"3 views: plain centre error median {np.median(e_plain):.4f} m, learned+refined {np.median(e_learn):.4f} m")
    assert np.median(e_plain) <= np.median(e_learn) < 2.0 * np.median(e_plain)


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    import time
    ctx = dqo.Context()
    t0 = time.perf_counter()
    status = dqo.dqo_wait_probe(ctx)
    dt = time.perf_counter() - t0
    assert status == dqo.DQO_ETIMEOUT
    assert 0.5 < dt < 30.0
    # the tensor-core path still works on the same context
    s, F, params, _ = _net_case(1109, 256)
    st = _state(params)
    X = torch.from_numpy(F.astype(np.float32)).cuda().to(torch.bfloat16)
    y = dqo.dqo_mlp_forward(ctx, st, X).cpu().numpy().astype(np.float64)
    ref = oracle.mlp_forward(F, params.astype(np.float64))["y"]
    assert np.abs(y - ref).max() < 2e-3
    assert not dqo.dqo_mlp_check(ctx)
    ctx.close()
