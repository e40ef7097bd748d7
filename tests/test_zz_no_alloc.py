"""The allocation-free depth order (dqo_depth_order_noalloc) against numpy's stable sort
and against the depth order the forward render computes with its own workspace.

dqo_depth_order_noalloc exists for callers that cannot allocate device memory while they
run (a real-time loop that must not take cudaMalloc's implicit synchronisation, a plugin
whose host framework owns the device memory, a fixed memory budget); its scratch is a
fixed array inside the library.  Every call shares that array and it keeps the previous
call's contents, so each case runs twice in a row.  This file is collected last so that,
if it fails, a run that stops at the first failure has already run every other test."""
import numpy as np
import pytest
import torch

from gpu_util import Render, tiny_case
from paper_2503_02223_gb300 import dqo, synth

pytestmark = pytest.mark.gpu


def _forward_keys_and_order(g, cam, nobj):
    r = Render(g, cam, nobj, None)
    r.forward()
    P = r.proj()
    rect = r.buffer(dqo.DQO_BUF_RECT, np.uint16).reshape(-1, 4)
    vis = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
    keys = np.where(vis, P[1, :, 2].copy().view(np.uint32), np.uint32(0xFFFFFFFF))
    order = r.buffer(dqo.DQO_BUF_DEPTH_ORDER, np.uint32)
    r.close()
    return keys, order


def _noalloc_twice(keys: np.ndarray):
    """Two calls in a row on the same keys; returns both orders after checking the status."""
    d_keys = torch.from_numpy(keys.view(np.int32)).cuda()
    outs = []
    for call in range(2):
        order = torch.full_like(d_keys, -7)
        status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        dqo.dqo_depth_order_noalloc(d_keys, order, status)
        torch.cuda.synchronize()
        assert status.item() == 0, f"call {call}: a sort wait gave up"
        outs.append(order.cpu().numpy().view(np.uint32).astype(np.int64))
    return outs


@pytest.mark.parametrize("case", ["tiny", "indoor"])
def test_noalloc_depth_order_matches_lexsort_and_forward_twice(case):
    if case == "tiny":
        g, cam, _ = tiny_case()
        # push some Gaussians behind the near plane so culled keys are present
        g = dict(g)
        g["means"] = g["means"].copy()
        g["means"][::7, 2] -= 5.0
        keys, ref = _forward_keys_and_order(g, cam, 4)
    else:
        kf = synth.indoor_keyframe(1002)
        keys, ref = _forward_keys_and_order(kf["gaussians"], kf["camera"], 31)
    expect = np.lexsort((np.arange(keys.size), keys))
    for call, got in enumerate(_noalloc_twice(keys)):
        assert np.array_equal(got, expect), f"call {call}"
        assert np.array_equal(got, ref.astype(np.int64)), f"call {call}"


@pytest.mark.parametrize("n", [1, 2, 622591, 1 << 20])
def test_noalloc_random_keys_with_duplicates_and_culled(n):
    # n = 1: the single-key path; 622591: just under 152 x 4096 keys, the most CTAs of the
    # 2048-key tiles on this GPU; 2^20: the largest size, 4096-key tiles
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    keys[rng.random(n) < 0.1] = 0xFFFFFFFF                        # culled Gaussians
    dup = rng.random(n) < 0.3
    keys[dup] = keys[rng.integers(0, n, int(dup.sum()))]           # duplicated depths
    keys[rng.random(n) < 0.05] = 0
    expect = np.argsort(keys, kind="stable")
    for call, got in enumerate(_noalloc_twice(keys)):
        assert np.array_equal(got, expect), f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = dqo.load()
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    assert lib.dqo_depth_order_noalloc(buf.data_ptr(), (1 << 20) + 1, buf.data_ptr(), None, None) == dqo.DQO_EINVAL
    assert lib.dqo_depth_order_noalloc(None, 5, None, None, None) == dqo.DQO_EINVAL
    assert lib.dqo_depth_order_noalloc(None, -1, None, None, None) == dqo.DQO_EINVAL
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    assert lib.dqo_depth_order_noalloc(None, 0, None, status.data_ptr(), None) == dqo.DQO_OK
    torch.cuda.synchronize()
    assert status.item() == 0
