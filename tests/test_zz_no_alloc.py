"""The allocation-free depth order (dqo_depth_order_noalloc) against the depth order the
forward render computes with its own workspace.

dqo_depth_order_noalloc exists for callers that cannot allocate device memory while they
run (a real-time loop that must not take cudaMalloc's implicit synchronisation, a plugin
whose host framework owns the device memory, a fixed memory budget); its scratch is a
fixed array inside the library.  This file is collected last so that, if it fails, a run
that stops at the first failure has already run every other test."""
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


@pytest.mark.parametrize("case", ["tiny", "indoor"])
def test_noalloc_depth_order_matches_forward_twice(case):
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
    d_keys = torch.from_numpy(keys.view(np.int32)).cuda()
    for call in range(2):   # the shared scratch keeps the previous call's contents
        order = torch.full_like(d_keys, -7)
        dqo.dqo_depth_order_noalloc(d_keys, order)
        torch.cuda.synchronize()
        got = order.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref), f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = dqo.load()
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    assert lib.dqo_depth_order_noalloc(buf.data_ptr(), (1 << 20) + 1, buf.data_ptr(), None) == dqo.DQO_EINVAL
    assert lib.dqo_depth_order_noalloc(None, 5, None, None) == dqo.DQO_EINVAL
    assert lib.dqo_depth_order_noalloc(None, 0, None, None) == dqo.DQO_OK
