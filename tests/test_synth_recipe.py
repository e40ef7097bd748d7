"""The synthetic workloads are what the design states (sizes, id layout, value
distributions): the generators hold no method arithmetic, so these checks are on their
outputs only."""
import numpy as np

from paper_2503_02223_gb300 import synth


def test_indoor_keyframe_recipe():
    kf = synth.indoor_keyframe(1002)
    g, cam, q = kf["gaussians"], kf["camera"], kf["quadrics"]
    n = g["means"].shape[0]
    assert n == 300_000
    assert (cam["width"], cam["height"], cam["fx"], cam["fy"]) == (1200, 680, 600.0, 600.0)
    ids = g["obj_id"]
    assert set(np.unique(ids)) == set(range(31))                  # walls 0, objects 1..30
    assert (ids > 0).sum() == 235_000 and (ids == 0).sum() == 65_000
    counts = np.bincount(ids, minlength=31)[1:]
    assert counts.min() >= 0.5 * 2000 * 235_000 / (30 * 20_000) and counts.max() <= 2 * 20_000
    assert np.all(g["flags"] == 1)
    obj = ids > 0
    assert abs(g["log_scales"][obj].mean() + 4.5) < 0.01 and abs(g["log_scales"][obj].std() - 0.5) < 0.01
    assert abs(g["opacity_logit"].mean() - 1.5) < 0.01 and abs(g["opacity_logit"].std() - 1.0) < 0.01
    assert g["rgb"].min() >= 0.0 and g["rgb"].max() <= 1.0
    # flattened wall Gaussians: the normal axis 2.3 below the in-plane ones in log scale
    wl = g["log_scales"][~obj]
    assert abs(wl[:, :2].mean() + 3.5) < 0.01 and abs(wl[:, 2].mean() + 5.8) < 0.01
    # 30 quadrics, each seen whole from up to 8 keyframes (an object none of them sees whole
    # has no view), one observed box per (quadric, view)
    assert q["params"].shape == (30, 9) and q["P"].shape == (8, 3, 4)
    per_q = np.diff(q["q_ptr"])
    assert per_q.max() <= 8 and (per_q > 0).sum() >= 25 and q["obs_bbox"].shape == (per_q.sum(), 4)
    assert per_q.sum() == 199
    assert np.all(q["obs_bbox"][:, 2] > q["obs_bbox"][:, 0]) and np.all(q["obs_bbox"][:, 3] > q["obs_bbox"][:, 1])


def test_indoor_targets_cover_the_image():
    kf = synth.indoor_keyframe(1002)
    t = synth.raycast_targets(kf)
    H, W = 680, 1200
    assert t["rgb"].shape == (H, W, 3) and t["depth"].shape == (H, W) and t["gt_id"].shape == (H, W)
    assert t["rgb"].dtype == np.float32 and t["gt_id"].dtype == np.int32
    hit = t["gt_id"] >= 0
    assert hit.mean() > 0.99                                      # inside a closed room
    d = t["depth"][hit]
    assert d.min() > 0.5 and d.max() < 8.0
    assert (t["gt_id"] > 0).mean() > 0.05                          # objects are in view


def test_tiny_case_recipe():
    g = synth.tiny_gaussians(1001, n=20_000)
    assert g["means"].shape == (20_000, 3)
    assert np.abs(g["means"]).max() <= 1.0
    assert abs(g["log_scales"].mean() + 4.0) < 0.02 and abs(g["log_scales"].std() - 0.5) < 0.02
    assert abs(g["opacity_logit"].std() - 1.0) < 0.02
    assert set(np.unique(g["obj_id"])) == {0, 1, 2, 3}
    cam = synth.tiny_camera()
    assert (cam["width"], cam["height"], cam["fx"]) == (320, 240, 300.0)
