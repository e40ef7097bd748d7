"""Readers for the text fixtures under tests/golden/ and the scenes they describe.  Every
expected value in a fixture comes from the paper (cited in the fixture's header); nothing
here computes an expected value."""
import os

import numpy as np

from paper_2503_02223_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_fixture(name: str):
    """(named constants, rows of floats) of a fixture file."""
    consts, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0][0].isalpha():
                consts[parts[0]] = float(parts[1])
            else:
                rows.append([float(x) for x in parts])
    return consts, rows


EQ11_Z, EQ11_RGB, EQ11_SIZE = 3.0, (0.4, 0.5, 0.6), 96


def eq11_case(alpha: float, depth_offset: float, colour_offset: float):
    """One opaque (OG) Gaussian of object 0 on the optical axis at depth EQ11_Z, opacity
    alpha, std 0.05 m; a 96x96 camera whose pixel (48, 48) is the Gaussian's centre (so
    alpha is reached there exactly); targets labelled only at that pixel, with depth and
    red channel offset from the rendered values alpha * z and alpha * rgb."""
    logit = float(np.log(alpha / (1.0 - alpha)))
    g = dict(means=np.array([[0.0, 0.0, EQ11_Z]]), log_scales=np.full((1, 3), np.log(0.05)),
             quats=np.array([[1.0, 0.0, 0.0, 0.0]]), opacity_logit=np.array([logit]),
             rgb=np.array([EQ11_RGB]), obj_id=np.array([0], np.int32), flags=np.array([1], np.uint8))
    n = EQ11_SIZE
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    cam = synth.make_camera(300.0, 300.0, n / 2, n / 2, n, n, vm)
    rgb = np.zeros((n, n, 3), np.float32)
    depth = np.zeros((n, n), np.float32)
    gt = np.full((n, n), -1, np.int32)
    c = n // 2
    rgb[c, c] = np.array(EQ11_RGB) * alpha
    rgb[c, c, 0] += colour_offset
    depth[c, c] = alpha * EQ11_Z + depth_offset
    gt[c, c] = 0
    return g, cam, dict(rgb=rgb, depth=depth, gt_id=gt), (c, c)
