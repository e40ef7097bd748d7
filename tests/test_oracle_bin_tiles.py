"""Pins of the oracle's tile-list builder on hand-made cases: the order is
(tile row-major, FP32 depth bit pattern, Gaussian index)."""
import numpy as np

import oracle


def f32bits(z):
    return np.asarray(z, np.float32).view(np.uint32)


def test_hand_case_order_and_ties():
    # 2x2 tiles.  G0 covers all tiles at z=2; G1 covers tile (1,0) at z=1; G2 covers the left
    # column at z=2 (same depth as G0 -> index order); G3 is invisible.
    rect = np.array([[0, 0, 2, 2], [1, 0, 2, 1], [0, 0, 1, 2], [0, 0, 2, 2]])
    zb = f32bits([2.0, 1.0, 2.0, 0.5])
    vis = np.array([1, 1, 1, 0], np.uint8)
    ranges, lst = oracle.bin_tiles(rect, zb, vis, 2, 2)
    tiles = [list(lst[s:e]) for s, e in ranges]
    assert tiles == [[0, 2], [1, 0], [0, 2], [0]]


def test_depth_bits_order_equals_float_order_for_positive_depths():
    rng = np.random.Generator(np.random.Philox(3))
    z = rng.uniform(0.2, 10.0, 500).astype(np.float32)
    rect = np.tile(np.array([[0, 0, 1, 1]]), (500, 1))
    ranges, lst = oracle.bin_tiles(rect, f32bits(z), np.ones(500, np.uint8), 1, 1)
    assert np.array_equal(lst, np.lexsort((np.arange(500), z)))
