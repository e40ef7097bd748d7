"""The pair emission's row of pair k in a tile rectangle of width w: floor((k + 1/2) * fl(1/w))
in single precision, truncated, for k < 2^21 (integer division past it).  (k + 1/2) / w lies
at least 1/(2w) from an integer, and the two roundings (of 1/w and of the product) move it
by a relative 2^-23 at most, so the truncation is floor(k / w) whenever k < 2^22.  These
tests check that claim in IEEE single precision (numpy float32, round to nearest like the
kernel's division and multiplication) at the worst cases: k just below and at multiples
of w, across widths up to 4096 tiles and k up to the 2^21 limit."""
import numpy as np


def _rows(k: np.ndarray, w: np.ndarray) -> np.ndarray:
    iw = (np.float32(1.0) / w.astype(np.float32)).astype(np.float32)
    kf = k.astype(np.float32) + np.float32(0.5)              # exact: k < 2^23
    return np.trunc((kf * iw).astype(np.float32)).astype(np.int64)


def test_row_is_floor_division_near_every_multiple():
    rng = np.random.default_rng(7)
    w = np.repeat(np.arange(1, 4097, dtype=np.int64), 64)
    q = rng.integers(0, (1 << 21) // w + 1)
    for d in (-1, 0, 1):                                       # just below, at, just above q * w
        k = np.clip(q * w + d, 0, (1 << 21) - 1)
        assert np.array_equal(_rows(k, w), k // w)
    k = (1 << 21) - 1 - rng.integers(0, 4096, w.shape[0])      # the top of the float range
    assert np.array_equal(_rows(k, w), k // w)


def test_row_is_floor_division_for_every_k_of_small_rectangles():
    for width in range(1, 257):
        k = np.arange(0, 256 * width, dtype=np.int64)           # every pair of a width x 256 rectangle
        assert np.array_equal(_rows(k, np.full_like(k, width)), k // width)
