"""Pins of the oracle's low-pass target (Sec. 3.1: blur of the grid, shrinking
radius).  The oracle's FP32 fmaf chain is compared with independent
computations:

* scipy.ndimage.correlate1d (mode 'constant') divided by the correlate1d of a
  ones-grid (= the in-range tap mass) along each axis, in FP64;
* a direct 2-D sum with the outer-product kernel and a 2-D mass map;
* invariants: a constant grid stays constant, a linear ramp is preserved away
  from the border (symmetric taps), and swapping the axes of the input swaps
  the axes of the output (catches a transposed pass).
"""
import numpy as np
import pytest
from scipy import ndimage


def _ref_blur(G, r, sigma):
    j = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-(j * j) / (2.0 * sigma * sigma)).astype(np.float32).astype(np.float64)
    H, W, D = G.shape
    ones = np.ones((H, W), np.float64)
    mx = ndimage.correlate1d(ones, k, axis=1, mode="constant", cval=0.0)
    my = ndimage.correlate1d(ones, k, axis=0, mode="constant", cval=0.0)
    t = ndimage.correlate1d(G.astype(np.float64), k, axis=0, mode="constant") / my[..., None]
    t = ndimage.correlate1d(t, k, axis=1, mode="constant") / mx[..., None]
    return t


@pytest.mark.parametrize("H,W,D,r,sigma", [(37, 53, 3, 5, 2.5), (64, 64, 14, 31, 15.5),
                                           (20, 9, 2, 12, 6.0), (16, 16, 1, 1, 0.5),
                                           (5, 40, 4, 7, 10.0)])
def test_blur_matches_scipy(orc, H, W, D, r, sigma):
    G = np.random.default_rng(1).random((H, W, D), dtype=np.float32)
    T = orc.blur(G, r, sigma)
    ref = _ref_blur(G, r, sigma)
    assert np.allclose(T, ref, rtol=2e-6, atol=2e-7)


def test_blur_matches_direct_2d(orc):
    H, W, D, r, sigma = 23, 31, 2, 6, 3.0
    G = np.random.default_rng(2).random((H, W, D), dtype=np.float32)
    j = np.arange(-r, r + 1)
    k = np.exp(-(j * j) / (2.0 * sigma * sigma)).astype(np.float32).astype(np.float64)
    K2 = np.outer(k, k)
    ref = np.zeros((H, W, D))
    for y in range(H):
        for x in range(W):
            y0, y1, x0, x1 = max(0, y - r), min(H, y + r + 1), max(0, x - r), min(W, x + r + 1)
            w = K2[y0 - y + r:y1 - y + r, x0 - x + r:x1 - x + r]
            ref[y, x] = np.tensordot(w, G[y0:y1, x0:x1].astype(np.float64), axes=([0, 1], [0, 1])) / w.sum()
    assert np.allclose(orc.blur(G, r, sigma), ref, rtol=2e-6, atol=2e-7)


def test_blur_constant_grid(orc):
    G = np.full((40, 33, 3), 0.3712, np.float32)
    T = orc.blur(G, 9, 4.5)
    assert np.max(np.abs(T.astype(np.float64) - 0.3712)) <= 4 * np.spacing(np.float32(0.3712))


def test_blur_preserves_linear_ramp_interior(orc):
    H, W, r = 30, 50, 6
    yy, xx = np.mgrid[0:H, 0:W]
    G = np.stack([xx * 0.01, yy * 0.02], -1).astype(np.float32)
    T = orc.blur(G, r, 3.0)
    inner = (slice(r, H - r), slice(r, W - r))
    assert np.allclose(T[inner], G[inner], atol=2e-6)


def test_blur_transpose_symmetry(orc):
    G = np.random.default_rng(3).random((21, 34, 2), dtype=np.float32)
    a = orc.blur(G, 4, 2.0)
    b = orc.blur(np.ascontiguousarray(G.transpose(1, 0, 2)), 4, 2.0).transpose(1, 0, 2)
    # the two pass orders differ only by FP32 rounding
    assert np.allclose(a, b, rtol=1e-6, atol=1e-7)


def test_taps_shape(orc):
    t = orc.taps(6, 3.0).astype(np.float64)
    assert t[6] == 1.0 and np.array_equal(t, t[::-1])
    assert np.all(np.diff(t[6:]) < 0)
    # edge tap of sigma = phi / 2 at j = phi: exp(-2)
    assert abs(t[-1] - np.exp(-2.0)) < 1e-7
