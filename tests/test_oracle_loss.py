"""Pins of the oracle's smoothness loss (Sec. 3.2: deviation of each grid value
from a Gaussian blur of the grid; squared deviation with channel weights).

* B x equals scipy.ndimage.correlate1d twice (zero padding, taps normalised
  over the full window).
* The analytic gradient (which uses B^T = B) equals central finite
  differences in FP64 to 1e-7 relative, on 16x16x3 and 32x32x5 grids with
  non-trivial channel weights (a dropped transpose or factor 2 fails).
* A constant grid has zero residual and zero gradient away from the border.
"""
import numpy as np
import pytest
from scipy import ndimage


def test_blur_matches_scipy(orc):
    x = np.random.default_rng(0).random((20, 24, 3))
    b = orc.smooth_taps64(1.0, 7)
    assert abs(b.sum() - 1.0) < 1e-15
    bx = ndimage.correlate1d(ndimage.correlate1d(x, b, axis=1, mode="constant"), b, axis=0,
                             mode="constant")
    L, _ = orc.smooth_loss64(x, 1.0, 7, want_grad=False)
    assert abs(L - ((x - bx) ** 2).mean()) <= 1e-14 * max(1.0, L)


@pytest.mark.parametrize("shape,sigma,ksize", [((16, 16, 3), 1.0, 7), ((32, 32, 5), 3.0, 5)])
def test_gradient_finite_differences(orc, shape, sigma, ksize):
    rng = np.random.default_rng(1)
    x = rng.random(shape)
    lam = rng.random(shape[2]) + 0.5
    g = 0.7
    _, grad = orc.smooth_loss64(x, sigma, ksize, lam, grad_loss=g)
    idx = [tuple(rng.integers(0, s) for s in shape) for _ in range(40)]
    idx += [(0, 0, 0), (shape[0] - 1, shape[1] - 1, shape[2] - 1), (0, shape[1] // 2, 1)]
    h = 1e-6
    for i in idx:
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = g * (orc.smooth_loss64(xp, sigma, ksize, lam, want_grad=False)[0]
                  - orc.smooth_loss64(xm, sigma, ksize, lam, want_grad=False)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 * np.abs(grad).max() + 1e-7 * abs(grad[i])


def test_constant_grid(orc):
    x = np.full((20, 20, 2), 0.25)
    _, grad = orc.smooth_loss64(x, 1.0, 7)
    assert np.abs(grad[6:-6, 6:-6]).max() < 1e-16
    assert np.abs(grad[0, 0]).max() > 0  # border: zero padding pulls the blur down
