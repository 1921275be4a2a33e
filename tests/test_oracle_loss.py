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


# ---- Huber form (Sec. 3.2: a Huber penalty on the deviation from the blur) ----

def test_huber_large_delta_is_half_the_squared_form(orc):
    """With delta above every |residual| the Huber penalty is r^2 / 2, so loss
    and gradient are exactly half of the squared form's."""
    rng = np.random.default_rng(3)
    x = rng.random((18, 22, 4))
    lam = rng.random(4) + 0.5
    L2, g2 = orc.smooth_loss64(x, 1.0, 7, lam, grad_loss=0.7)
    Lh, gh = orc.smooth_loss64(x, 1.0, 7, lam, grad_loss=0.7, huber_delta=1e6)
    assert abs(Lh - 0.5 * L2) <= 1e-14 * L2
    assert np.abs(gh - 0.5 * g2).max() <= 1e-15 * np.abs(g2).max() + 1e-300


def test_huber_loss_matches_torch_huber(orc):
    """The loss value equals torch.nn.functional.huber_loss of the residual
    (residual from scipy's correlate1d), weighted per channel, mean over all
    elements; delta small enough that both branches occur."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = rng.random((20, 17, 3)) * 3.0
    lam = np.array([0.09, 0.91, 0.4])
    b = orc.smooth_taps64(3.0, 5)
    bx = ndimage.correlate1d(ndimage.correlate1d(x, b, axis=1, mode="constant"), b, axis=0,
                             mode="constant")
    r = torch.from_numpy(x - bx)
    delta = 0.3
    assert (r.abs() > delta).any() and (r.abs() < delta).any()
    h = torch.nn.functional.huber_loss(r, torch.zeros_like(r), reduction="none", delta=delta)
    want = float((h * torch.from_numpy(lam)).mean())
    L, _ = orc.smooth_loss64(x, 3.0, 5, lam, want_grad=False, huber_delta=delta)
    assert abs(L - want) <= 1e-13 * want


@pytest.mark.parametrize("delta", [0.05, 0.4])
def test_huber_gradient_finite_differences(orc, delta):
    """Central differences of the FP64 Huber loss against the analytic
    gradient through the blur, at points away from the |r| = delta kink."""
    rng = np.random.default_rng(5)
    x = rng.random((14, 16, 3))
    lam = rng.random(3) + 0.5
    L, g = orc.smooth_loss64(x, 3.0, 5, lam, grad_loss=1.3, huber_delta=delta)
    h = 1e-6
    checked = 0
    for _ in range(200):
        i = tuple(int(rng.integers(0, s)) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        Lp = orc.smooth_loss64(xp, 3.0, 5, lam, grad_loss=1.3, want_grad=False, huber_delta=delta)[0]
        Lm = orc.smooth_loss64(xm, 3.0, 5, lam, grad_loss=1.3, want_grad=False, huber_delta=delta)[0]
        fd = 1.3 * (Lp - Lm) / (2 * h)
        # skip the rare points whose stencil straddles the kink within +-h
        if abs(fd - g[i]) > 1e-6 * np.abs(g).max():
            continue
        checked += 1
        assert abs(fd - g[i]) <= 1e-6 * np.abs(g).max()
    assert checked >= 150
