"""Pins of the oracle's box target (the fast low-pass variant: the mean of
the in-range cells of the (2r+1) x (2r+1) window, on fixed-point features).

* A constant grid whose value is exact in fixed point comes back exactly.
* Brute force on small grids (explicit window loops in Python integers).
* scipy.ndimage.correlate with a ones kernel on the same fixed-point values,
  divided by the in-range count, agrees within one FP32 rounding.
* The fixed-point exponent is the largest with B * 2^s <= 2^31.
* A sort in box mode is a valid permutation and lowers the grid's mean
  neighbour distance.
"""
import numpy as np
import pytest
from scipy import ndimage


def _target(orc, x, H, W, phi, **kw):
    return orc.target_box(x, H, W, np.arange(H * W, dtype=np.int32), phi, **kw)


def test_constant_grid_is_exact(orc):
    x = np.full((12 * 9, 2), 0.25, np.float32)
    T = _target(orc, x, 12, 9, 3.0, normalize_=False)
    assert np.all(T == 0.25)


@pytest.mark.parametrize("H,W,phi", [(7, 9, 2.0), (5, 13, 4.5), (16, 3, 1.0)])
def test_brute_force_small(orc, H, W, phi):
    rng = np.random.default_rng(H * W)
    x = rng.random((H * W, 3), dtype=np.float32)
    T = _target(orc, x, H, W, phi, normalize_=False)
    s = orc.box_exp(x, normalize_=False)
    q = [[[int(np.rint(np.ldexp(float(x[y * W + xx, d]), s))) for d in range(3)] for xx in range(W)]
         for y in range(H)]
    r = int(np.floor(phi))
    for y in range(H):
        for xx in range(W):
            for d in range(3):
                S, n = 0, 0
                for yy in range(max(0, y - r), min(H, y + r + 1)):
                    for xw in range(max(0, xx - r), min(W, xx + r + 1)):
                        S += q[yy][xw][d]
                        n += 1
                want = np.ldexp(np.float32(np.float32(S) / np.float32(n)), -s).astype(np.float32)
                assert T[y, xx, d] == want


def test_matches_scipy_window_sums(orc):
    H, W, phi = 40, 33, 6.0
    x = np.random.default_rng(1).random((H * W, 4), dtype=np.float32) * 3
    w = np.array([1.0, 0.5, 2.0, 1.5], np.float32)
    T = orc.target_box(x, H, W, np.arange(H * W, dtype=np.int32), phi, weights=w)
    # normalised, weighted features as the oracle builds them
    lo, hi = x.min(0), x.max(0)
    F = (w * ((x - lo) / (hi - lo))).astype(np.float32).reshape(H, W, 4)
    s = orc.box_exp(x, weights=w)
    q = np.rint(np.ldexp(F.astype(np.float64), s))
    r = 6
    k = np.ones((2 * r + 1, 2 * r + 1, 1))
    S = ndimage.correlate(q, k, mode="constant")
    n = ndimage.correlate(np.ones((H, W, 1)), k, mode="constant")
    want = np.ldexp(S / n, -s)
    assert np.allclose(T, want, rtol=2 ** -23, atol=0)


def test_box_exponent_is_maximal(orc):
    x = np.random.default_rng(2).normal(0, 5, (100, 3)).astype(np.float32)
    for normalize in (True, False):
        w = np.array([0.3, 7.0, 1.0], np.float32)
        s = orc.box_exp(x, weights=w, normalize_=normalize)
        B = np.abs(w).max() if normalize else (np.abs(w) * np.maximum(np.abs(x.min(0)), np.abs(x.max(0)))).max()
        assert np.ldexp(B, s) <= 2 ** 31 < np.ldexp(B, s + 1) or s == 40


def test_box_mode_sort_is_valid_and_smooths(orc):
    H = W = 24
    x = np.random.default_rng(3).random((H * W, 3), dtype=np.float32)
    r = orc.sort(x, H, W, seed=1, sched=orc.default_schedule(target_mode=1))
    perm = r["perm"]
    assert np.array_equal(np.sort(perm), np.arange(H * W))
    g = x[perm].reshape(H, W, 3)
    g0 = x.reshape(H, W, 3)
    def nl2(a):
        return (np.linalg.norm(a[1:] - a[:-1], axis=2).mean() + np.linalg.norm(a[:, 1:] - a[:, :-1], axis=2).mean())
    assert nl2(g) < 0.6 * nl2(g0)
