"""Pins of the oracle's preparation steps (Sec. 3.1: sort on activated
values, largest square grid with the lowest-opacity Gaussians pruned;
Sec. 3.3: coordinate contraction).

* grid_select equals a stable numpy lexsort by (-logit, index) on data with
  ties, -0/+0 and NaN, for several sizes around perfect squares.
* activate_3dgs inverts the contraction (sign(x) log1p(|x|) returns the
  parameter), exp/log round-trips the scale, quaternions come out unit
  length (zero stays zero), the sigmoid is symmetric (s(-v) = 1 - s(v)) and
  equals 1/2 at 0, and the DC colour passes through.
"""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 3, 4, 15, 16, 17, 1000, 4097])
def test_grid_select_matches_lexsort(orc, n):
    rng = np.random.default_rng(n)
    op = rng.integers(-4, 5, n).astype(np.float32) * 0.5  # many ties
    op[rng.random(n) < 0.05] = np.nan
    op[rng.random(n) < 0.05] = -0.0
    side, keep = orc.grid_select(op)
    assert side == int(np.floor(np.sqrt(n)))
    key = np.where(np.isnan(op), -np.inf, op.astype(np.float64) + 0.0)
    nan_last = np.isnan(op).astype(np.int64)
    order = np.lexsort((np.arange(n), -key, nan_last))  # last key is primary
    want = np.sort(order[:side * side])
    assert np.array_equal(keep, want)


def test_activation_invariants(orc):
    rng = np.random.default_rng(1)
    raw = rng.normal(0, 2, (500, 14)).astype(np.float32)
    raw[0, 6:10] = 0.0
    out = orc.activate_3dgs(raw).astype(np.float64)
    r64 = raw.astype(np.float64)
    back = np.sign(out[:, :3]) * np.log1p(np.abs(out[:, :3]))
    assert np.allclose(back, r64[:, :3], rtol=1e-6, atol=1e-6)
    assert np.allclose(np.log(out[:, 3:6]), r64[:, 3:6], rtol=1e-6, atol=1e-6)
    norms = np.linalg.norm(out[1:, 6:10], axis=1)
    assert np.allclose(norms, 1.0, atol=1e-6) and np.all(out[0, 6:10] == 0)
    neg = raw.copy()
    neg[:, 10] = -neg[:, 10]
    s_neg = orc.activate_3dgs(neg)[:, 10].astype(np.float64)
    assert np.allclose(s_neg, 1.0 - out[:, 10], atol=1e-7)
    zero = raw[:1].copy()
    zero[0, 10] = 0.0
    assert orc.activate_3dgs(zero)[0, 10] == 0.5
    assert np.array_equal(out[:, 11:14], r64[:, 11:14])
