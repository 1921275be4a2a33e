"""Pins of the oracle's quantisation (Sec. 3.4: clip each attribute channel
to a range, round to the nearest of q equally spaced values).

* Values on the levels map to their own index (exactly representable grid).
* Values below / above the range (and NaN) give the first / last level / 0.
* Away from ties the code is the nearest level found by FP64 brute force.
* Exact ties round to the even code; a degenerate range gives 0.
* Dequantisation: levels of a range whose step is a power of two come back
  exactly; code 0 is lo; a degenerate range gives lo; every value is within
  half a step (plus rounding) of the clipped input it was quantised from.
"""
import numpy as np


def test_levels_map_to_their_index(orc):
    q = 2 ** 10 + 1
    k = np.arange(q)
    x = (k / (q - 1)).astype(np.float32).reshape(-1, 1)
    codes = orc.quantize(x, [0.0], [1.0], [q])
    assert np.array_equal(codes[:, 0], k)


def test_clip_nan_and_degenerate(orc):
    x = np.array([[-5.0, 0.5], [7.0, 0.5], [np.nan, 0.5], [2.0, 0.5]], np.float32)
    codes = orc.quantize(x, [-2.0, 0.5], [4.0, 0.5], [64, 32])
    assert codes[:, 0].tolist() == [0, 63, 0, 42]  # (2+2)/6*63 = 42
    assert codes[:, 1].tolist() == [0, 0, 0, 0]    # hi == lo


def test_nearest_level_brute_force(orc):
    rng = np.random.default_rng(0)
    lo, hi = np.float32(-1.0), np.float32(2.0)
    for q in [32, 64, 16384]:
        x = rng.uniform(-1.5, 2.5, 20000).astype(np.float32).reshape(-1, 1)
        codes = orc.quantize(x, [lo], [hi], [q])[:, 0].astype(np.int64)
        v = np.clip(x[:, 0].astype(np.float64), lo, hi)
        pos = (v - lo) / (hi - lo) * (q - 1)
        far = np.abs(pos - np.floor(pos) - 0.5) > 1e-3
        levels = np.arange(q)
        nearest = np.abs(pos[:, None] - levels[None, :]).argmin(1) if q <= 64 else np.rint(pos).astype(np.int64)
        assert np.array_equal(codes[far], nearest[far])
        assert np.all(np.abs(codes - pos) <= 0.5 + 1e-3)


def test_ties_round_to_even(orc):
    q = 9  # q - 1 = 8: t * 8 = k + 1/2 exactly for x = (k + 1/2) / 8
    k = np.arange(8)
    x = ((k + 0.5) / 8).astype(np.float32).reshape(-1, 1)
    codes = orc.quantize(x, [0.0], [1.0], [q])[:, 0]
    want = [int(np.rint(v)) for v in (k + 0.5)]  # numpy rint: half to even
    assert codes.tolist() == want and all(c % 2 == 0 for c in codes)


def test_dequantize_closed_forms(orc):
    codes = np.arange(5, dtype=np.uint16).reshape(-1, 1).repeat(3, 1)
    got = orc.dequantize(codes, [0.0, -1.0, 3.0], [1.0, 3.0, 3.0], [5, 5, 7])
    assert got[:, 0].tolist() == [0.0, 0.25, 0.5, 0.75, 1.0]   # step 1/4
    assert got[:, 1].tolist() == [-1.0, 0.0, 1.0, 2.0, 3.0]    # step 1
    assert got[:, 2].tolist() == [3.0] * 5                     # hi == lo: lo


def test_dequantize_inverts_quantize_within_half_a_step(orc):
    rng = np.random.default_rng(1)
    lo = np.array([-1.0, 0.0, -6.0], np.float32)
    hi = np.array([2.0, 1.0, 12.0], np.float32)
    q = np.array([64, 2 ** 14, 256], np.int32)
    x = rng.uniform(-8, 14, (5000, 3)).astype(np.float32)
    back = orc.dequantize(orc.quantize(x, lo, hi, q), lo, hi, q).astype(np.float64)
    v = np.clip(x.astype(np.float64), lo, hi)
    step = (hi.astype(np.float64) - lo) / (q - 1)
    assert np.all(np.abs(back - v) <= 0.5 * step + 4e-7 * np.abs(hi - lo).max())
