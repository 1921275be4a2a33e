"""Pins of the oracle's random sources (Philox4x32-10 + keyed Feistel permutation).

* Philox: published known-answer vectors (tests/golden/philox4x32_10_kat.txt,
  Salmon et al. SC'11 / Random123) -- a wrong constant, round count, key bump
  or word order fails them.
* Permutation: exhaustive bijection for every domain size up to 2^12 and
  sampled sizes up to 2^20; chi-square uniformity of where one element lands.
* Block shift: always inside [0, min(beta, side - beta + 1)).
"""
import os

import numpy as np
import pytest

from conftest import GOLDEN


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t, 16) for t in line.split()]
                rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox(ctr, key)
        assert [int(v) for v in got] == want


def test_philox_uniform_bits(orc):
    # 4 x 4096 outputs on consecutive counters: every bit is a fair coin
    outs = np.array([orc.philox([i, 7, 0, 0], [1, 2]) for i in range(4096)], dtype=np.uint64)
    bits = np.array([(outs >> b) & 1 for b in range(32)])
    frac = bits.mean(axis=(1, 2))
    # 16384 draws per bit: 5 sigma = 5 * 0.5 / sqrt(16384) ~ 0.0195
    assert np.all(np.abs(frac - 0.5) < 0.02)


@pytest.mark.parametrize("n", list(range(1, 65)) + [100, 255, 256, 257, 1000, 4095, 4096])
def test_prp_is_bijection_small(orc, n):
    t = orc.prp_table(123, orc.TAG_GROUP, 5, n)
    assert sorted(t.tolist()) == list(range(n))


@pytest.mark.parametrize("n", [2 ** 14 + 3, 2 ** 16, 3 * 2 ** 17 + 11, 2 ** 20])
def test_prp_is_bijection_large(orc, n):
    t = orc.prp_table(9, orc.TAG_INIT, 0, n)
    assert np.array_equal(np.sort(t), np.arange(n, dtype=np.uint32))


def test_prp_streams_differ(orc):
    a = orc.prp_table(1, orc.TAG_GROUP, 0, 256)
    b = orc.prp_table(1, orc.TAG_GROUP, 1, 256)
    c = orc.prp_table(2, orc.TAG_GROUP, 0, 256)
    d = orc.prp_table(1, orc.TAG_INIT, 0, 256)
    assert not np.array_equal(a, b) and not np.array_equal(a, c) and not np.array_equal(a, d)


def test_prp_uniform_landing(orc):
    # where element 0 lands over 4000 counters: chi-square over 16 bins of [0, 256)
    n, trials = 256, 4000
    land = np.array([orc.prp(77, orc.TAG_GROUP, c, n, 0) for c in range(trials)])
    hist = np.bincount(land * 16 // n, minlength=16)
    exp = trials / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 45.0  # 15 dof, p ~ 1e-4


@pytest.mark.parametrize("H,W,beta", [(64, 64, 32), (64, 64, 64), (24, 40, 16), (17, 17, 16),
                                      (1448, 1448, 724), (100, 30, 30)])
def test_shift_range(orc, H, W, beta):
    my, mx = min(beta, H - beta + 1), min(beta, W - beta + 1)
    seen_y, seen_x = set(), set()
    for e in range(300):
        dy, dx = orc.shift(5, e, beta, H, W)
        assert 0 <= dy < my and 0 <= dx < mx
        seen_y.add(dy)
        seen_x.add(dx)
    assert len(seen_y) == min(my, len(seen_y)) and len(seen_y) >= min(my, 20)
