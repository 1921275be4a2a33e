"""Pins of the oracle's schedule and feature preparation (Sec. 3.1).

* Radius levels: phi0 = w/2 - 1, phi <- 0.95 phi, stop below 1; the count is
  the closed form floor(ln(phi0) / ln(1/0.95)) + 1 (64 -> 67, 512 -> 109,
  1024 -> 122, 1448 -> 129) and the values follow phi0 * 0.95^L.
* State machine, checked with closed forms: with an unreachable tolerance
  every level is exactly one improving and two stalled iterations (3L
  iterations, 2L epochs, L redraws); every level of a real run has >= 3
  iterations and the level trace never decreases.
* Snapshots: a run split into several calls (permutation + state) equals the
  run in one call, and a fresh start equals a resume from the initial random
  placement.
* Normalisation: per channel to [0, 1] (min -> 0, max -> 1 exactly), then the
  weight; a constant channel maps to 0.
"""
import json
import math
import os

import numpy as np
import pytest

from conftest import GOLDEN


def test_levels_closed_form(orc):
    pv = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["schedule"]
    for side, want in [(64, 67), (512, 109), (1024, 122), (1448, 129)]:
        phis = orc.levels(side, side)
        phi0 = side / 2 - 1
        assert len(phis) == want == math.floor(math.log(phi0) / math.log(1 / pv["shrink"])) + 1
        assert phis[0] == phi0 and phis[-1] >= pv["phi_min"] and phis[-1] * pv["shrink"] < 1
        L = np.arange(len(phis))
        assert np.allclose(phis, phi0 * pv["shrink"] ** L, rtol=1e-12)


def test_levels_small_and_rectangular(orc):
    assert orc.levels(3, 3).tolist() == [1.0]          # phi0 < 1: one level at phi = 1
    assert orc.levels(1, 1).tolist() == [1.0]
    assert orc.levels(40, 100)[0] == 19.0               # min side drives phi0


def test_unreachable_tolerance_gives_three_per_level(orc):
    x = np.random.default_rng(0).random((32 * 48, 3), dtype=np.float32)
    r = orc.sort(x, 32, 48, seed=1, sched=orc.default_schedule(tol=1e9))
    L = len(orc.levels(32, 48))
    st = r["state"]
    assert st.it == 3 * L and st.epoch == 2 * L and st.redraws == L and st.done == 1
    assert np.array_equal(r["trace_level"], np.repeat(np.arange(L), 3))


def test_level_trace_properties(orc):
    x = np.random.default_rng(1).random((48 * 48, 3), dtype=np.float32)
    r = orc.sort(x, 48, 48, seed=2)
    lv = r["trace_level"]
    assert np.all(np.diff(lv) >= 0) and lv[0] == 0 and lv[-1] == len(orc.levels(48, 48)) - 1
    counts = np.bincount(lv)
    assert counts.min() >= 3
    assert r["state"].done == 1 and r["iterations"] == len(lv)
    # every level ends with two non-improving iterations
    k = r["state"].scale_exp
    d = r["trace_S"].astype(np.float64) / (48 * 48 * 2.0 ** k)
    for L in range(lv[-1] + 1):
        idx = np.nonzero(lv == L)[0]
        a, b, c = d[idx[-3]], d[idx[-2]], d[idx[-1]]
        assert not (b < a and a - b >= 1e-4 * a)
        assert not (c < b and b - c >= 1e-4 * b)


def _initial(orc, seed, n):
    t = orc.prp_table(seed, orc.TAG_INIT, 0, n)
    perm = np.empty(n, np.int32)
    perm[t] = np.arange(n, dtype=np.int32)
    return perm


def test_snapshot_resume_equals_single_run(orc):
    H, W = 40, 40
    x = np.random.default_rng(5).random((H * W, 3), dtype=np.float32)
    full = orc.sort(x, H, W, seed=11)
    perm, state, tS = None, None, []
    for cap in [1, 7, 30, 200, 10 ** 9]:
        r = orc.sort(x, H, W, seed=11, sched=orc.default_schedule(max_iters=cap),
                     perm_in=perm, state=state)
        perm, state = r["perm"], r["state"]
        tS.append(r["trace_S"])
        if state.done:
            break
    assert state.done and np.array_equal(perm, full["perm"])
    assert np.array_equal(np.concatenate(tS), full["trace_S"])
    fresh1 = orc.sort(x, H, W, seed=11, sched=orc.default_schedule(max_iters=1))
    res1 = orc.sort(x, H, W, seed=11, sched=orc.default_schedule(max_iters=1),
                    perm_in=_initial(orc, 11, H * W), state=orc.State())
    assert np.array_equal(fresh1["perm"], res1["perm"])


def test_seed_changes_result(orc):
    x = np.random.default_rng(6).random((32 * 32, 3), dtype=np.float32)
    a = orc.sort(x, 32, 32, seed=1)["perm"]
    b = orc.sort(x, 32, 32, seed=1)["perm"]
    c = orc.sort(x, 32, 32, seed=2)["perm"]
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_normalize(orc):
    rng = np.random.default_rng(7)
    x = rng.normal(size=(500, 4)).astype(np.float32) * [1, 10, 0.01, 3]
    x[:, 3] = 2.5  # constant channel
    x = x.astype(np.float32)
    w = np.array([1.0, 2.0, 0.5, 7.0], np.float32)
    F = orc.normalize(x, w)
    for d in range(3):
        assert F[:, d].min() == 0.0 and F[:, d].max() == w[d]
        i = np.argmax(x[:, d])
        assert F[i, d] == w[d]
    assert np.all(F[:, 3] == 0.0)
    ref = (x[:, :3].astype(np.float64) - x[:, :3].min(0)) / (x[:, :3].max(0) - x[:, :3].min(0)) * w[:3]
    assert np.allclose(F[:, :3], ref, rtol=1e-6, atol=1e-7)
    G = orc.normalize(x, w, normalize=False)
    assert np.array_equal(G, (x * w).astype(np.float32))


def test_scale_exponent(orc):
    x = np.random.default_rng(8).random((1000, 14), dtype=np.float32)
    assert orc.scale_exp(x) == 32
    for wscale in [1e6, 1e9, 1e12]:
        w = np.full(14, wscale, np.float32)
        k = orc.scale_exp(x, w)
        m = 1000 * math.sqrt(14 * float(np.float32(wscale)) ** 2)
        assert k < 32 and math.ldexp(m, k) < 2 ** 62
        assert k == 0 or math.ldexp(m, k + 1) >= 2 ** 62


def test_quality_band_small(orc):
    """Statistical: a 64x64 random colour grid gets much smoother (not exact)."""
    x = np.random.default_rng(0).random((64 * 64, 3), dtype=np.float32)
    r = orc.sort(x, 64, 64, seed=0)
    g0 = x.reshape(64, 64, 3)
    g1 = x[r["perm"]].reshape(64, 64, 3)
    v0 = orc.metrics(g0, 255.0)[1]
    v1 = orc.metrics(g1, 255.0)[1]
    assert v0 > 3000 and v1 < v0 / 10
    assert orc.metrics(g1)[0] < orc.metrics(g0)[0] / 4
