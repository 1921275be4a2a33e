"""Pins of the oracle's grid metrics.

* VAD (supplementary, "Sorting performance": variance of the absolute
  differences of all neighbouring values over all channels) of a shuffled
  U[0,1) 512x512x3 grid on the 0..255 scale matches the closed form
  255^2/18 = 3612.5 of |U1 - U2| and the paper's 3607.45 (both within 1 %).
* Mean neighbour L2 and VAD equal a direct numpy evaluation.
"""
import json
import os

import numpy as np

from conftest import GOLDEN


def test_vad_closed_form_and_paper_value(orc):
    pv = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["vad_shuffled_512x512x3"]
    g = np.random.default_rng(0).random((512, 512, 3), dtype=np.float32)
    vad = orc.metrics(g, pv["scale"])[1]
    assert abs(vad - 255.0 ** 2 / 18.0) / 3612.5 < 0.01
    assert abs(vad - pv["value"]) / pv["value"] < 0.01


def test_metrics_direct(orc):
    g = np.random.default_rng(1).random((13, 17, 4), dtype=np.float32)
    nl2, vad = orc.metrics(g, 2.0)
    d = g.astype(np.float64)
    dh = d[:, 1:] - d[:, :-1]
    dv = d[1:] - d[:-1]
    l2 = np.concatenate([np.sqrt((dh ** 2).sum(-1)).ravel(), np.sqrt((dv ** 2).sum(-1)).ravel()])
    a = np.abs(np.concatenate([dh.ravel(), dv.ravel()])) * 2.0
    assert abs(nl2 - l2.mean()) < 1e-12
    assert abs(vad - a.var()) < 1e-10


def test_3x3_sort_against_all_arrangements(orc):
    """Brute force over all 9! = 362,880 arrangements of a 3x3 grid: the
    optimal mean neighbour L2 E* is a lower bound for the sort's result (a
    heuristic, so only the bound is asserted and the gap is printed), the
    oracle's metric of the optimal arrangement equals E*, and the sort's
    result lies below the mean over all arrangements."""
    import itertools
    x = np.random.default_rng(9).random((9, 3), dtype=np.float32)
    F = orc.normalize(x).astype(np.float64)
    perms = np.array(list(itertools.permutations(range(9))), dtype=np.int8)
    G = F[perms].reshape(-1, 3, 3, 3)
    dh = np.sqrt(((G[:, :, 1:] - G[:, :, :-1]) ** 2).sum(-1)).reshape(len(perms), -1)
    dv = np.sqrt(((G[:, 1:] - G[:, :-1]) ** 2).sum(-1)).reshape(len(perms), -1)
    E = np.concatenate([dh, dv], axis=1).mean(axis=1)
    best = int(np.argmin(E))
    e_star = float(E[best])
    nl2_best = orc.metrics(F[perms[best]].reshape(3, 3, 3).astype(np.float32))[0]
    assert abs(nl2_best - e_star) < 1e-6
    r = orc.sort(x, 3, 3, seed=0)
    e_plas = orc.metrics(F[r["perm"]].reshape(3, 3, 3).astype(np.float32))[0]
    assert e_plas >= e_star - 1e-6
    assert e_plas < float(E.mean())
    print(f"3x3: E* = {e_star:.5f}, PLAS = {e_plas:.5f}, mean = {E.mean():.5f}")
