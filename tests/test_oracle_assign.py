"""Pins of the oracle's assignment step (Sec. 3.1 "Blockwise Linear
Assignment": groups of four, best of the 24 permutations by total distance to
the target).

* The 24 permutations come in the lexicographic order of itertools.
* The group step is an exact 4x4 linear assignment problem: the chosen
  permutation's cost equals scipy.optimize.linear_sum_assignment's optimum
  (and is that assignment when the optimum is unique); an asymmetric cost
  matrix catches a transposed C.
* Ties go to the lexicographically first permutation (the identity for a
  constant matrix).
* Tiny grids: on a 2x2 grid one iteration reaches the best of all 24
  arrangements for the target of that iteration (brute force in FP64); on a
  3x3 grid each of the two groups is brute-force optimal and the leftover cell
  stays.
* Invariants over many iterations: the output is a bijection, the summed
  squared distance to the iteration's target never increases, and the
  schedule's residual (the exact fixed-point sum of per-cell L2 distances)
  equals numpy's FP64 sum within the rounding of its terms.
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment


def test_perm24_order(orc):
    assert orc.perm24().tolist() == [list(p) for p in itertools.permutations(range(4))]


def test_best_perm_is_linear_assignment(orc):
    rng = np.random.default_rng(0)
    P = orc.perm24()
    for _ in range(500):
        C = rng.random((4, 4), dtype=np.float32) * rng.choice([1e-3, 1.0, 50.0])
        k = orc.best_perm(C)
        rows, cols = linear_sum_assignment(C.astype(np.float64))
        opt = C.astype(np.float64)[rows, cols].sum()
        got = sum(float(C[i, P[k][i]]) for i in range(4))
        assert got <= opt * (1 + 4e-7) + 1e-12
        if len({round(sum(float(C[i, p[i]]) for i in range(4)), 5) for p in P}) == 24:
            assert list(P[k]) == list(cols)


def test_best_perm_transposed_matrix_differs(orc):
    # C[i][j] = cost of element i at position j; a strongly asymmetric matrix
    C = np.array([[0, 9, 9, 9], [9, 9, 0, 9], [9, 9, 9, 0], [9, 0, 9, 9]], np.float32)
    P = orc.perm24()
    assert list(P[orc.best_perm(C)]) == [0, 2, 3, 1]
    assert list(P[orc.best_perm(C.T.copy())]) == [0, 3, 1, 2]


def test_best_perm_ties_first(orc):
    assert orc.best_perm(np.ones((4, 4), np.float32)) == 0
    C = np.zeros((4, 4), np.float32)
    C[0, 0] = 1.0  # identity now costs 1; (0,1,...) orders with element 0 elsewhere cost 0
    P = orc.perm24()
    k = orc.best_perm(C)
    costs = [sum(C[i, p[i]] for i in range(4)) for p in P]
    assert k == int(np.argmin(costs))


def _initial(orc, seed, n):
    """Initial random placement: Gaussian i sits at cell pi0(i)."""
    t = orc.prp_table(seed, orc.TAG_INIT, 0, n)
    perm = np.empty(n, np.int32)
    perm[t] = np.arange(n, dtype=np.int32)
    return perm


def _sq(a, b):
    d = a.astype(np.float64) - b.astype(np.float64)
    return (d * d).sum(-1)


def test_2x2_one_iteration_is_optimal(orc):
    for seed in range(20):
        x = np.random.default_rng(seed).random((4, 3), dtype=np.float32)
        r = orc.sort(x, 2, 2, seed=seed, sched=orc.default_schedule(max_iters=1), want_target=True)
        F = orc.normalize(x)
        T = r["T"].reshape(4, 3)
        best = min(_sq(F[list(p)], T).sum() for p in itertools.permutations(range(4)))
        got = _sq(F[r["perm"]], T).sum()
        assert got <= best * (1 + 1e-6) + 1e-12


def test_3x3_groups_optimal_leftover_fixed(orc):
    for seed in range(10):
        x = np.random.default_rng(100 + seed).random((9, 2), dtype=np.float32)
        s0 = orc.sort(x, 3, 3, seed=seed, sched=orc.default_schedule(max_iters=1), want_target=True)
        init = _initial(orc, seed, 9)
        st = s0["state"]
        assert st.it == 1
        T = s0["T"].reshape(9, 2)
        F = orc.normalize(x)
        pi = orc.prp_table(seed, orc.TAG_GROUP, 0, 9)  # beta = 3: one block, shift 0
        after = s0["perm"]
        for g in range(2):
            cells = [int(pi[4 * g + k]) for k in range(4)]
            elems = [int(init[c]) for c in cells]
            assert sorted(after[cells].tolist()) == sorted(elems)
            best = min(_sq(F[[elems[i] for i in p]], T[cells]).sum()
                       for p in itertools.permutations(range(4)))
            got = _sq(F[after[cells]], T[cells]).sum()
            assert got <= best * (1 + 1e-6) + 1e-12
        left = int(pi[8])
        assert after[left] == init[left]


@pytest.mark.parametrize("H,W,D", [(16, 16, 3), (24, 40, 5), (33, 17, 2)])
def test_invariants_per_iteration(orc, H, W, D):
    x = np.random.default_rng(H * W).random((H * W, D), dtype=np.float32)
    F = orc.normalize(x)
    phis = orc.levels(H, W)
    perm = _initial(orc, 3, H * W)
    state = None
    for it in range(40):
        r = orc.sort(x, H, W, seed=3, sched=orc.default_schedule(max_iters=it + 1),
                     perm_in=perm, state=state if state is not None else orc.State(),
                     want_target=True)
        new = r["perm"]
        assert np.array_equal(np.sort(new), np.arange(H * W))
        T = r["T"].reshape(H * W, D)
        lvl = (state.level if state is not None else 0)
        assert np.array_equal(T, orc.target(x, H, W, perm, phis[lvl]).reshape(H * W, D))
        before, after = _sq(F[perm], T).sum(), _sq(F[new], T).sum()
        assert after <= before * (1 + 1e-9) + 1e-12
        # the schedule's residual: the sum over all cells of the (non-squared)
        # L2 distance to this iteration's target, each term rounded to a
        # multiple of 2^-k; numpy in FP64 gives it independently (the FP32
        # per-cell distances differ from it by a few ulp)
        k = r["state"].scale_exp
        e = np.sqrt(((F[new].astype(np.float64) - T.astype(np.float64)) ** 2).sum(axis=1))
        S = float(r["trace_S"][0]) * 2.0 ** -k
        assert abs(S - e.sum()) <= H * W * 2.0 ** -k + 4e-7 * e.sum()
        assert r["state"].d_last == r["trace_S"][0] / (H * W * 2.0 ** k)
        perm, state = new, r["state"]
        if state.done:
            break
