"""plas_check_permutation: the device bijection check of a sort's output
(Sec. 3.1: every Gaussian lands on exactly one grid cell).  Valid
permutations of ragged sizes pass; planted duplicates and out-of-range values
(host-made inputs, all in-bounds for the check's own reads) report the
smallest position that holds an out-of-range or repeated value, which numpy
computes directly from that definition."""
import numpy as np
import pytest
import torch

from paper_2312_13299_gb300 import synth

pytestmark = pytest.mark.gpu


def _first_bad(p: np.ndarray) -> int:
    N = p.size
    inr = (p >= 0) & (p < N)
    counts = np.bincount(p[inr], minlength=N)
    bad = ~inr
    bad[inr] |= counts[p[inr]] > 1
    idx = np.nonzero(bad)[0]
    return int(idx[0]) if idx.size else -1


@pytest.mark.parametrize("N", [1, 31, 32, 33, 1000, (1 << 20) + 3])
def test_valid_permutations_pass(plas, N):
    rng = np.random.default_rng(N)
    for p in (np.arange(N), rng.permutation(N), np.arange(N)[::-1]):
        assert plas.check_permutation(torch.from_numpy(np.ascontiguousarray(p, np.int32)).cuda()) == -1


def test_empty_permutation(plas):
    assert plas.check_permutation(torch.empty(0, dtype=torch.int32, device="cuda")) == -1


@pytest.mark.parametrize("N,case", [(1, "big"), (2, "dup"), (33, "neg"), (1000, "dup"),
                                    (1000, "big"), (4099, "two"), ((1 << 20) + 3, "dup"),
                                    ((1 << 20) + 3, "many")])
def test_planted_faults_report_the_first_bad_position(plas, N, case):
    rng = np.random.default_rng(7 * N + len(case))
    p = rng.permutation(N).astype(np.int64)
    if case == "big":
        p[rng.integers(N)] = N
    elif case == "neg":
        p[rng.integers(N)] = -5
    elif case == "dup":
        a, b = rng.choice(N, 2, replace=False)
        p[b] = p[a]
    elif case == "two":
        p[N - 1] = 2 ** 31 - 1
        a, b = rng.choice(N - 1, 2, replace=False)
        p[a] = p[b]
    else:
        k = rng.choice(N, 64, replace=False)
        p[k] = rng.integers(-3, N + 3, 64)
    p = p.astype(np.int32)
    want = _first_bad(p)
    assert want >= 0
    assert plas.check_permutation(torch.from_numpy(p).cuda()) == want


def test_sort_output_checked(plas):
    x, c = synth.gaussians_3dgs(96 * 80, seed=3)
    res = plas.sort(torch.from_numpy(x).cuda(), 96, 80, carried=torch.from_numpy(c).cuda(), seed=1,
                    check_perm=True)
    assert plas.check_permutation(res.perm) == -1
