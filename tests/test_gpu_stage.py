"""Preparation before the sort on the GPU (Sec. 3.1, Sec. 3.3): the kept set
of the largest square grid bit-exact against the oracle; activation within
a few ulp of the FP64 oracle; and the whole chain raw -> activate -> select
-> sort equal to the oracle sorting the same kept features."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 17, 4096, 5000, 1 << 20, 1_234_567])
def test_grid_select_bitexact(plas, orc, n):
    rng = np.random.default_rng(n)
    op = (rng.integers(-200, 200, n) * 0.05).astype(np.float32)  # ties
    op[rng.random(n) < 0.01] = np.nan
    op[rng.random(n) < 0.01] = -0.0
    side, keep = plas.grid_select(torch.from_numpy(op).cuda())
    oside, okeep = orc.grid_select(op)
    assert side == oside
    assert np.array_equal(keep.cpu().numpy(), okeep)


def test_grid_select_strided_view(plas, orc):
    raw = np.random.default_rng(3).normal(size=(10000, 14)).astype(np.float32)
    t = torch.from_numpy(raw).cuda()
    side, keep = plas.grid_select(t[:, 10])
    assert np.array_equal(keep.cpu().numpy(), orc.grid_select(raw[:, 10])[1])


def test_activation_close_to_fp64(plas, orc):
    raw = np.random.default_rng(4).normal(0, 2, (50000, 14)).astype(np.float32)
    raw[0, 6:10] = 0.0
    got = plas.activate_3dgs(torch.from_numpy(raw).cuda()).cpu().numpy()
    want = orc.activate_3dgs(raw)
    tol = 4 * np.spacing(np.abs(want).astype(np.float32)) + 1e-30
    assert np.all(np.abs(got - want) <= tol)


@pytest.mark.parametrize("n,stride", [(1, 14), (255, 59), (257, 59), (100_003, 59), (4096, 15)])
def test_activation_strided_rows_and_tails(plas, orc, n, stride):
    """Rows of the 59-channel layout (only the first 14 are read), blocks of
    256 rows cut by a ragged tail, and a single row: within a few ulp of the
    FP64 oracle, and the extra columns never leak into the output."""
    rng = np.random.default_rng(n + stride)
    raw = rng.normal(0, 2, (n, stride)).astype(np.float32)
    got = plas.activate_3dgs(torch.from_numpy(raw).cuda()).cpu().numpy()
    want = orc.activate_3dgs(raw)
    assert got.shape == (n, 14)
    tol = 4 * np.spacing(np.abs(want).astype(np.float32)) + 1e-30
    assert np.all(np.abs(got - want) <= tol)


def test_prepare_then_sort_matches_oracle(plas, orc):
    rng = np.random.default_rng(5)
    raw = rng.normal(0, 1.5, (70 * 70 + 123, 14)).astype(np.float32)
    rt = torch.from_numpy(raw).cuda()
    feats = plas.activate_3dgs(rt)
    side, keep = plas.grid_select(rt[:, 10])
    assert side == 70
    x = plas.select_rows(feats, keep)
    got = plas.sort(x, side, side, seed=9)
    want = orc.sort(x.cpu().numpy(), side, side, seed=9)
    assert np.array_equal(got.perm.cpu().numpy(), want["perm"])
