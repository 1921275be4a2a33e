"""Pin of the oracle's output gather (Sec. 3: every attribute plane follows
the one permutation found by the sort; the permutation is in gather form,
sorted[p] = input[perm[p]]).

The oracle's gather is checked against numpy's own fancy indexing
``src[perm]``, an independent definition, on random permutations of several
row counts and widths, including one row, one channel and 45 channels (the
carried SH-rest attributes).  A scatter (``out[perm] = src``) in its place
fails every case with a non-involutive permutation, which is also checked."""
import numpy as np
import pytest


@pytest.mark.parametrize("N,C", [(1, 1), (2, 3), (7, 1), (1000, 45), (4096, 14), (513, 64)])
def test_gather_equals_numpy_indexing(orc, N, C):
    rng = np.random.default_rng(N * 100 + C)
    src = rng.standard_normal((N, C)).astype(np.float32)
    perm = rng.permutation(N).astype(np.int32)
    got = orc.gather(src, perm)
    assert np.array_equal(got, src[perm])
    if N > 2:
        # gather and scatter differ unless perm is its own inverse
        inv = np.empty_like(perm)
        inv[perm] = np.arange(N, dtype=np.int32)
        if not np.array_equal(inv, perm):
            scattered = np.empty_like(src)
            scattered[perm] = src
            assert not np.array_equal(got, scattered)


def test_gather_of_a_cycle(orc):
    """A 3-cycle by hand: row p of the output is row perm[p] of the input."""
    src = np.array([[10.0], [20.0], [30.0]], np.float32)
    perm = np.array([2, 0, 1], np.int32)
    assert orc.gather(src, perm)[:, 0].tolist() == [30.0, 10.0, 20.0]
