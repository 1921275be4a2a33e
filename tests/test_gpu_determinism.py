"""Race canary: a sort is a pure function of its inputs (counter-based random
streams, exact integer residual sums, order-free swaps of disjoint groups).
Ten reruns of the same 3DGS-shaped 256x256x14 sort, on the default stream
and on a side stream, give bit-identical permutations, carried attributes
and per-iteration residual sums; a data race in any kernel would show up as
a difference between reruns."""
import numpy as np
import pytest
import torch

from paper_2312_13299_gb300 import synth

pytestmark = pytest.mark.gpu


def test_ten_reruns_identical(plas):
    side = 256
    x, c = synth.gaussians_3dgs(side * side, seed=11)
    xc, cc = torch.from_numpy(x).cuda(), torch.from_numpy(c).cuda()
    first = plas.sort(xc, side, side, carried=cc, seed=4, trace_cap=1 << 15)
    n = first.state["it"]
    assert 0 < n <= 1 << 15
    side_stream = torch.cuda.Stream()
    for k in range(10):
        if k % 2:
            with torch.cuda.stream(side_stream):
                res = plas.sort(xc, side, side, carried=cc, seed=4, trace_cap=1 << 15)
            side_stream.synchronize()
        else:
            res = plas.sort(xc, side, side, carried=cc, seed=4, trace_cap=1 << 15)
        assert res.state["it"] == n
        assert torch.equal(res.perm, first.perm)
        assert torch.equal(res.carried, first.carried)
        assert torch.equal(res.trace_S, first.trace_S)
    assert plas.check_permutation(first.perm) == -1
