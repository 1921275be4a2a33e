"""Quantisation of the sorted attribute grids (Sec. 3.4) on the GPU: codes
bit-exact against the oracle (the integer is decided in FP32 on both sides),
the round trip within half a level, and argument checks."""
import numpy as np
import pytest
import torch

from paper_2312_13299_gb300 import synth

pytestmark = pytest.mark.gpu

# the paper's q per attribute and clip ranges; coordinates and scale use the
# data's own range (the paper gives none)
def _paper_config(x):
    C = x.shape[1]
    lo = np.zeros(C, np.float32)
    hi = np.zeros(C, np.float32)
    q = np.zeros(C, np.int32)
    for c in range(C):
        if c < 3:        # coordinates
            lo[c], hi[c], q[c] = x[:, c].min(), x[:, c].max(), 2 ** 14
        elif c < 6:      # scale
            lo[c], hi[c], q[c] = x[:, c].min(), x[:, c].max(), 2 ** 6
        elif c < 10:     # rotation
            lo[c], hi[c], q[c] = -1.0, 2.0, 2 ** 6
        elif c < 11:     # opacity
            lo[c], hi[c], q[c] = -6.0, 12.0, 2 ** 6
        elif c < 14:     # DC colour, stored as 8 bits
            lo[c], hi[c], q[c] = -2.0, 4.0, 2 ** 8
        else:            # SH rest
            lo[c], hi[c], q[c] = -1.0, 1.0, 2 ** 5
    return lo, hi, q


def test_quantize_bitexact_and_round_trip(plas, orc):
    x = synth.loss_grid(96, 80, seed=5).reshape(-1, 59).astype(np.float32)
    x[::97, 3] *= 50.0                       # out-of-range and extreme values
    x[5, 10], x[6, 11], x[7, 20] = np.nan, np.inf, -np.inf
    lo, hi, q = _paper_config(np.nan_to_num(x, nan=0.0, posinf=0.0, neginf=0.0))
    want = orc.quantize(x, lo, hi, q)
    codes = plas.quantize(torch.from_numpy(x).cuda(), lo, hi, q)
    got = (codes.to(torch.int32) & 0xFFFF).cpu().numpy()
    assert np.array_equal(got, want.astype(np.int32))
    back = plas.dequantize(codes, lo, hi, q).cpu().numpy()
    finite = np.isfinite(x)
    v = np.clip(np.where(finite, x, 0.0), lo, hi)
    step = (hi - lo) / (q - 1)
    err = np.abs(back - v)
    assert np.all(err[finite] <= (0.5 * step + 1e-6 * np.abs(hi - lo) + 1e-7)[None, :].repeat(x.shape[0], 0)[finite])


def test_quantize_rejects_bad_ranges(plas):
    x = torch.rand(10, 2, device="cuda")
    with pytest.raises(RuntimeError):
        plas.quantize(x, [0.0, 1.0], [1.0, 0.0], [4, 4])
    with pytest.raises(RuntimeError):
        plas.quantize(x, [0.0, 0.0], [1.0, 1.0], [1, 4])


@pytest.mark.parametrize("N,C,offset", [(1, 1, 0), (3, 1, 0), (4097, 3, 0), (1001, 7, 1), (300000, 59, 0),
                                        (999, 256, 0), (2, 5, 3), (70000, 14, 2)])
def test_quantize_dequantize_bitexact_shapes(plas, orc, N, C, offset):
    """Both directions bit for bit against the oracle: element counts that
    are not a multiple of 4, one channel, the maximum of 256 channels, many
    grid-stride steps, and views that start off a 16-byte boundary (the
    scalar path)."""
    rng = np.random.default_rng(N * C + offset)
    x = rng.normal(0, 2, N * C + offset).astype(np.float32)
    lo = rng.uniform(-3, 0, C).astype(np.float32)
    hi = (lo + rng.uniform(0, 4, C)).astype(np.float32)
    hi[::5] = lo[::5]                                   # degenerate ranges
    q = rng.integers(2, 65537, C).astype(np.int32)
    xt = torch.from_numpy(x).cuda()[offset:].view(N, C)
    xs = x[offset:].reshape(N, C)
    want = orc.quantize(xs, lo, hi, q)
    codes = plas.quantize(xt, lo, hi, q)
    assert np.array_equal((codes.to(torch.int32) & 0xFFFF).cpu().numpy(), want.astype(np.int32))
    ct = torch.from_numpy(np.concatenate([np.zeros(offset, np.uint16), want.ravel()]).view(np.int16)).cuda()
    back = plas.dequantize(ct[offset:].view(N, C), lo, hi, q).cpu().numpy()
    assert np.array_equal(back.view(np.uint32), orc.dequantize(want, lo, hi, q).view(np.uint32))
