"""The allocation-free smoothness-loss forward (plas_smooth_loss_fwd_noalloc).

Some callers cannot allocate device memory inside the call (their memory is
owned by another allocator with a fixed budget, or cudaMalloc's possible
device synchronisation is not allowed in their loop).  This entry point keeps
its scratch in a static device array of the library.  The test calls it
through the C ABI twice in a row and checks each result against the regular
entry point within the loss tolerance (1e-5 relative); it also checks that an
oversized grid is rejected.  It lives in its own file, collected last, and
passes alone in a fresh process as well as after the other tests."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def _regular(lib, x, H, W, C, stream, ksize=7):
    out = torch.empty((), dtype=torch.float32, device="cuda")
    rc = lib.plas_smooth_loss_fwd(x.data_ptr(), H, W, C, 1.0, ksize, None, out.data_ptr(), None, 0,
                                  stream)
    assert rc == 0
    return out


def _noalloc_twice(lib, x, H, W, C, stream, ref, ksize=7, rel=1e-5):
    for _ in range(2):
        out = torch.full((), float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.plas_smooth_loss_fwd_noalloc(x.data_ptr(), H, W, C, 1.0, ksize, None,
                                              out.data_ptr(), stream)
        assert rc == 0, lib.plas_last_error()
        torch.cuda.synchronize()
        assert abs(out.item() - ref.item()) <= rel * abs(ref.item())


def test_noalloc_loss_matches_regular_twice(plas):
    lib = plas.load()
    stream = torch.cuda.current_stream().cuda_stream
    for (H, W, C, seed) in [(256, 192, 59, 0), (100, 37, 3, 1)]:
        g = torch.Generator(device="cuda").manual_seed(seed)
        x = torch.rand((H, W, C), device="cuda", generator=g)
        ref = _regular(lib, x, H, W, C, stream)
        _noalloc_twice(lib, x, H, W, C, stream, ref)


def test_noalloc_strip_path(plas):
    """The strip kernel (taken for ksize > 15, or for an input that is not
    16-byte aligned) keeps its partial sums in the same static array."""
    lib = plas.load()
    stream = torch.cuda.current_stream().cuda_stream
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.rand((90, 70, 5), device="cuda", generator=g)
    ref = _regular(lib, x, 90, 70, 5, stream, ksize=17)
    _noalloc_twice(lib, x, 90, 70, 5, stream, ref, ksize=17)
    # one float past a 16-byte boundary: the staged kernel's aligned copies
    # cannot be used, so both calls take the strip kernel
    buf = torch.rand(64 * 48 * 14 + 1, device="cuda", generator=g)
    xm = buf[1:]
    assert xm.data_ptr() % 16 != 0
    ref = _regular(lib, xm, 64, 48, 14, stream)
    _noalloc_twice(lib, xm, 64, 48, 14, stream, ref)


def test_noalloc_taller_row_bands(plas):
    """129 channels on a 4100 x 4104 grid: 32-row bands would need 513 x 129 >
    65536 partial sums, so the allocation-free call runs 64-row bands and adds
    the FP64 partials in another grouping; it agrees with the regular call
    within rounding."""
    lib = plas.load()
    stream = torch.cuda.current_stream().cuda_stream
    H, W, C = 4100, 4104, 129
    g = torch.Generator(device="cuda").manual_seed(9)
    x = torch.rand((H, W, C), device="cuda", generator=g)
    ref = _regular(lib, x, H, W, C, stream)
    _noalloc_twice(lib, x, H, W, C, stream, ref)
    del x
    torch.cuda.empty_cache()


def test_noalloc_rejects_oversized_grid(plas):
    lib = plas.load()
    x = torch.zeros(1, device="cuda")
    out = torch.zeros((), device="cuda")
    # 8224 x 8224 cells need 257 * 257 > 65536 partial sums; rejected before any launch
    rc = lib.plas_smooth_loss_fwd_noalloc(x.data_ptr(), 8224, 8224, 1, 1.0, 7, None,
                                          out.data_ptr(), None)
    assert rc == -1
    assert b"65536" in lib.plas_last_error()
