"""Host-only entry points of the C ABI, called without a GPU: the schedule
defaults (Sec. 3.1 and the supplementary's threshold), the level count
against the oracle's own schedule, workspace sizes, status strings and the
argument checks that return before any device work."""
import ctypes

import pytest

import paper_2312_13299_gb300 as plas
from paper_2312_13299_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return plas.load()


def test_default_schedule_values(lib):
    s = _lib.plas_schedule()
    assert lib.plas_default_schedule(ctypes.byref(s)) == 0
    assert (s.phi0, s.shrink, s.phi_min, s.tol, s.sigma_ratio, s.min_block) == (0.0, 0.95, 1.0, 1e-4, 2.0, 16)
    assert (s.shuffle_init, s.normalize, s.max_iters, s.target_mode) == (1, 1, 0, 0)
    py = plas.Schedule()
    assert (py.shrink, py.phi_min, py.tol, py.sigma_ratio, py.min_block) == (
        s.shrink, s.phi_min, s.tol, s.sigma_ratio, s.min_block)
    assert lib.plas_default_schedule(None) == _lib.PLAS_ERR_INVALID_ARG


@pytest.mark.parametrize("H,W,kw", [(64, 64, {}), (1024, 1024, {}), (1448, 1448, {}), (40, 100, {}),
                                    (3, 3, {}), (1, 7, {}), (256, 256, {"shrink": 0.8}),
                                    (200, 300, {"phi0": 50.0, "phi_min": 2.5})])
def test_level_count_matches_oracle(lib, orc, H, W, kw):
    got = plas.num_levels(H, W, plas.Schedule(**kw))
    want = len(orc.levels(H, W, orc.default_schedule(**kw)))
    assert got == want


def test_level_count_rejects_bad_schedules(lib):
    with pytest.raises(RuntimeError):
        plas.num_levels(0, 5)
    with pytest.raises(RuntimeError):
        plas.num_levels(8, 8, plas.Schedule(shrink=1.0))


def test_workspace_sizes(lib):
    a = plas.sort_workspace_bytes(512, 512, 14)
    b = plas.sort_workspace_bytes(1024, 1024, 14)
    assert 0 < a < b
    assert plas.sort_workspace_bytes(1024, 1024, 14, plas.Schedule(target_mode=1)) > b
    assert plas.sort_workspace_bytes(0, 5, 3) == 0
    assert plas.sort_workspace_bytes(8, 8, 17) == 0        # unsupported channel count
    assert plas.sort_workspace_bytes(1 << 14, 1 << 14, 3) == 0  # more than 2^26 cells


def test_status_strings(lib):
    for code, word in [(0, "ok"), (-1, "invalid"), (-2, "memory"), (-3, "CUDA"), (-4, "timed out"),
                       (-5, "NaN"), (-6, "budget"), (-7, "internal"), (-8, "permutation")]:
        assert word in lib.plas_status_string(code).decode()
    assert "unknown" in lib.plas_status_string(-99).decode()


def test_permutation_check_argument_errors(lib):
    first = ctypes.c_int(7)
    assert lib.plas_check_permutation(None, 0, ctypes.byref(first), None) == 0
    assert first.value == -1
    assert lib.plas_check_permutation(None, -1, None, None) == _lib.PLAS_ERR_INVALID_ARG
    assert lib.plas_check_permutation(None, 5, None, None) == _lib.PLAS_ERR_INVALID_ARG
    assert lib.plas_check_permutation(None, (1 << 30) + 1, None, None) == _lib.PLAS_ERR_INVALID_ARG


def test_loss_rejects_grids_taller_than_the_launch_limit(lib):
    """The strip kernel of the smoothness loss (ksize > 15) runs one CTA row
    per 32 grid rows; a grid that would need more than CUDA's 65535 CTA rows
    is rejected before any launch or allocation (the pointers are never
    dereferenced)."""
    fake = ctypes.c_void_p(256)
    H = 65536 * 32  # ceil(H / 32) = 65536 > 65535
    for fn in ("plas_smooth_loss_fwd",):
        rc = getattr(lib, fn)(fake, H, 1, 1, 1.0, 17, None, fake, None, 0, None)
        assert rc == _lib.PLAS_ERR_INVALID_ARG
        assert b"65535" in lib.plas_last_error()
    rc = lib.plas_smooth_loss_bwd(fake, H, 1, 1, 1.0, 17, None, fake, fake, None, 0, None)
    assert rc == _lib.PLAS_ERR_INVALID_ARG
