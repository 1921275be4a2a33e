"""The C ABI: the library builds for sm_103a here (nvcc cross-compiles), loads
without a GPU, and exports exactly the functions include/plas.h declares; the
Python binding declares a prototype for each of them.  No compute call is made."""
import ctypes
import os
import re
import subprocess

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "plas.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return set(re.findall(r"\b(plas_[a-z0-9_]+)\s*\(", src))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["plas_sort", "plas_smooth_loss_fwd", "plas_smooth_loss_bwd", "plas_batch_sort",
                 "plas_sort_workspace_bytes", "plas_default_schedule", "plas_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2312_13299_gb300 import _lib, build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    declared = _declared()
    assert declared <= exported, declared - exported
    lib = ctypes.CDLL(path)
    for n in declared:
        assert hasattr(lib, n)
    assert declared == set(_lib.SIGNATURES)


def test_library_is_sm103a_only():
    from paper_2312_13299_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert "-fmad=false" in build.NVFLAGS


# (fir_small_below, fir_medium_below, assign_ctas_per_sm) when nothing is installed
DEFAULT_TUNING = (12, 96, 4)


def test_tuning_table_round_trip_host_only():
    """The launch-shape table is host state: install, look up (nearest cell
    count for the same D), validate and remove -- no device work."""
    import paper_2312_13299_gb300 as plas
    assert plas.get_tuning(64, 64, 5)["small_fused"] == 1   # both passes in one launch by default
    plas.set_tuning(64, 64, 5, fir_small_below=7, fir_medium_below=40, assign_ctas_per_sm=3)
    try:
        t = plas.get_tuning(64, 64, 5)
        assert (t["fir_small_below"], t["fir_medium_below"], t["assign_ctas_per_sm"]) == (7, 40, 3)
        assert t["small_fused"] == 1
        plas.set_tuning(64, 64, 5, small_fused=False)
        assert plas.get_tuning(64, 64, 5)["small_fused"] == 0
        assert plas.get_tuning(64, 64, 5)["fir_small_below"] == 7
        assert plas.get_tuning(70, 60, 5)["fir_small_below"] == 7   # nearest entry, same D
        d = plas.get_tuning(64, 64, 6)                              # other D: defaults
        assert (d["fir_small_below"], d["fir_medium_below"], d["assign_ctas_per_sm"]) == (
            DEFAULT_TUNING)
        import pytest
        with pytest.raises(RuntimeError):
            plas.set_tuning(64, 64, 5, assign_ctas_per_sm=17)
        with pytest.raises(RuntimeError):
            plas.set_tuning(64, 64, 5, fir_medium_below=-1)
    finally:
        plas.set_tuning(64, 64, 5)
    assert plas.get_tuning(64, 64, 5)["assign_ctas_per_sm"] == DEFAULT_TUNING[2]
