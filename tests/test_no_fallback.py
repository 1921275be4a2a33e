"""The product path has no CPU fallback: the binding refuses host tensors
before any work, and a missing CUDA library is an error, not a silent
substitute.  Runs without a GPU."""
import pytest
import torch


def test_host_tensors_are_refused():
    import paper_2312_13299_gb300 as plas
    x = torch.rand(16 * 16, 3)
    with pytest.raises(ValueError, match="CUDA"):
        plas.sort(x, 16, 16)
    with pytest.raises(ValueError, match="CUDA"):
        plas.smooth_loss(torch.rand(8, 8, 3), 1.0, 7)
    with pytest.raises(ValueError, match="CUDA"):
        plas.check_permutation(torch.arange(4, dtype=torch.int32))
    with pytest.raises(ValueError, match="CUDA"):
        plas.activate_3dgs(torch.rand(4, 14))


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2312_13299_gb300 import _lib, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent" / "libplas.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()
