"""The product path has no CPU fallback (no GPU needed): without the built library the binding
raises instead of computing anything, and without a CUDA device creating a context fails with the
library's CUDA status."""
import pytest

from paper_1810_09784_gb300 import gfh


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(gfh, "_LIB_PATH", tmp_path / "libgfh.so")
    monkeypatch.setattr(gfh, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        gfh.lib()
    with pytest.raises(RuntimeError, match="missing"):
        gfh.Context(0, None)


def test_no_device_no_context(built_lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(built_lib.GfhError) as e:
        built_lib.Context(0, None)
    assert e.value.args and "gfh_create" in str(e.value)
