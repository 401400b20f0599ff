"""The C-ABI library loads and exports every symbol include/lym1.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "lym1.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lym1_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    from paper_2606_02711_gb300 import build
    try:
        build.build()
    except (RuntimeError, FileNotFoundError) as e:
        pytest.skip(f"nvcc unavailable: {e}")
    import paper_2606_02711_gb300.lym1 as L
    return L


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.SIGNATURES)


def test_strerror_and_no_device_status(L):
    assert L.strerror(0) == "ok"
    assert "invalid" in L.strerror(L.EINVAL)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2606_02711_gb300.lym1 as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        L.lib()
