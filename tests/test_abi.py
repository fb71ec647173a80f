"""The C-ABI library builds for sm_103a, loads, and exports every symbol
declared in include/sipstokes.h (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sipstokes.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sip_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1607_03777_gb300 import build, _lib
    build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_header_declares_entry_points():
    names = declared_functions()
    assert "sip_apply_A" in names and "sip_problem_create" in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1607_03777_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_problem_desc_layout_matches_header(lib):
    """sip_problem_desc_default fills the struct through the ctypes layout."""
    from paper_1607_03777_gb300 import _lib
    d = _lib.ProblemDesc()
    f = lib.sip_problem_desc_default
    f.argtypes = [ctypes.POINTER(_lib.ProblemDesc)]
    f(ctypes.byref(d))
    assert (d.cheb_steps_p, d.cheb_steps_h, d.eig_iters) == (2, 3, 10)
    assert (d.cheb_lo, d.cheb_hi, d.penalty_scale) == (0.1, 1.1, 1.0)


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    """Loading fails loudly when the compiled library is absent."""
    from paper_1607_03777_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()
