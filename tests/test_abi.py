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


def test_struct_layouts_match_header(tmp_path):
    """Every field of sip_problem_desc, sip_solve_opts and sip_solve_report
    sits at the same offset in the C header (compiled as C) as in the
    ctypes binding, and the sizes agree."""
    import shutil
    import subprocess
    from paper_1607_03777_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sip_problem_desc": _lib.ProblemDesc, "sip_solve_opts": _lib.SolveOpts,
               "sip_solve_report": _lib.SolveReport}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sipstokes.h"',
             "int main(void) {"]
    expect = []
    for cname, cls in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {fname}));')
            expect.append(getattr(cls, fname).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == expect


def test_solve_opts_defaults(lib):
    """sip_solve_opts_default: the paper's settings and the library defaults."""
    from paper_1607_03777_gb300 import _lib
    o = _lib.SolveOpts()
    f = lib.sip_solve_opts_default
    f.argtypes = [ctypes.POINTER(_lib.SolveOpts)]
    f(ctypes.byref(o))
    assert (o.rtol, o.max_outer, o.restart, o.inner_rtol, o.max_inner) == (1e-8, 500, 100, 1e-3, 200)
    assert (o.inner_loop, o.inner_krylov, o.inner_norm, o.inner_restart) == (0, 0, 0, 30)
    assert (o.outer_krylov, o.refine) == (0, 0)
