"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/*.h declares; the Python binding covers exactly those names.
No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ras_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2411_00546_gb300 import build, ras
    if not os.path.exists(ras.LIB_PATH):
        build.build()
    return ras.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ras_create", "ras_set_eps", "ras_apply", "ras_newton_ras_solve", "ras_raspen_solve",
                     "ras_jvp", "ras_residual", "ras_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_matches_header(lib_path):
    from paper_2411_00546_gb300 import ras
    assert set(ras.exported_symbols()) == _declared()
    ras.lib()
    o = ras.ras_default_opts()
    # the paper's settings (Sec. 5): tol 1e-10, inner 1e-8, eps0 1, gamma 1/5, sigma 1.1
    assert (o.tol, o.inner_tol, o.eps0, o.gamma, o.sigma) == (1e-10, 1e-8, 1.0, 0.2, 1.1)
    assert ras.ras_launch_count() >= 0


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of the boundary has the same size and field offsets in C
    (gcc on include/ras.h) and in the ctypes binding."""
    import shutil
    import subprocess
    from paper_2411_00546_gb300 import ras
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    structs = [ras.ras_opts, ras.ras_stats, ras.ras_problem_desc, ras.ras_state, ras.ras_tuning,
               ras.ras_tune_report]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ras.h"', "int main(void) {"]
    expect = []
    for S in structs:
        name = S.__name__
        lines.append('printf("%%zu\\n", sizeof(%s));' % name)
        expect.append(ctypes.sizeof(S))
        for field, _ in S._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (name, field))
            expect.append(getattr(S, field).offset)
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect
