"""The C-ABI library loads and exports every symbol include/coldproj.h declares (no GPU needed)."""
import os
import re

import pytest

import paper_1509_07720_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names.update(re.findall(r"CDP_API\s+[\w\s\*]*?\b(cdp_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1509_07720_gb300 import build

    build.build_library()
    return pkg.load_library()


def test_header_declares_symbols():
    names = _declared()
    assert {"cdp_create", "cdp_destroy", "cdp_project", "cdp_check", "cdp_strerror"} <= names
    assert names == set(pkg.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_without_gpu(lib):
    assert pkg.cdp_strerror(0) == "ok"
    assert "index" in pkg.cdp_strerror(-2)
    assert pkg.cdp_strerror(12345) == "unknown error"


def test_argument_errors_without_gpu(lib):
    # invalid arguments are rejected on the host before anything touches a device
    prob = pkg.cdp_problem()
    prob.dim = 4
    assert pkg.cdp_project(None, prob, pkg.CDP_FP64) == -1
    import ctypes

    assert lib.cdp_create(None, 0) == -1
    assert lib.cdp_check(None, None) == -1


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler gives the header's structs."""
    import ctypes
    import subprocess

    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "coldproj.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(cdp_problem), sizeof(cdp_stats),\n'
        "         offsetof(cdp_problem, cell_mass), offsetof(cdp_stats, error_flags), offsetof(cdp_stats, n_deferred),\n"
        "         offsetof(cdp_stats, accuracy_bound), sizeof(cdp_step_problem));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    want = [ctypes.sizeof(pkg.cdp_problem), ctypes.sizeof(pkg.cdp_stats), pkg.cdp_problem.cell_mass.offset,
            pkg.cdp_stats.error_flags.offset, pkg.cdp_stats.n_deferred.offset, pkg.cdp_stats.accuracy_bound.offset,
            ctypes.sizeof(pkg.cdp_step_problem)]
    assert got == want
