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


def test_struct_layout_matches_header():
    import ctypes

    # int, pad, 2 x int64, 3 pointers, 2 pointers, 3 int32, pad, 6 doubles, int, pad, pointer
    assert ctypes.sizeof(pkg.cdp_problem) == 8 + 16 + 24 + 16 + 16 + 48 + 8 + 8
    assert ctypes.sizeof(pkg.cdp_stats) == 14 * 8 + 8
