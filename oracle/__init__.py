"""CPU oracle for the exact mesh-to-grid projection (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` import this
package. The library (``paper_1509_07720_gb300``) never does, and shares no code with it.

``oracle.c`` computes the plain definition of the projection (Sect. 3, Eq. firstOrder; output of
Algorithm 2): m_V = sum over simplices S of the integral of the linear interpolant of the vertex
densities over S intersected with cell V, by clipping every simplex against every cell of its
bounding box and integrating exactly on the clipped pieces. It is pinned by the tests in
``tests/test_oracle_pins.py`` against closed forms, invariants, an independent exact-rational
slicing integrator and Monte Carlo.

The shared object is compiled from ``oracle.c`` with the host C compiler on first use (or by
``build()``); it is plain C with OpenMP, no CUDA.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ERRORS = {0: "ok", -1: "bad argument", -2: "vertex index out of range",
          -4: "simplex spans half a periodic box or more"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile liboracle.so from oracle.c if it is missing or older than the source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        llp = ctypes.POINTER(ctypes.c_longlong)
        common = [ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong, dp, dp, dp, ip, dp, ip, dp, dp,
                  ctypes.c_int]
        lib.cdo_project.argtypes = common + [dp, llp, llp, ctypes.c_int]
        lib.cdo_project.restype = ctypes.c_int
        lib.cdo_project_cells.argtypes = common + [ctypes.c_longlong, llp, dp, ctypes.c_int]
        lib.cdo_project_cells.restype = ctypes.c_int
        lib.cdo_simplex_mass.argtypes = common + [dp]
        lib.cdo_simplex_mass.restype = ctypes.c_int
        lib.cdo_max_threads.argtypes = []
        lib.cdo_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


def _args(mesh):
    d = mesh.dim
    pos = [np.ascontiguousarray(mesh.pos[a], dtype=np.float64) for a in range(d)]
    while len(pos) < 3:
        pos.append(pos[0])
    simp = np.ascontiguousarray(mesh.simplices, dtype=np.int32)
    rho = np.ascontiguousarray(mesh.rho, dtype=np.float64)
    grid = np.ascontiguousarray(mesh.grid, dtype=np.int32)
    lo = np.ascontiguousarray(mesh.box_lo, dtype=np.float64)
    ln = np.ascontiguousarray(mesh.box_len, dtype=np.float64)
    keep = (pos, simp, rho, grid, lo, ln)
    args = [d, mesh.n_verts, mesh.n_simplices, _ptr(pos[0]), _ptr(pos[1]), _ptr(pos[2]),
            _ptr(simp, ctypes.c_int), _ptr(rho), _ptr(grid, ctypes.c_int), _ptr(lo), _ptr(ln),
            int(bool(mesh.periodic))]
    return args, keep


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle error {rc}: {ERRORS.get(rc, 'unknown')}")


def project(mesh, nthreads: int = 0, stats: bool = False):
    """Cell masses (float64 array shaped ``mesh.grid``). With ``stats``, also returns
    (n_pieces, n_cells_tested): nonzero (simplex, cell) pairs and clipped bounding-box pairs."""
    lib = _load()
    args, keep = _args(mesh)
    out = np.zeros(int(np.prod(mesh.grid)), dtype=np.float64)
    npieces = ctypes.c_longlong(0)
    ntested = ctypes.c_longlong(0)
    rc = lib.cdo_project(*args, _ptr(out), ctypes.byref(npieces), ctypes.byref(ntested), int(nthreads))
    _check(rc)
    out = out.reshape(mesh.grid)
    if stats:
        return out, int(npieces.value), int(ntested.value)
    return out


def project_cells(mesh, cells, nthreads: int = 0):
    """Masses of the flat C-order cell indices ``cells`` only."""
    lib = _load()
    args, keep = _args(mesh)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros(cells.size, dtype=np.float64)
    rc = lib.cdo_project_cells(*args, cells.size, _ptr(cells, ctypes.c_longlong), _ptr(out), int(nthreads))
    _check(rc)
    return out


def simplex_mass(mesh):
    """|vol(S)| * mean(rho over its vertices) per simplex (world units)."""
    lib = _load()
    args, keep = _args(mesh)
    out = np.zeros(mesh.n_simplices, dtype=np.float64)
    _check(lib.cdo_simplex_mass(*args, _ptr(out)))
    return out


def max_threads() -> int:
    return int(_load().cdo_max_threads())
