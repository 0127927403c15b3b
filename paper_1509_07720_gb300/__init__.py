"""GB300-native exact projection of piecewise-linear simplicial meshes onto regular grids.

Thin Python binding of the C ABI declared in ``include/coldproj.h`` (library
``libcoldproj.so``, built in-tree from ``csrc/`` by ``build.py``). The functions here only
marshal arguments: every step of the projection runs in the CUDA kernels. PyTorch is used for
device memory and streams only. There is no CPU fallback: if the library is missing or no GPU is
present, the calls raise.

Low-level names mirror the ABI (``cdp_create``, ``cdp_project``, ``cdp_check``, ...). The
``Projector`` class wraps them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "CDP_FP64", "CDP_FP32_MIXED", "CdpError", "cdp_problem", "cdp_stats", "load_library", "library_path",
    "cdp_create", "cdp_destroy", "cdp_project", "cdp_check", "cdp_strerror", "cdp_timing_enable",
    "cdp_timing_read", "cdp_project_batched", "cdp_vertex_density", "cdp_poisson", "cdp_force", "cdp_drift",
    "cdp_kick", "cdp_step_batched", "cdp_step_problem", "Projector", "EXPORTED_SYMBOLS",
    "cdp_project_noalloc", "CDP_NOALLOC_MAX_VERTS", "CDP_NOALLOC_MAX_SIMPLICES", "cdp_autotune",
    "CDP_ACCURACY_OFF", "cdp_project_amr", "CDP_AMR_MAX_LEVEL",
]

CDP_FP64 = 0
CDP_FP32_MIXED = 1
# OR'ed into a precision: no accuracy control (every simplex by Franklin's sum)
CDP_ACCURACY_OFF = 0x100
# deepest level of cdp_project_amr (grids divided by 2^level)
CDP_AMR_MAX_LEVEL = 6

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libcoldproj.so")
_lib = None

# every symbol the header declares (checked by the CPU tests)
EXPORTED_SYMBOLS = ("cdp_create", "cdp_destroy", "cdp_project", "cdp_check", "cdp_strerror",
                    "cdp_timing_enable", "cdp_timing_read", "cdp_project_batched", "cdp_vertex_density",
                    "cdp_poisson", "cdp_force", "cdp_drift", "cdp_kick", "cdp_step_batched",
                    "cdp_project_noalloc", "cdp_autotune", "cdp_project_amr")


class CdpError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {cdp_strerror(code)} ({code})" if what else f"{cdp_strerror(code)} ({code})")


class cdp_problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n_verts", ctypes.c_int64),
        ("n_simplices", ctypes.c_int64),
        ("pos", ctypes.c_void_p * 3),
        ("simplices", ctypes.c_void_p),
        ("rho", ctypes.c_void_p),
        ("grid", ctypes.c_int32 * 3),
        ("box_lo", ctypes.c_double * 3),
        ("box_len", ctypes.c_double * 3),
        ("periodic", ctypes.c_int),
        ("cell_mass", ctypes.c_void_p),
    ]


class cdp_step_problem(ctypes.Structure):
    _fields_ = [
        ("mesh", cdp_problem),
        ("vel", ctypes.c_void_p * 3),
        ("acc", ctypes.c_void_p * 3),
        ("simplex_mass", ctypes.c_void_p),
        ("phi", ctypes.c_void_p),
    ]


class cdp_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "n_zero_volume", "n_single_cell", "n_small", "n_large", "n_large_tiles",
        "corners_a", "corners_b", "corners_c", "corners_d", "exact_fallbacks")] + [
        ("large_corners", ctypes.c_uint64 * 4), ("error_flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
        ("n_deferred", ctypes.c_uint64), ("n_clipped", ctypes.c_uint64), ("accuracy_bound", ctypes.c_double)]

    def as_dict(self):
        d = {n: int(getattr(self, n)) for n, _ in self._fields_
             if n not in ("reserved", "large_corners", "accuracy_bound")}
        d["large_corners"] = [int(v) for v in self.large_corners]
        d["accuracy_bound"] = float(self.accuracy_bound)
        return d


def library_path() -> str:
    return _LIB_PATH


def load_library(path: str | None = None):
    """Load libcoldproj.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"{p} not found: build it with `python -m paper_1509_07720_gb300.build`")
    lib = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    lib.cdp_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.cdp_create.restype = ctypes.c_int
    lib.cdp_destroy.argtypes = [vp]
    lib.cdp_destroy.restype = None
    lib.cdp_project.argtypes = [vp, ctypes.POINTER(cdp_problem), ctypes.c_int, ctypes.c_int, vp,
                                ctypes.POINTER(cdp_stats)]
    lib.cdp_project.restype = ctypes.c_int
    lib.cdp_project_amr.argtypes = [vp, ctypes.POINTER(cdp_problem), ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                    ctypes.POINTER(cdp_stats)]
    lib.cdp_project_amr.restype = ctypes.c_int
    lib.cdp_check.argtypes = [vp, vp]
    lib.cdp_check.restype = ctypes.c_int
    lib.cdp_timing_enable.argtypes = [vp, ctypes.c_int]
    lib.cdp_timing_enable.restype = ctypes.c_int
    lib.cdp_timing_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.cdp_timing_read.restype = ctypes.c_int
    lib.cdp_autotune.argtypes = [vp, ctypes.POINTER(cdp_problem), ctypes.c_int, ctypes.c_char_p,
                                 ctypes.POINTER(ctypes.c_int * 3)]
    lib.cdp_autotune.restype = ctypes.c_int
    dp = ctypes.c_void_p
    arr3 = ctypes.c_void_p * 3
    lib.cdp_project_batched.argtypes = [vp, ctypes.POINTER(cdp_problem), ctypes.c_int, ctypes.c_int, vp]
    lib.cdp_project_batched.restype = ctypes.c_int
    lib.cdp_vertex_density.argtypes = [vp, ctypes.POINTER(cdp_problem), dp, dp, vp]
    lib.cdp_vertex_density.restype = ctypes.c_int
    lib.cdp_poisson.argtypes = [vp, ctypes.c_int, ctypes.c_int32 * 3, ctypes.c_double * 3, ctypes.c_double, dp, dp, vp]
    lib.cdp_poisson.restype = ctypes.c_int
    lib.cdp_force.argtypes = [vp, ctypes.c_int, ctypes.c_int32 * 3, ctypes.c_double * 3, ctypes.c_double * 3, dp,
                              ctypes.c_int64, arr3, arr3, vp]
    lib.cdp_force.restype = ctypes.c_int
    lib.cdp_drift.argtypes = [vp, ctypes.c_int, ctypes.c_int64, arr3, arr3, ctypes.c_double, ctypes.c_double * 3,
                              ctypes.c_double * 3, ctypes.c_int, vp]
    lib.cdp_drift.restype = ctypes.c_int
    lib.cdp_kick.argtypes = [vp, ctypes.c_int, ctypes.c_int64, arr3, arr3, ctypes.c_double, vp]
    lib.cdp_kick.restype = ctypes.c_int
    lib.cdp_step_batched.argtypes = [vp, ctypes.POINTER(cdp_step_problem), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
    lib.cdp_step_batched.restype = ctypes.c_int
    lib.cdp_project_noalloc.argtypes = [ctypes.POINTER(cdp_problem), ctypes.c_int, ctypes.c_int, vp, vp]
    lib.cdp_project_noalloc.restype = ctypes.c_int
    lib.cdp_strerror.argtypes = [ctypes.c_int]
    lib.cdp_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def cdp_strerror(code: int) -> str:
    try:
        return load_library().cdp_strerror(int(code)).decode()
    except OSError:
        return f"error {code}"


def _raise(rc, what):
    if rc != 0:
        raise CdpError(rc, what)


def cdp_create(device: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _raise(load_library().cdp_create(ctypes.byref(ctx), int(device)), "cdp_create")
    return ctx


def cdp_destroy(ctx) -> None:
    load_library().cdp_destroy(ctx)


def cdp_project(ctx, prob: cdp_problem, precision: int, accumulate: int = 0, stream: int = 0,
                stats: cdp_stats | None = None) -> int:
    """Raw call; returns the ABI's status code (0 = ok)."""
    return load_library().cdp_project(ctx, ctypes.byref(prob), int(precision), int(accumulate),
                                      ctypes.c_void_p(stream), ctypes.byref(stats) if stats is not None else None)


def cdp_project_amr(ctx, prob: cdp_problem, precision: int, max_level: int, accumulate: int = 0, stream: int = 0,
                    stats: cdp_stats | None = None) -> int:
    """Raw call; returns the ABI's status code (0 = ok)."""
    return load_library().cdp_project_amr(ctx, ctypes.byref(prob), int(precision), int(max_level), int(accumulate),
                                          ctypes.c_void_p(stream), ctypes.byref(stats) if stats is not None else None)


def cdp_check(ctx, stream: int = 0) -> int:
    return load_library().cdp_check(ctx, ctypes.c_void_p(stream))


def cdp_timing_enable(ctx, enable: bool) -> int:
    return load_library().cdp_timing_enable(ctx, int(bool(enable)))


def cdp_timing_read(ctx):
    """(per-kernel totals in ms [vertex records, set-up, main kernel, large tetrahedra (3D), accuracy
    control], timed calls)."""
    buf = (ctypes.c_double * 5)()
    calls = ctypes.c_int(0)
    rc = load_library().cdp_timing_read(ctx, buf, 5, ctypes.byref(calls))
    if rc < 0:
        raise CdpError(rc, "cdp_timing_read")
    return list(buf), int(calls.value)


def cdp_autotune(ctx, prob, precision: int, cache_path=None) -> tuple:
    """(return code, (grid multiplier, size-class threshold, tile edge)) of the C call of the same name."""
    chosen = (ctypes.c_int * 3)()
    path = None if cache_path is None else os.fsencode(cache_path)
    rc = load_library().cdp_autotune(ctx, ctypes.byref(prob), int(precision), path, chosen)
    return rc, tuple(int(v) for v in chosen)


def _i3(v):
    a = (ctypes.c_int32 * 3)()
    for i, x in enumerate(v):
        a[i] = int(x)
    return a


def _d3(v):
    a = (ctypes.c_double * 3)()
    for i, x in enumerate(v):
        a[i] = float(x)
    return a


def _p3(ts):
    a = (ctypes.c_void_p * 3)()
    for i, t in enumerate(ts):
        a[i] = t.data_ptr() if t is not None else None
    return a


def cdp_project_batched(ctx, probs, precision: int, stream: int = 0) -> int:
    arr = (cdp_problem * len(probs))(*probs)
    return load_library().cdp_project_batched(ctx, arr, len(probs), int(precision), ctypes.c_void_p(stream))


# largest vertex and simplex counts of cdp_project_noalloc (its static device scratch)
CDP_NOALLOC_MAX_VERTS = 262144
CDP_NOALLOC_MAX_SIMPLICES = 1572864


def cdp_project_noalloc(prob: cdp_problem, precision: int, accumulate: int = 0, error_flags_ptr: int = 0,
                        stream: int = 0) -> int:
    """Projection on the current device with library-owned static scratch (no allocation)."""
    return load_library().cdp_project_noalloc(ctypes.byref(prob), int(precision), int(accumulate),
                                              ctypes.c_void_p(error_flags_ptr), ctypes.c_void_p(stream))


def cdp_vertex_density(ctx, prob: cdp_problem, simplex_mass_ptr: int, rho_out_ptr: int, stream: int = 0) -> int:
    return load_library().cdp_vertex_density(ctx, ctypes.byref(prob), ctypes.c_void_p(simplex_mass_ptr),
                                             ctypes.c_void_p(rho_out_ptr), ctypes.c_void_p(stream))


def cdp_poisson(ctx, dim, grid, box_len, four_pi_G, mass_ptr, phi_ptr, stream: int = 0) -> int:
    return load_library().cdp_poisson(ctx, int(dim), _i3(grid), _d3(box_len), float(four_pi_G),
                                      ctypes.c_void_p(mass_ptr), ctypes.c_void_p(phi_ptr), ctypes.c_void_p(stream))


def cdp_force(ctx, dim, grid, box_lo, box_len, phi_ptr, n, pos, acc, stream: int = 0) -> int:
    return load_library().cdp_force(ctx, int(dim), _i3(grid), _d3(box_lo), _d3(box_len), ctypes.c_void_p(phi_ptr),
                                    int(n), _p3(pos), _p3(acc), ctypes.c_void_p(stream))


def cdp_drift(ctx, dim, n, pos, vel, dt, box_lo, box_len, periodic, stream: int = 0) -> int:
    return load_library().cdp_drift(ctx, int(dim), int(n), _p3(pos), _p3(vel), float(dt), _d3(box_lo),
                                    _d3(box_len), int(bool(periodic)), ctypes.c_void_p(stream))


def cdp_kick(ctx, dim, n, vel, acc, dt, stream: int = 0) -> int:
    return load_library().cdp_kick(ctx, int(dim), int(n), _p3(vel), _p3(acc), float(dt), ctypes.c_void_p(stream))


def cdp_step_batched(ctx, steps, precision: int, dt: float, four_pi_G: float, use_graph: bool,
                     stream: int = 0) -> int:
    """steps: a ctypes array (or list) of cdp_step_problem; keep the same array object to replay a graph."""
    if not isinstance(steps, ctypes.Array):
        steps = (cdp_step_problem * len(steps))(*steps)
    return load_library().cdp_step_batched(ctx, steps, len(steps), int(precision), float(dt), float(four_pi_G),
                                           int(bool(use_graph)), ctypes.c_void_p(stream))


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Projector:
    """Owns one library context on a CUDA device and projects meshes held in torch tensors.

    pos: float64 tensor [D, Nv] (or a list of D tensors), simplices: int32 [Ns, D+1],
    rho: float64 [Nv], all on the context's device, contiguous. Output: float64 tensor shaped
    ``grid`` (new, or ``out`` when given).
    """

    def __init__(self, device: int = 0):
        self.device = int(device)
        self._ctx = cdp_create(self.device)

    def close(self):
        if self._ctx is not None:
            cdp_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def make_problem(pos, simplices, rho, grid, box_lo, box_len, periodic, out) -> cdp_problem:
        import torch

        dim = len(grid)
        p = cdp_problem()
        p.dim = dim
        rows = [pos[a] for a in range(dim)]
        for a in range(dim):
            t = rows[a]
            if t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("pos rows must be contiguous float64")
            p.pos[a] = t.data_ptr()
        if simplices.dtype != torch.int32 or not simplices.is_contiguous() or simplices.dim() != 2 \
                or simplices.shape[1] != dim + 1:
            raise ValueError("simplices must be a contiguous int32 [Ns, D+1] tensor")
        if rho.dtype != torch.float64 or not rho.is_contiguous():
            raise ValueError("rho must be contiguous float64")
        if out.dtype != torch.float64 or not out.is_contiguous() or tuple(out.shape) != tuple(grid):
            raise ValueError("out must be a contiguous float64 tensor shaped like the grid")
        p.n_verts = int(rho.numel())
        p.n_simplices = int(simplices.shape[0])
        p.simplices = simplices.data_ptr() if simplices.numel() else None
        p.rho = rho.data_ptr() if rho.numel() else None
        for a in range(dim):
            p.grid[a] = int(grid[a])
            p.box_lo[a] = float(box_lo[a])
            p.box_len[a] = float(box_len[a])
        p.periodic = 1 if periodic else 0
        p.cell_mass = out.data_ptr()
        return p

    def project(self, pos, simplices, rho, grid, box_lo=None, box_len=None, periodic=True,
                precision=CDP_FP32_MIXED, out=None, accumulate=False, stream=None, stats=False):
        import torch

        dim = len(grid)
        box_lo = box_lo if box_lo is not None else (0.0,) * dim
        box_len = box_len if box_len is not None else (1.0,) * dim
        if out is None:
            out = torch.empty(tuple(grid), dtype=torch.float64, device=f"cuda:{self.device}")
        prob = self.make_problem(pos, simplices, rho, grid, box_lo, box_len, periodic, out)
        st = cdp_stats() if stats else None
        rc = cdp_project(self._ctx, prob, precision, int(bool(accumulate)), _stream_handle(stream), st)
        _raise(rc, "cdp_project")
        if stats:
            return out, st.as_dict()
        return out

    def project_amr(self, pos, simplices, rho, grid, max_level, box_lo=None, box_len=None, periodic=True,
                    precision=CDP_FP32_MIXED, out=None, accumulate=False, stream=None, stats=False):
        """Projection through the levels 0 .. max_level (grid / 2^level) and donor-cell gather onto
        `grid` (cdp_project_amr)."""
        import torch

        dim = len(grid)
        box_lo = box_lo if box_lo is not None else (0.0,) * dim
        box_len = box_len if box_len is not None else (1.0,) * dim
        if out is None:
            out = torch.empty(tuple(grid), dtype=torch.float64, device=f"cuda:{self.device}")
        prob = self.make_problem(pos, simplices, rho, grid, box_lo, box_len, periodic, out)
        st = cdp_stats() if stats else None
        rc = cdp_project_amr(self._ctx, prob, precision, int(max_level), int(bool(accumulate)),
                             _stream_handle(stream), st)
        _raise(rc, "cdp_project_amr")
        if stats:
            return out, st.as_dict()
        return out

    def check(self, stream=None):
        _raise(cdp_check(self._ctx, _stream_handle(stream)), "cdp_check")

    def autotune(self, pos, simplices, rho, grid, box_lo=None, box_len=None, periodic=True,
                 precision=CDP_FP32_MIXED, out=None, cache_path=None):
        """Tune the launch shape of this context on the given problem (its projection is written into
        `out`); returns (grid multiplier, size-class threshold, tile edge)."""
        import torch

        dim = len(grid)
        box_lo = box_lo if box_lo is not None else (0.0,) * dim
        box_len = box_len if box_len is not None else (1.0,) * dim
        if out is None:
            out = torch.empty(tuple(grid), dtype=torch.float64, device=f"cuda:{self.device}")
        prob = self.make_problem(pos, simplices, rho, grid, box_lo, box_len, periodic, out)
        rc, chosen = cdp_autotune(self._ctx, prob, precision, cache_path)
        _raise(rc, "cdp_autotune")
        return chosen

    def timing(self, enable=None):
        """Enable/disable per-kernel timing, or (enable=None) read the totals."""
        if enable is None:
            return cdp_timing_read(self._ctx)
        _raise(cdp_timing_enable(self._ctx, enable), "cdp_timing_enable")
