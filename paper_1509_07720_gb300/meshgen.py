"""Seeded synthetic inputs: simplicial meshes, displacements and vertex densities.

This module only SYNTHESISES inputs. It holds none of the projection arithmetic and is shared by
the CUDA path's tests/benchmark and by the CPU oracle's tests, so both always see the same data.

The meshes follow the structure of the paper's runs (Sect. 4.1, initial conditions): a regular
simplicial tessellation of the Lagrangian (u = 0) sheet of a periodic box, whose vertices are then
moved by a smooth displacement field, with a per-vertex density.

* 3D: every Lagrangian cube is split into 6 tetrahedra (Kuhn/Freudenthal split: for each
  permutation pi of the axes, {c, c+e_pi1, c+e_pi1+e_pi2, c+(1,1,1)}); it is translation
  invariant, hence conforming on the torus.
* 2D: every Lagrangian square is split along its (0,0)-(1,1) diagonal into 2 triangles.
* Displacements: two orthogonal sine waves (the paper's 2-sine test, Sect. 5.1), or a seeded
  curl-free Gaussian random field psi = grad(phi) whose power spectrum is proportional to k^-2
  for 0 < |k| <= kmax (k in units of the fundamental mode), scaled to a stated rms.
* Densities: uniform, or lognormal rho = exp(sigma * z), z ~ N(0, 1).

All random numbers come from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

__all__ = [
    "Mesh",
    "kuhn_mesh_3d",
    "kuhn_box_mesh_3d",
    "square_box_mesh_2d",
    "square_mesh_2d",
    "sine_displacement_2d",
    "grf_displacement",
    "lognormal_density",
    "make_config",
    "random_simplices",
    "CONFIG_NAMES",
    "smooth_field_3d",
    "bisection_levels",
    "bisect_mesh",
    "StepProblem",
    "simplex_volumes",
    "make_batch",
    "cfl_dt",
    "quantize_positions",
    "shift_mesh",
    "permute_vertex_order",
    "stratified_subset",
    "degenerate_meshes",
    "isolated_simplices",
    "mixed_size_simplices",
    "concat_meshes",
]


@dataclasses.dataclass
class Mesh:
    """One projection problem: a simplicial mesh with per-vertex density and a target grid.

    pos       : float64 [D, Nv]  vertex positions (world units), SoA
    simplices : int32   [Ns, D+1] vertex indices per simplex
    rho       : float64 [Nv]     per-vertex density
    grid      : tuple of D ints  cells per axis (axis 0 slowest in the output array)
    box_lo    : tuple of D floats
    box_len   : tuple of D floats
    periodic  : bool
    """

    pos: np.ndarray
    simplices: np.ndarray
    rho: np.ndarray
    grid: tuple
    box_lo: tuple
    box_len: tuple
    periodic: bool = True
    name: str = ""

    @property
    def dim(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_verts(self) -> int:
        return int(self.pos.shape[1])

    @property
    def n_simplices(self) -> int:
        return int(self.simplices.shape[0])

    def subset(self, idx) -> "Mesh":
        """Same vertices, only the simplices listed in ``idx``."""
        return dataclasses.replace(self, simplices=np.ascontiguousarray(self.simplices[idx]))


# --------------------------------------------------------------------------------------------
# Tessellations of the periodic Lagrangian lattice
# --------------------------------------------------------------------------------------------

def kuhn_mesh_3d(n: int):
    """Periodic n^3 lattice, 6 tetrahedra per cube. Returns (q [3, n^3] in [0,1), tets [6n^3, 4])."""
    idx = np.arange(n, dtype=np.int64)
    i, j, k = np.meshgrid(idx, idx, idx, indexing="ij")
    q = np.stack([i.ravel(), j.ravel(), k.ravel()]).astype(np.float64) / n

    def vid(a, b, c):
        return ((a % n) * n + (b % n)) * n + (c % n)

    ci, cj, ck = i.ravel(), j.ravel(), k.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        off = np.zeros(3, dtype=np.int64)
        verts = [vid(ci, cj, ck)]
        for ax in perm[:2]:
            off[ax] += 1
            verts.append(vid(ci + off[0], cj + off[1], ck + off[2]))
        verts.append(vid(ci + 1, cj + 1, ck + 1))
        tets.append(np.stack(verts, axis=1))
    # cube-major order: the 6 tetrahedra of one cube are adjacent in memory
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return q, tets


def kuhn_box_mesh_3d(n: int):
    """Non-periodic n^3 cubes over [0,1]^3 ((n+1)^3 vertices), 6 tetrahedra per cube."""
    m = n + 1
    idx = np.arange(m, dtype=np.int64)
    i, j, k = np.meshgrid(idx, idx, idx, indexing="ij")
    q = np.stack([i.ravel(), j.ravel(), k.ravel()]).astype(np.float64) / n
    c = np.arange(n, dtype=np.int64)
    ci, cj, ck = (a.ravel() for a in np.meshgrid(c, c, c, indexing="ij"))

    def vid(a, b, cc):
        return (a * m + b) * m + cc

    tets = []
    for perm in itertools.permutations(range(3)):
        off = np.zeros(3, dtype=np.int64)
        verts = [vid(ci, cj, ck)]
        for ax in perm[:2]:
            off[ax] += 1
            verts.append(vid(ci + off[0], cj + off[1], ck + off[2]))
        verts.append(vid(ci + 1, cj + 1, ck + 1))
        tets.append(np.stack(verts, axis=1))
    return q, np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)


def square_box_mesh_2d(n: int):
    """Non-periodic n^2 squares over [0,1]^2 ((n+1)^2 vertices), 2 triangles per square."""
    m = n + 1
    idx = np.arange(m, dtype=np.int64)
    i, j = np.meshgrid(idx, idx, indexing="ij")
    q = np.stack([i.ravel(), j.ravel()]).astype(np.float64) / n
    c = np.arange(n, dtype=np.int64)
    ci, cj = (a.ravel() for a in np.meshgrid(c, c, indexing="ij"))

    def vid(a, b):
        return a * m + b

    t0 = np.stack([vid(ci, cj), vid(ci + 1, cj), vid(ci + 1, cj + 1)], axis=1)
    t1 = np.stack([vid(ci, cj), vid(ci + 1, cj + 1), vid(ci, cj + 1)], axis=1)
    return q, np.stack([t0, t1], axis=1).reshape(-1, 3).astype(np.int32)


def square_mesh_2d(n: int):
    """Periodic n^2 lattice, 2 triangles per square. Returns (q [2, n^2], tris [2n^2, 3])."""
    idx = np.arange(n, dtype=np.int64)
    i, j = np.meshgrid(idx, idx, indexing="ij")
    q = np.stack([i.ravel(), j.ravel()]).astype(np.float64) / n

    def vid(a, b):
        return (a % n) * n + (b % n)

    ci, cj = i.ravel(), j.ravel()
    t0 = np.stack([vid(ci, cj), vid(ci + 1, cj), vid(ci + 1, cj + 1)], axis=1)
    t1 = np.stack([vid(ci, cj), vid(ci + 1, cj + 1), vid(ci, cj + 1)], axis=1)
    tris = np.stack([t0, t1], axis=1).reshape(-1, 3).astype(np.int32)
    return q, tris


# --------------------------------------------------------------------------------------------
# Displacement fields and densities
# --------------------------------------------------------------------------------------------

def sine_displacement_2d(q: np.ndarray, a1: float, a2: float) -> np.ndarray:
    """x = q_x + a1 sin(2 pi q_x), y = q_y + a2 sin(2 pi q_y) (two orthogonal sine waves)."""
    x = q.copy()
    x[0] += a1 * np.sin(2 * np.pi * q[0])
    x[1] += a2 * np.sin(2 * np.pi * q[1])
    return x


def grf_displacement(n: int, dim: int, rms_cells: float, kmax: float, rng) -> np.ndarray:
    """Curl-free Gaussian random displacement on the n^dim Lagrangian lattice.

    psi = grad(phi); |psi_k|^2 proportional to k^-2 for 0 < |k| <= kmax, zero above (spherical
    cutoff, k in units of the fundamental). White noise comes from ``rng``. The field is scaled so
    that rms |psi| over the vertices equals ``rms_cells`` Lagrangian cells (cell = 1/n).
    Returns psi as [dim, n^dim] (box units).
    """
    shape = (n,) * dim
    white = rng.standard_normal(shape)
    wk = np.fft.rfftn(white)
    freqs = [np.fft.fftfreq(n, d=1.0 / n)] * (dim - 1) + [np.fft.rfftfreq(n, d=1.0 / n)]
    kv = np.meshgrid(*freqs, indexing="ij")
    k2 = sum(kk * kk for kk in kv)
    k = np.sqrt(k2)
    amp = np.zeros_like(k)
    sel = (k > 0) & (k <= kmax)
    amp[sel] = 1.0 / k2[sel]  # |phi_k|^2 ~ k^-4  =>  |psi_k|^2 ~ k^-2
    phik = wk * amp
    psi = np.empty((dim,) + shape)
    for a in range(dim):
        psi[a] = np.fft.irfftn(1j * 2 * np.pi * kv[a] * phik, s=shape, axes=tuple(range(dim)))
    psi = psi.reshape(dim, -1)
    rms = math.sqrt(float(np.mean(np.sum(psi * psi, axis=0))))
    if rms > 0:
        psi *= (rms_cells / n) / rms
    return psi


def lognormal_density(nv: int, sigma: float, rng) -> np.ndarray:
    """rho = exp(sigma z), z ~ N(0,1) (median 1)."""
    return np.exp(sigma * rng.standard_normal(nv))


# --------------------------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------------------------

CONFIG_NAMES = {
    "c1a": "2D 64^2 Lagrangian squares (8192 triangles), two sine waves a=(0.15, 0.10), rho=1, 128^2 grid",
    "c1b": "2D 64^2 Lagrangian squares (8192 triangles), two sine waves a=(0.45, 0.30) (folded), rho=1, 128^2 grid",
    "c2": "3D 32^3 Kuhn cubes (196,608 tets), GRF k^-2 k<=16 rms 0.5 cell, rho=1, 128^3 grid",
    "c3": "3D 128^3 Kuhn cubes (12,582,912 tets), GRF k^-2 k<=16 rms 4 cells, lognormal rho sigma=0.5, 256^3 grid",
    "c4": "3D undisplaced 64^3 Kuhn base bisected along longest edges to 50,331,953 tets (levels 0-14, "
          "volumes over 4 decades), lognormal rho sigma=1, 512^3 grid",
}


def _wrap(x: np.ndarray) -> np.ndarray:
    return x - np.floor(x)


def smooth_field_3d(pts: np.ndarray, rng, kmax: int = 3) -> np.ndarray:
    """A seeded smooth periodic field at points [3, N] of the unit box: a sum of the Fourier modes
    0 < |k| <= kmax with Gaussian amplitudes and uniform phases."""
    out = np.zeros(pts.shape[1])
    r = np.arange(-kmax, kmax + 1)
    for kx in r:
        for ky in r:
            for kz in r:
                k2 = kx * kx + ky * ky + kz * kz
                if k2 == 0 or k2 > kmax * kmax:
                    continue
                amp = rng.standard_normal() / k2
                ph = rng.uniform(0.0, 2.0 * np.pi)
                out += amp * np.cos(2.0 * np.pi * (kx * pts[0] + ky * pts[1] + kz * pts[2]) + ph)
    return out


def bisection_levels(field: np.ndarray, target: int, max_level: int = 13, spread: float = 4.0) -> np.ndarray:
    """Refinement level of every base simplex, floor(c + spread z) clipped to [0, max_level] with z
    the standardised field; c is the smallest offset (bisection search) for which the refined
    count sum(2^level) reaches ``target``."""
    z = (field - field.mean()) / field.std()

    def levels(c):
        return np.clip(np.floor(c + spread * z), 0, max_level).astype(np.int64)

    lo, hi = -4.0 * spread, float(max_level) + 4.0 * spread
    if int(np.sum(1 << levels(hi))) < target:
        raise ValueError("target count out of reach")
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if int(np.sum(1 << levels(mid))) >= target:
            hi = mid
        else:
            lo = mid
    return levels(hi)


def bisect_mesh(q: np.ndarray, tets: np.ndarray, levels: np.ndarray):
    """Non-conforming longest-edge bisection on the periodic unit box.  Base tetrahedron b is split
    levels[b] times: each split cuts a tetrahedron through the midpoint of its longest edge (ties to
    the first edge in the order (0,1), (0,2), (0,3), (1,2), (1,3), (2,3)) into two children, and
    every split makes its own midpoint vertex (hanging nodes are allowed).  Returns
    (positions [3, Nv] in [0, 1), tetrahedra [Ns, 4] int32, number of base vertices)."""
    nbase = q.shape[1]
    total_new = int(np.sum((1 << levels.astype(np.int64)) - 1))
    pos = np.empty((3, nbase + total_new))
    pos[:, :nbase] = q
    nv = nbase
    done = []
    cur = tets.astype(np.int64)
    lev = levels.astype(np.int64)
    ea = np.array([0, 0, 0, 1, 1, 2])
    eb = np.array([1, 2, 3, 2, 3, 3])
    # the two vertices off each edge
    ep = np.array([2, 1, 1, 0, 0, 0])
    eq = np.array([3, 3, 2, 3, 2, 1])
    while cur.shape[0]:
        split = lev > 0
        done.append(cur[~split])
        t = cur[split]
        left = lev[split] - 1
        if t.shape[0] == 0:
            break
        x = pos[:, t]                           # [3, n, 4]
        d = x - x[:, :, :1]
        d -= np.round(d)                        # minimal image relative to vertex 0
        xu = x[:, :, :1] + d
        e2 = np.stack([np.sum((xu[:, :, eb[e]] - xu[:, :, ea[e]]) ** 2, axis=0) for e in range(6)], axis=1)
        e = np.argmax(e2, axis=1)
        rows = np.arange(t.shape[0])
        a, b = t[rows, ea[e]], t[rows, eb[e]]
        p, r = t[rows, ep[e]], t[rows, eq[e]]
        mid = 0.5 * (xu[:, rows, ea[e]] + xu[:, rows, eb[e]])
        m = np.arange(nv, nv + t.shape[0])
        pos[:, m] = _wrap(mid)
        nv += t.shape[0]
        c1 = np.stack([a, m, p, r], axis=1)
        c2 = np.stack([m, b, p, r], axis=1)
        cur = np.concatenate([c1, c2])
        lev = np.concatenate([left, left])
    out = np.concatenate(done).astype(np.int32)
    return pos[:, :nv], out, nbase


def make_config(name: str, scale: int | None = None) -> Mesh:
    """Build one named workload.

    c1a/c1b: 2D sine-wave meshes; c2/c3: 3D random-field meshes; c4: a bisected (adaptive) 3D mesh.
    ``scale`` overrides the Lagrangian lattice size n (the grid keeps the same ratio to n), for
    reduced test cases.
    """
    if name in ("c1a", "c1b"):
        n = scale or 64
        q, tris = square_mesh_2d(n)
        a1, a2 = (0.15, 0.10) if name == "c1a" else (0.45, 0.30)
        x = _wrap(sine_displacement_2d(q, a1, a2))
        rho = np.ones(q.shape[1])
        g = 2 * n
        return Mesh(x, tris, rho, (g, g), (0.0, 0.0), (1.0, 1.0), True, name)
    if name == "c2":
        n = scale or 32
        rng = np.random.default_rng(1002)
        q, tets = kuhn_mesh_3d(n)
        x = _wrap(q + grf_displacement(n, 3, 0.5, 16.0, rng))
        rho = np.ones(q.shape[1])
        g = 4 * n
        return Mesh(x, tets, rho, (g, g, g), (0.0,) * 3, (1.0,) * 3, True, name)
    if name == "c3":
        n = scale or 128
        rng = np.random.default_rng(1003)
        q, tets = kuhn_mesh_3d(n)
        x = _wrap(q + grf_displacement(n, 3, 4.0, 16.0, rng))
        rho = lognormal_density(q.shape[1], 0.5, rng)
        g = 2 * n
        return Mesh(x, tets, rho, (g, g, g), (0.0,) * 3, (1.0,) * 3, True, name)
    if name == "c4":
        # undisplaced n^3 Kuhn base (vertices on grid nodes and planes), bisected to 32x the base
        # count with refinement levels 0..14 (volumes over 4 decades) set by a smooth seeded field,
        # lognormal(1) densities
        n = scale or 64
        rng = np.random.default_rng(1004)
        q, tets = kuhn_mesh_3d(n)
        # base centroids, at the minimal image of vertex 0
        x = q[:, tets]
        d = x - x[:, :, :1]
        d -= np.round(d)
        cen = _wrap(x[:, :, 0] + d.mean(axis=2))
        lev = bisection_levels(smooth_field_3d(cen, rng), 32 * tets.shape[0], max_level=14, spread=7.0)
        pos, t2, _ = bisect_mesh(q, tets, lev)
        rho = lognormal_density(pos.shape[1], 1.0, rng)
        g = 8 * n
        return Mesh(pos, t2, rho, (g, g, g), (0.0,) * 3, (1.0,) * 3, True, name)
    raise ValueError(f"unknown workload {name!r}")


@dataclasses.dataclass
class StepProblem:
    """One problem of the batched time step: the mesh (rho is recomputed by the step from the
    simplex masses), vertex velocities [D, Nv] (box units per time) and simplex masses [Ns]."""

    mesh: Mesh
    vel: np.ndarray
    masses: np.ndarray


def simplex_volumes(mesh: Mesh) -> np.ndarray:
    """|V| of every simplex at the minimal image of its vertex 0 (world units)."""
    p = mesh.pos[:, mesh.simplices]
    e = p[:, :, 1:] - p[:, :, :1]
    L = np.asarray(mesh.box_len, dtype=np.float64)[:, None, None]
    e -= np.round(e / L) * L
    if mesh.dim == 3:
        return np.abs(np.einsum("in,in->n", e[:, :, 0], np.cross(e[:, :, 1].T, e[:, :, 2].T).T)) / 6.0
    return np.abs(e[0, :, 0] * e[1, :, 1] - e[1, :, 0] * e[0, :, 1]) / 2.0


def make_batch(name: str = "c5", count: int = 64, ns_range=(1e3, 2e6)) -> list:
    """The batched workload: ``count`` independent problems, dimension alternating 3D / 2D, simplex
    counts log-uniform in ``ns_range`` (rounded to a Lagrangian lattice), grids drawn from
    {64, 128, 256}^D, seeded GRF (3D, rms 0.5 Lagrangian cell) or two-sine (2D) displacements.
    Every simplex carries the mass of a unit density over its displaced volume, and the vertices
    move with the displacement itself as velocity (growth rate 1), so the step's densities start
    near 1 where the sheet is single-stream."""
    if name != "c5":
        raise ValueError(f"unknown batch {name!r}")
    rng = np.random.default_rng(1005)
    out = []
    for i in range(count):
        dim = 3 if i % 2 == 0 else 2
        ns = math.exp(rng.uniform(math.log(ns_range[0]), math.log(ns_range[1])))
        g = int(rng.choice([64, 128, 256]))
        if dim == 3:
            n = max(2, int(round((ns / 6.0) ** (1.0 / 3.0))))
            q, simp = kuhn_mesh_3d(n)
            psi = grf_displacement(n, 3, 0.5, 16.0, rng)
        else:
            n = max(2, int(round(math.sqrt(ns / 2.0))))
            q, simp = square_mesh_2d(n)
            a1, a2 = rng.uniform(0.02, 0.12, size=2)
            psi = sine_displacement_2d(q, a1, a2) - q
        x = _wrap(q + psi)
        mesh = Mesh(x, simp, np.ones(x.shape[1]), (g,) * dim, (0.0,) * dim, (1.0,) * dim, True, f"c5[{i}]")
        out.append(StepProblem(mesh, np.ascontiguousarray(psi), simplex_volumes(mesh)))
    return out


def cfl_dt(problems, courant: float = 0.25) -> float:
    """Common time step: courant x (smallest cell) / (largest vertex speed), 1e-3 if all are at rest."""
    vmax = max(float(np.max(np.abs(p.vel))) for p in problems)
    h = min(min(p.mesh.box_len[a] / p.mesh.grid[a] for a in range(p.mesh.dim)) for p in problems)
    return courant * h / vmax if vmax > 0 else 1e-3


def random_simplices(dim: int, ns: int, grid: int, size: float, rng, periodic: bool = True,
                     rho_sigma: float = 0.5) -> Mesh:
    """``ns`` independent random simplices (each with its own D+1 vertices) in a unit box.

    Vertex 0 is uniform in the box; the others are vertex 0 plus uniform offsets in
    [-size, size] grid cells. Used for small parity and stress cases.
    """
    h = 1.0 / grid
    v0 = rng.random((dim, ns))
    offs = (rng.random((dim, ns, dim)) * 2 - 1) * size * h
    pos = np.empty((dim, ns * (dim + 1)))
    pos[:, 0::dim + 1] = v0
    for i in range(dim):
        pos[:, i + 1::dim + 1] = v0 + offs[:, :, i]
    if periodic:
        pos = _wrap(pos)
    simp = np.arange(ns * (dim + 1), dtype=np.int32).reshape(ns, dim + 1)
    rho = lognormal_density(ns * (dim + 1), rho_sigma, rng) if rho_sigma > 0 else np.ones(ns * (dim + 1))
    return Mesh(pos, simp, rho, (grid,) * dim, (0.0,) * dim, (1.0,) * dim, periodic, "random")


# --------------------------------------------------------------------------------------------
# Degenerate and transformed inputs (parity edge cases)
# --------------------------------------------------------------------------------------------

def _dyadic(v, bits: int):
    """v rounded to a multiple of 2^-bits (exactly representable, and exact under shifts by
    multiples of 2^-bits that stay in range)."""
    return np.round(np.asarray(v, dtype=np.float64) * (1 << bits)) / float(1 << bits)


def quantize_positions(mesh: Mesh, bits: int = 30) -> Mesh:
    """The mesh with every coordinate rounded to a multiple of 2^-bits box lengths (unit box)."""
    return dataclasses.replace(mesh, pos=np.ascontiguousarray(_wrap(_dyadic(mesh.pos, bits))))


def shift_mesh(mesh: Mesh, cells) -> Mesh:
    """The periodic unit-box mesh translated by an integer number of grid cells per axis (exact for
    dyadic coordinates and power-of-two grids)."""
    off = np.array([c / g for c, g in zip(cells, mesh.grid)], dtype=np.float64)[:, None]
    return dataclasses.replace(mesh, pos=np.ascontiguousarray(_wrap(mesh.pos + off)))


def permute_vertex_order(mesh: Mesh, rng) -> Mesh:
    """The same simplices with the vertex indices of each one listed in a random order (even and
    odd permutations alike)."""
    d1 = mesh.simplices.shape[1]
    keys = rng.random(mesh.simplices.shape)
    order = np.argsort(keys, axis=1)
    simp = np.take_along_axis(mesh.simplices, order, axis=1)
    return dataclasses.replace(mesh, simplices=np.ascontiguousarray(simp.astype(np.int32)))


def stratified_subset(mesh: Mesh, fraction_inv: int, rng) -> Mesh:
    """About 1/fraction_inv of the simplices, drawn at random within each volume class (classes =
    rounded log2 of the volume below the largest), so that every refinement level is represented."""
    vol = simplex_volumes(mesh)
    vmax = float(vol.max()) if vol.size else 1.0
    cls = np.round(np.log2(vmax / np.maximum(vol, vmax * 2.0 ** -60))).astype(np.int64)
    idx = []
    for c in np.unique(cls):
        ii = np.flatnonzero(cls == c)
        k = (ii.size + fraction_inv - 1) // fraction_inv
        idx.append(rng.choice(ii, k, replace=False))
    idx = np.sort(np.concatenate(idx)) if idx else np.zeros(0, dtype=np.int64)
    return mesh.subset(idx)


def _assemble(dim, groups, grid, rng, periodic=True, rho_sigma=0.5):
    """Mesh from a list of simplices given by their vertex coordinates ([n, D+1, D] arrays in box
    units) plus index-level degeneracies: each group is (coords, index_pattern) where
    index_pattern (or None) rewrites the simplex's index row, e.g. (0, 0, 1, 2) repeats vertex 0."""
    pos_list, simp_list, nv = [], [], 0
    for coords, pattern in groups:
        n = coords.shape[0]
        pos_list.append(coords.reshape(n * (dim + 1), dim).T)
        base = nv + (dim + 1) * np.arange(n)[:, None]
        rows = base + np.arange(dim + 1)[None, :]
        if pattern is not None:
            rows = base + np.asarray(pattern)[None, :]
        simp_list.append(rows)
        nv += n * (dim + 1)
    pos = np.concatenate(pos_list, axis=1)
    if periodic:
        pos = _wrap(pos)
    simp = np.concatenate(simp_list).astype(np.int32)
    rho = lognormal_density(nv, rho_sigma, rng)
    return Mesh(np.ascontiguousarray(pos), np.ascontiguousarray(simp), rho, (grid,) * dim, (0.0,) * dim,
                (1.0,) * dim, periodic, "degenerate")


def degenerate_meshes(dim: int, grid: int, rng) -> dict:
    """Named meshes of the degenerate configurations the method must handle (Sect. 3.3), each as
    (mesh, number of zero-volume simplices it contains by construction):

      zero_volume  generic simplices mixed with flat ones on dyadic coordinates (all vertices on
                   one plane in 3D, one line in 2D: exactly flat after the fixed-point conversion),
                   simplices naming one vertex twice, simplices with two distinct vertices at one
                   position, and (3D) simplices with three collinear vertices
      slivers      nearly flat simplices: a flat dyadic base and an apex 2^-30 or 1.3e-7 cells off
                   its plane (line), and needles with nearly collinear vertices
      grid_planes  simplices with a facet (3D) / an edge (2D) exactly in a grid plane (line) at
                   off-lattice positions, in pairs on both sides of that plane
      grid_lines   3D: simplices with an edge exactly along a grid line at off-lattice positions,
                   and facets through a grid node; 2D: vertices on grid lines and nodes, and edges
                   through a grid node
    Coordinates are in the periodic unit box with `grid` cells per axis (a power-of-two grid keeps
    the dyadic coordinates exact in grid units)."""
    h = 1.0 / grid
    D = dim

    def generic(n, size):
        # vertex 0 uniform in the box, the others within `size` cells of it
        v0 = rng.random((n, 1, D))
        return np.concatenate([v0, v0 + (rng.random((n, D, D)) * 2 - 1) * size * h], axis=1)

    def on_hyperplane(n, m, size):
        # m points per simplex on the hyperplane x_{D-1} = c + slope . (x_0 .. x_{D-2}), with a
        # dyadic anchor c, dyadic slopes and dyadic in-plane offsets: the coordinates are exact
        anchor = _dyadic(rng.random((n, 1, D)), 12)
        slope = _dyadic(rng.uniform(-1, 1, (n, 1, D - 1)), 3)
        t = _dyadic((rng.random((n, m, D - 1)) * 2 - 1) * size * h, 12)
        pts = np.empty((n, m, D))
        pts[:, :, :D - 1] = anchor[:, :, :D - 1] + t
        pts[:, :, D - 1] = anchor[:, :, D - 1] + np.sum(slope * t, axis=2)
        return pts

    out = {}
    # ---- zero volume
    groups = [(generic(40, 3.0), None), (on_hyperplane(20, D + 1, 3.0), None)]
    groups.append((generic(10, 2.5), (0, 0) + tuple(range(1, D))))    # vertex 0 named twice
    same = generic(10, 2.5)
    same[:, 1] = same[:, 0]                                           # two vertices at one position
    groups.append((same, None))
    nzero = 40
    if D == 3:
        col = _dyadic(generic(10, 2.5), 12)
        col[:, 2] = col[:, 0] + 0.5 * (col[:, 1] - col[:, 0])          # midpoint of edge 01: exact
        groups.append((col, None))
        nzero += 10
    out["zero_volume"] = (_assemble(D, groups, grid, rng), nzero)
    # ---- slivers
    s_groups = [(generic(20, 3.0), None)]
    for height in (2.0 ** -30, 1.3e-7):
        base = on_hyperplane(30, D, 3.0)
        apex = base.mean(axis=1, keepdims=True)
        apex[:, :, D - 1] += height * h
        s_groups.append((np.concatenate([base, apex], axis=1), None))
    nd = generic(30, 4.0)
    nd[:, 2] = nd[:, 0] + (0.5 + 1e-7 * rng.standard_normal((30, D))) * (nd[:, 1] - nd[:, 0])
    s_groups.append((nd, None))                                       # needles
    out["slivers"] = (_assemble(D, s_groups, grid, rng), 0)
    # ---- facets (edges) in grid planes (lines), in pairs on both sides
    g_groups = []
    for ax in range(D):
        n = 20
        face = generic(n, 3.0)[:, :D]
        face[:, :, ax] = rng.integers(0, grid, (n, 1)) * h
        others = [a for a in range(D) if a != ax]
        for side in (1.0, -1.0):
            apex = face.mean(axis=1, keepdims=True)
            apex[:, :, ax] += side * rng.uniform(0.3, 3.0, (n, 1)) * h
            apex[:, :, others] += (rng.random((n, 1, D - 1)) - 0.5) * h
            g_groups.append((np.concatenate([face, apex], axis=1), None))
    out["grid_planes"] = (_assemble(D, g_groups, grid, rng), 0)
    # ---- edges along grid lines and through grid nodes
    l_groups = []
    node = lambda n: rng.integers(0, grid, (n, 1, D)) * h
    if D == 3:
        for ax in range(3):
            n = 20
            edge = np.repeat(node(n), 2, axis=1)
            edge[:, :, ax] = rng.random((n, 1)) + np.array([0.0, 1.0]) * rng.uniform(0.5, 4.0, (n, 1)) * h
            rest = edge.mean(axis=1, keepdims=True) + (rng.random((n, 2, 3)) * 2 - 1) * 2.5 * h
            l_groups.append((np.concatenate([edge, rest], axis=1), None))
        n = 20
        c = node(n)
        u = _dyadic((rng.random((n, 2, 3)) * 2 - 1) * 2.0 * h, 14)
        tri = np.concatenate([c + u[:, :1], c + u[:, 1:], c - u[:, :1] - u[:, 1:]], axis=1)  # centroid on the node
        apex = c + _dyadic((rng.random((n, 1, 3)) * 2 - 1) * 2.0 * h, 14)
        l_groups.append((np.concatenate([tri, apex], axis=1), None))
    else:
        n = 30
        v = generic(n, 3.0)
        v[:, 0, 0] = np.round(v[:, 0, 0] * grid) * h                  # vertex 0 on a grid line
        v[:, 1] = np.round(v[:, 1] * grid) * h                        # vertex 1 on a grid node
        l_groups.append((v, None))
        c = node(n)
        u = _dyadic((rng.random((n, 1, 2)) * 2 - 1) * 2.5 * h, 14)
        w = _dyadic((rng.random((n, 1, 2)) * 2 - 1) * 2.5 * h, 14)
        l_groups.append((np.concatenate([c + u, c - u, c + w], axis=1), None))  # edge 01 through the node
    out["grid_lines"] = (_assemble(D, l_groups, grid, rng), 0)
    return out


def isolated_simplices(dim: int, blocks: int, block_cells: int, rng):
    """One simplex in each cubic block of `block_cells` cells of a (blocks * block_cells)^dim grid
    (unit box, not periodic), so that every block's cells hold the pieces of one simplex only.
    Shapes cycle through five kinds (returned per simplex): 0 generic (edges 1-5 cells), 1 nearly
    flat (an apex 10^-9 .. 1 times the size off the plane of the other vertices), 2 needle-like
    (vertices nearly on a line), 3 a facet nearly parallel to a grid plane, 4 small (under a cell).
    Densities are lognormal with sigma in {0.3, 1, 2} per simplex.  Returns (mesh, kinds, vertex
    coordinates [n, dim + 1, dim] in grid units)."""
    n = blocks ** dim
    grid = blocks * block_cells
    idx = np.stack(np.meshgrid(*[np.arange(blocks)] * dim, indexing="ij"), axis=0).reshape(dim, -1).T
    kind = rng.integers(0, 5, n)
    V = np.zeros((n, dim + 1, dim))
    for i in range(n):
        c = idx[i] * block_cells + block_cells / 2.0 + rng.uniform(-1.5, 1.5, dim)
        k = kind[i]
        size = rng.uniform(1.0, 5.0)
        if k == 0:
            V[i] = c + rng.uniform(-size, size, (dim + 1, dim))
        elif k == 1:
            base = rng.uniform(-size, size, (dim, dim))
            nrm = np.linalg.svd(base - base.mean(0))[2][-1]
            apex = base.mean(0) + rng.uniform(-0.3, 0.3, dim) * size
            apex = apex - np.dot(apex - base[0], nrm) * nrm + nrm * 10.0 ** (-rng.uniform(0, 9)) * size
            V[i] = c + np.vstack([base, apex])
        elif k == 2:
            a = rng.uniform(-size, size, dim)
            b = rng.uniform(-size, size, dim)
            pts = [a, b] + [a + rng.uniform(0.2, 0.8) * (b - a) + 10.0 ** (-rng.uniform(0, 7)) * rng.standard_normal(dim)
                            for _ in range(dim - 1)]
            V[i] = c + np.array(pts)
        elif k == 3:
            ax = rng.integers(0, dim)
            base = rng.uniform(-size, size, (dim, dim))
            base[:, ax] = rng.uniform(-1, 1) + 10.0 ** (-rng.uniform(0, 8)) * rng.standard_normal(dim)
            V[i] = c + np.vstack([base, rng.uniform(-size, size, dim)])
        else:
            V[i] = c + rng.uniform(-0.6, 0.6, (dim + 1, dim))
        lo = idx[i] * block_cells + 0.5
        hi = (idx[i] + 1) * block_cells - 0.5
        if np.any(V[i] < lo) or np.any(V[i] > hi):  # keep every simplex inside its own block
            V[i] = idx[i] * block_cells + block_cells / 2.0 + rng.uniform(-2.0, 2.0, (dim + 1, dim))
            kind[i] = 0
    pos = np.ascontiguousarray((V.reshape(-1, dim) / grid).T)
    simp = np.arange(n * (dim + 1), dtype=np.int32).reshape(n, dim + 1)
    sig = rng.choice([0.3, 1.0, 2.0], n)
    rho = np.exp(np.repeat(sig, dim + 1) * rng.standard_normal(n * (dim + 1)))
    return Mesh(pos, simp, rho, (grid,) * dim, (0.0,) * dim, (1.0,) * dim, False, "isolated"), kind, V


def concat_meshes(meshes) -> Mesh:
    """One mesh holding the simplices of several meshes on the same grid and box (vertices kept
    apart, indices offset)."""
    m0 = meshes[0]
    pos = np.concatenate([m.pos for m in meshes], axis=1)
    offs = np.cumsum([0] + [m.n_verts for m in meshes[:-1]])
    simp = np.concatenate([m.simplices + o for m, o in zip(meshes, offs)]).astype(np.int32)
    rho = np.concatenate([m.rho for m in meshes])
    return Mesh(pos, simp, rho, m0.grid, m0.box_lo, m0.box_len, m0.periodic, "concat")


def mixed_size_simplices(dim: int, grid: int, counts_sizes, rng, periodic: bool = True) -> Mesh:
    """Random simplices of several sizes in one mesh: ``counts_sizes`` = [(count, size in cells), ...]
    as ``random_simplices`` (smallest perpendicular heights spread over the levels of a hierarchy
    of grids)."""
    return concat_meshes([random_simplices(dim, n, grid, s, rng, periodic) for n, s in counts_sizes])

