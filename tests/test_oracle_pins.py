"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test pins the oracle to something other than itself: closed forms of the projection
(Sect. 3.1 volume formula worked on the unit cube/square, Appendix C's first-order result), the
tiling and mass invariants of an exact projection, an independent exact-rational slicing
integrator (``exact_slicing.py``), and Monte Carlo sampling of each simplex (the paper's own
check, Sect. 5.2: random sampling of each simplex with particles).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1509_07720_gb300 import meshgen as mg

import exact_slicing


def _mesh(pos, simp, rho, grid, periodic=True, lo=None, ln=None):
    d = pos.shape[0]
    lo = lo or (0.0,) * d
    ln = ln or (1.0,) * d
    return mg.Mesh(np.ascontiguousarray(pos, dtype=np.float64), np.ascontiguousarray(simp, dtype=np.int32),
                   np.ascontiguousarray(rho, dtype=np.float64), tuple(grid), lo, ln, periodic)


def _smooth_periodic_3d(n=8, grid=12, seed=5):
    rng = np.random.default_rng(seed)
    q, t = mg.kuhn_mesh_3d(n)
    x = q + mg.grf_displacement(n, 3, 0.3, 2.0, rng)
    return _mesh(x - np.floor(x), t, np.ones(q.shape[1]), (grid,) * 3)


def _flipped(mesh, q):
    """Simplices whose orientation differs from the undisplaced lattice (folds)."""
    def sv(pos):
        p = pos[:, mesh.simplices]
        d = p[:, :, 1:] - p[:, :, :1]
        d -= np.round(d)
        if mesh.dim == 3:
            return np.einsum("ij,ij->j", d[:, :, 0], np.cross(d[:, :, 1].T, d[:, :, 2].T).T)
        return d[0, :, 0] * d[1, :, 1] - d[1, :, 0] * d[0, :, 1]
    return int(np.sum(np.sign(sv(mesh.pos)) != np.sign(sv(q))))


# ------------------------------------------------------------------------------------------
# P1 / P2: closed forms on the unit cube and unit square
# ------------------------------------------------------------------------------------------

def test_unit_cube_volume_and_first_moment():
    """Six Kuhn tetrahedra tile the unit cube: volume 1 (rho = 1) and integral of x = 1/2."""
    q, t = mg.kuhn_box_mesh_3d(1)
    m = oracle.project(_mesh(q, t, np.ones(q.shape[1]), (1, 1, 1), periodic=False))
    assert m.shape == (1, 1, 1) and abs(m[0, 0, 0] - 1.0) < 1e-15
    for a in range(3):
        m = oracle.project(_mesh(q, t, q[a], (1, 1, 1), periodic=False))
        assert abs(m[0, 0, 0] - 0.5) < 1e-15


def test_unit_square_area_and_first_moment():
    q, t = mg.square_box_mesh_2d(1)
    m = oracle.project(_mesh(q, t, np.ones(q.shape[1]), (1, 1), periodic=False))
    assert abs(m[0, 0] - 1.0) < 1e-15
    m = oracle.project(_mesh(q, t, q[1], (1, 1), periodic=False))
    assert abs(m[0, 0] - 0.5) < 1e-15


@pytest.mark.parametrize("lag,grid", [(4, 4), (4, 8), (2, 8), (4, 5), (3, 7)])
def test_linear_density_cell_centres_3d(lag, grid):
    """rho = a + b.x on a mesh tiling [0,1]^3: every cell gets h^3 rho(cell centre) exactly
    (the integral of a linear function over a box is its value at the centre times the volume)."""
    q, t = mg.kuhn_box_mesh_3d(lag)
    coef = np.array([1.25, -0.5, 2.0, 0.75])
    rho = coef[0] + coef[1:] @ q
    m = oracle.project(_mesh(q, t, rho, (grid,) * 3, periodic=False))
    h = 1.0 / grid
    c = (np.arange(grid) + 0.5) * h
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    expect = h ** 3 * (coef[0] + coef[1] * X + coef[2] * Y + coef[3] * Z)
    assert np.max(np.abs(m - expect)) <= 1e-14 * np.max(np.abs(expect))


@pytest.mark.parametrize("lag,grid", [(4, 4), (4, 8), (3, 7)])
def test_linear_density_cell_centres_2d(lag, grid):
    q, t = mg.square_box_mesh_2d(lag)
    rho = 0.5 + 1.5 * q[0] - 0.25 * q[1]
    m = oracle.project(_mesh(q, t, rho, (grid, grid), periodic=False))
    h = 1.0 / grid
    c = (np.arange(grid) + 0.5) * h
    X, Y = np.meshgrid(c, c, indexing="ij")
    expect = h * h * (0.5 + 1.5 * X - 0.25 * Y)
    assert np.max(np.abs(m - expect)) <= 1e-14 * np.max(np.abs(expect))


# ------------------------------------------------------------------------------------------
# P3 total mass, P4 single cell, P5 tiling, P6 aligned lattice
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,size,grid", [(2, 0.3, 16), (2, 3.0, 16), (3, 0.4, 16), (3, 2.5, 16), (3, 6.0, 32)])
def test_total_mass(dim, size, grid):
    rng = np.random.default_rng(11 + dim)
    mesh = mg.random_simplices(dim, 300, grid, size, rng)
    m = oracle.project(mesh)
    ref = oracle.simplex_mass(mesh).sum()
    assert abs(m.sum() - ref) <= 1e-13 * ref


def test_total_mass_workloads():
    for name, sc in (("c1b", 32), ("c2", 16)):
        mesh = mg.make_config(name, sc)
        m = oracle.project(mesh)
        ref = oracle.simplex_mass(mesh).sum()
        assert abs(m.sum() - ref) <= 1e-13 * ref


def test_single_cell_simplex():
    """A simplex strictly inside one cell deposits all of its mass there (Algorithm 2, step 1)."""
    pos = np.array([[0.30, 0.32, 0.41, 0.35], [0.55, 0.60, 0.52, 0.58], [0.71, 0.73, 0.74, 0.79]]) / 4 + 0.5
    mesh = _mesh(pos, [[0, 1, 2, 3]], [1.0, 2.0, 3.0, 4.0], (4, 4, 4))
    m = oracle.project(mesh)
    ref = oracle.simplex_mass(mesh)[0]
    cell = tuple(int(np.floor(pos[a, 0] * 4)) for a in range(3))
    assert abs(m[cell] - ref) <= 1e-16 and np.count_nonzero(m) == 1
    # explicit volume from the determinant: |det|/6 * mean(rho)
    d = pos[:, 1:] - pos[:, :1]
    assert abs(ref - abs(np.linalg.det(d)) / 6 * 2.5) <= 1e-15 * ref


def test_tiling_smooth_periodic_3d():
    """An unfolded mesh tiling the periodic box with rho = 1 gives h^3 in every cell."""
    mesh = _smooth_periodic_3d()
    q, _ = mg.kuhn_mesh_3d(8)
    assert _flipped(mesh, q) == 0
    m = oracle.project(mesh)
    assert np.max(np.abs(m * 12 ** 3 - 1.0)) < 1e-13


def test_tiling_bisected_mesh():
    """The bisected adaptive mesh (workload c4 at base 4^3: hanging nodes, volumes over 3-4 decades,
    vertices on grid planes) still partitions the periodic box: with rho = 1 every cell gets h^3,
    and the simplex volumes add up to the box volume."""
    m = mg.make_config("c4", 4)
    ones = mg.Mesh(m.pos, m.simplices, np.ones(m.n_verts), m.grid, m.box_lo, m.box_len, True)
    vol = oracle.simplex_mass(ones)
    assert abs(vol.sum() - 1.0) < 1e-14
    assert vol.max() / vol.min() >= 2 ** 11
    cm = oracle.project(ones)
    assert np.max(np.abs(cm * 32 ** 3 - 1.0)) < 1e-12


def test_bisection_generator_counts():
    """The level rule reaches its target count exactly as sum(2^level), and every split adds one
    vertex and one simplex."""
    q, tets = mg.kuhn_mesh_3d(4)
    rng = np.random.default_rng(3)
    lev = mg.bisection_levels(rng.standard_normal(tets.shape[0]), 8 * tets.shape[0], max_level=6, spread=2.0)
    assert int(np.sum(1 << lev.astype(np.int64))) >= 8 * tets.shape[0]
    pos, t2, nb = mg.bisect_mesh(q, tets, lev)
    assert t2.shape[0] == int(np.sum(1 << lev.astype(np.int64)))
    assert pos.shape[1] - nb == t2.shape[0] - tets.shape[0]
    assert np.all((pos >= 0) & (pos < 1))


def test_tiling_sine_waves_2d():
    """Workload c1a (two sine waves, single stream): h^2 in every cell."""
    mesh = mg.make_config("c1a")
    q, _ = mg.square_mesh_2d(64)
    assert _flipped(mesh, q) == 0
    m = oracle.project(mesh)
    assert np.max(np.abs(m * 128 ** 2 - 1.0)) < 1e-13


def test_folded_sine_waves_multistream():
    """Workload c1b folds: cells are covered by 1, 3 or more streams. The total is the sum of the
    unsigned simplex masses (more than the box volume) and some cell is multi-stream."""
    mesh = mg.make_config("c1b")
    q, _ = mg.square_mesh_2d(64)
    assert _flipped(mesh, q) > 0
    m = oracle.project(mesh)
    ref = oracle.simplex_mass(mesh).sum()
    assert abs(m.sum() - ref) <= 1e-13 * ref and ref > 1.5
    assert m.max() * 128 ** 2 > 2.5


@pytest.mark.parametrize("lag,grid", [(8, 16), (8, 8), (8, 4), (4, 12)])
def test_aligned_kuhn_lattice(lag, grid):
    """Undisplaced Kuhn lattice: vertices on grid nodes/planes; still h^3 per cell (rho = 1)."""
    q, t = mg.kuhn_mesh_3d(lag)
    m = oracle.project(_mesh(q, t, np.ones(q.shape[1]), (grid,) * 3))
    assert np.max(np.abs(m * grid ** 3 - 1.0)) < 1e-13


# ------------------------------------------------------------------------------------------
# P7 shift, permutation and reflection equivariance, P8 linearity and vertex-order invariance
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_shift_by_one_cell(dim):
    """Shifting every vertex by exactly one cell (dyadic sizes) shifts the result exactly."""
    rng = np.random.default_rng(21)
    mesh = mg.random_simplices(dim, 200, 16, 2.0, rng, periodic=False)
    # keep away from the box boundary; coordinates on a 2^-30 lattice so that a shift by 1/16 is exact
    mesh.pos = np.round((0.25 + 0.5 * mesh.pos) * 2.0 ** 30) / 2.0 ** 30
    base = oracle.project(mesh)
    for ax in range(dim):
        sh = mg.Mesh(mesh.pos.copy(), mesh.simplices, mesh.rho, mesh.grid, mesh.box_lo, mesh.box_len, False)
        sh.pos[ax] += 1.0 / 16
        out = oracle.project(sh)
        assert np.array_equal(out, np.roll(base, 1, axis=ax))


def test_axis_permutation():
    rng = np.random.default_rng(22)
    mesh = mg.random_simplices(3, 200, 8, 2.0, rng)
    base = oracle.project(mesh)
    perm = (2, 0, 1)
    pm = mg.Mesh(mesh.pos[list(perm)].copy(), mesh.simplices, mesh.rho, mesh.grid, mesh.box_lo, mesh.box_len, True)
    out = oracle.project(pm)
    assert np.max(np.abs(out - np.transpose(base, perm))) <= 1e-14 * base.max()


@pytest.mark.parametrize("dim", [2, 3])
def test_axis_reflection(dim):
    """Reflecting the periodic box along an axis (x -> 1 - x) reflects the cells (i -> N - 1 - i);
    every simplex changes orientation, and its mass stays positive."""
    rng = np.random.default_rng(24)
    mesh = mg.random_simplices(dim, 200, 8, 2.0, rng)
    base = oracle.project(mesh)
    for ax in range(dim):
        pos = mesh.pos.copy()
        pos[ax] = np.mod(1.0 - pos[ax], 1.0)
        rm = mg.Mesh(pos, mesh.simplices, mesh.rho, mesh.grid, mesh.box_lo, mesh.box_len, True)
        out = oracle.project(rm)
        assert np.max(np.abs(out - np.flip(base, axis=ax))) <= 1e-14 * base.max()
        assert abs(out.sum() - base.sum()) <= 1e-13 * base.sum()


@pytest.mark.parametrize("dim", [2, 3])
def test_linearity_and_vertex_order(dim):
    rng = np.random.default_rng(23)
    mesh = mg.random_simplices(dim, 300, 12, 3.0, rng)
    r2 = np.exp(rng.standard_normal(mesh.n_verts))
    a = oracle.project(mesh)
    b = oracle.project(mg.Mesh(mesh.pos, mesh.simplices, r2, mesh.grid, mesh.box_lo, mesh.box_len, True))
    c = oracle.project(mg.Mesh(mesh.pos, mesh.simplices, mesh.rho + 2.0 * r2, mesh.grid, mesh.box_lo,
                               mesh.box_len, True))
    assert np.max(np.abs(c - (a + 2.0 * b))) <= 1e-13 * np.max(np.abs(c))
    # reversing / rotating the vertex order of every simplex changes nothing but rounding
    rev = np.ascontiguousarray(mesh.simplices[:, ::-1])
    d = oracle.project(mg.Mesh(mesh.pos, rev, mesh.rho, mesh.grid, mesh.box_lo, mesh.box_len, True))
    assert np.max(np.abs(d - a)) <= 1e-13 * np.max(np.abs(a))


# ------------------------------------------------------------------------------------------
# P9 exact rational reference (independent slicing integrator), P10 Monte Carlo
# ------------------------------------------------------------------------------------------

def _exact_cells(mesh, s, n):
    """Exact (Fraction) masses of every bounding-box cell of simplex s (grid units, periodic
    minimal image of vertex 0). Returns {flat cell index: mass in world units as float}."""
    d = mesh.dim
    idx = mesh.simplices[s]
    u = [[Fraction(float(mesh.pos[a, v])) * n for a in range(d)] for v in idx]
    for i in range(1, d + 1):
        for a in range(d):
            dd = u[i][a] - u[0][a]
            if dd > n / 2:
                u[i][a] -= n
            elif dd < -n / 2:
                u[i][a] += n
    r = [Fraction(float(mesh.rho[v])) for v in idx]
    lo = [min(int(np.floor(v[a])) for v in u) for a in range(d)]
    hi = [max(int(np.floor(v[a])) for v in u) for a in range(d)]
    out = {}
    h = Fraction(1, n) ** d
    import itertools
    for c in itertools.product(*[range(lo[a], hi[a] + 1) for a in range(d)]):
        box = tuple((Fraction(c[a]), Fraction(c[a] + 1)) for a in range(d))
        m = exact_slicing.mass3(u, r, box) if d == 3 else exact_slicing.mass2(u, r, box)
        flat = 0
        for a in range(d):
            flat = flat * n + (c[a] % n)
        out[flat] = out.get(flat, 0.0) + float(m * h)
    return out


@pytest.mark.parametrize("dim,ns,size", [(2, 25, 1.9), (3, 8, 1.6)])
def test_exact_rational_reference(dim, ns, size):
    """Oracle == exact rational integral (to 1e-14 of the largest cell), cell by cell."""
    n = 8
    rng = np.random.default_rng(31 + dim)
    mesh = mg.random_simplices(dim, ns, n, size, rng)
    got = oracle.project(mesh).ravel()
    exact = np.zeros_like(got)
    for s in range(ns):
        for k, v in _exact_cells(mesh, s, n).items():
            exact[k] += v
    assert np.max(np.abs(got - exact)) <= 1e-14 * np.max(np.abs(exact))


def test_exact_rational_degenerate_vertices():
    """Vertices exactly on grid planes and nodes (measure-zero ties) against exact rationals."""
    n = 8
    pos = np.array([[1, 3, 1, 2, 4, 2, 3, 3], [1, 1, 3, 2, 2, 5, 2, 4], [2, 2, 2, 5, 1, 3, 3, 1]], float) / n
    simp = np.array([[0, 1, 2, 3], [4, 5, 6, 7]], np.int32)
    mesh = _mesh(pos, simp, [1.0, 2.0, 0.5, 1.5, 1.0, 3.0, 2.0, 0.25], (n,) * 3)
    got = oracle.project(mesh).ravel()
    exact = np.zeros_like(got)
    for s in range(2):
        for k, v in _exact_cells(mesh, s, n).items():
            exact[k] += v
    assert np.max(np.abs(got - exact)) <= 1e-14 * np.max(np.abs(exact))


@pytest.mark.parametrize("dim", [2, 3])
def test_monte_carlo(dim):
    """Uniform samples of each simplex, weighted by rho, agree with the oracle within 5 sigma."""
    n = 6
    rng = np.random.default_rng(41 + dim)
    mesh = mg.random_simplices(dim, 3, n, 1.4, rng)
    got = oracle.project(mesh).ravel()
    vol = oracle.simplex_mass(mg.Mesh(mesh.pos, mesh.simplices, np.ones(mesh.n_verts), mesh.grid,
                                      mesh.box_lo, mesh.box_len, True))
    nsamp = 2_000_000
    est = np.zeros_like(got)
    var = np.zeros_like(got)
    for s in range(mesh.n_simplices):
        idx = mesh.simplices[s]
        p = mesh.pos[:, idx] * n
        for i in range(1, dim + 1):
            p[:, i] -= n * np.round((p[:, i] - p[:, 0]) / n)
        w = rng.dirichlet(np.ones(dim + 1), size=nsamp)  # uniform barycentric coordinates
        x = w @ p.T
        r = w @ mesh.rho[idx]
        cells = np.floor(x).astype(np.int64) % n
        flat = np.zeros(nsamp, dtype=np.int64)
        for a in range(dim):
            flat = flat * n + cells[:, a]
        wv = r * vol[s] / nsamp
        est += np.bincount(flat, weights=wv, minlength=got.size)
        # Var(sum of N i.i.d. terms X/N) <= E[X^2]/N, estimated by the sum of (X/N)^2
        var += np.bincount(flat, weights=wv * wv, minlength=got.size)
    sig = np.sqrt(var)
    mask = sig > 0
    assert np.all(np.abs(got - est)[mask] <= 5 * sig[mask] + 1e-12)
    # a cell that holds a fraction q of a simplex's mass receives none of its N samples with
    # probability (1 - q)^N < exp(-q N): cells without a sample hold less than 20 / N of the
    # largest simplex mass (probability of a false failure below e^-20 per cell)
    smax = float(np.max(oracle.simplex_mass(mesh)))
    assert np.all(np.abs(got[~mask]) <= 20.0 / nsamp * smax)


# ------------------------------------------------------------------------------------------
# Sampled cells and error paths
# ------------------------------------------------------------------------------------------

def test_project_cells_matches_full():
    mesh = mg.make_config("c2", 8)
    full = oracle.project(mesh).ravel()
    rng = np.random.default_rng(3)
    cells = rng.choice(full.size, 200, replace=False)
    part = oracle.project_cells(mesh, cells)
    assert np.max(np.abs(part - full[cells])) <= 1e-15 * full.max()


def test_errors():
    pos = np.array([[0.125, 0.625, 0.25], [0.125, 0.125, 0.25]])
    with pytest.raises(oracle.OracleError):  # an offset of exactly half the periodic box is ambiguous
        oracle.project(_mesh(pos, [[0, 1, 2]], [1, 1, 1], (4, 4)))
    # every vertex within half a box of vertex 0, but the simplex spans half the box along x: its
    # shape would depend on which vertex is listed first, so it is rejected
    wide = np.array([[0.5, 0.25, 0.75], [0.5, 0.55, 0.5]])
    with pytest.raises(oracle.OracleError):
        oracle.project(_mesh(wide, [[0, 1, 2]], [1, 1, 1], (8, 8)))
    # just under half a box is accepted, and then any vertex order gives the same cells
    narrow = np.array([[0.5, 0.25, 0.75 - 1.0 / 64], [0.5, 0.55, 0.5]])
    a = oracle.project(_mesh(narrow, [[0, 1, 2]], [1, 2, 3], (8, 8)))
    b = oracle.project(_mesh(narrow, [[2, 0, 1]], [1, 2, 3], (8, 8)))
    assert np.max(np.abs(a - b)) <= 1e-15 * a.max()
    with pytest.raises(oracle.OracleError):  # vertex index out of range
        oracle.project(_mesh(pos, [[0, 1, 5]], [1, 1, 1], (4, 4)))


def test_thread_count_is_per_call():
    """A call on one thread gives the same cells and leaves the process-wide thread count as it was."""
    mesh = mg.random_simplices(3, 300, 8, 2.0, np.random.default_rng(25))
    before = oracle.max_threads()
    one = oracle.project(mesh, nthreads=1)
    assert oracle.max_threads() == before
    assert np.max(np.abs(one - oracle.project(mesh))) <= 1e-14 * one.max()
