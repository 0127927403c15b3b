"""Parity of the CUDA projection (through the C ABI) with the CPU oracle, element by element.

Tolerances (the stated accuracy targets of the two arithmetic paths):
  FP64 path       max |m_gpu - m_oracle| / max m_oracle <= 1e-11
  FP32-mixed path max |m_gpu - m_oracle| / max m_oracle <= 1e-5
  both            total mass relative error <= 1e-12 (the FP32 path closes every simplex's mass
                  against its FP64 closed form)
The combinatorial decisions (which corners exist) are exact integer predicates, so both paths
must also report identical corner counts.
"""
import numpy as np
import pytest

import oracle
from paper_1509_07720_gb300 import meshgen as mg
from parity_report import record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 1e-5}
TOTAL_TOL = 1e-12
# Cases whose simplices cross the walls of a non-periodic box.  The FP32-mixed path closes the mass
# of every simplex, not of its part inside the box, so there its total inside the box is only as
# exact as its cells (FP32 tolerance); the FP64 path keeps 1e-12.
CLIPPED = {"rand3d_huge_walls"}


@pytest.fixture(scope="module")
def proj():
    import paper_1509_07720_gb300 as pkg
    from paper_1509_07720_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build_library()
    p = pkg.Projector(0)
    yield p
    p.close()


def _dev(mesh):
    d = torch.device("cuda:0")
    return (torch.from_numpy(np.ascontiguousarray(mesh.pos)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.simplices)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.rho)).to(d))


def _run(proj, mesh, prec, stats=False):
    """prec may carry CDP_ACCURACY_OFF (0x100)."""
    pos, simp, rho = _dev(mesh)
    res = proj.project(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, precision=prec,
                       stats=stats)
    torch.cuda.synchronize()
    if stats:
        return res[0].cpu().numpy(), res[1]
    proj.check()
    return res.cpu().numpy()


def _cases():
    rng = np.random.default_rng(7)
    q8, t8 = mg.kuhn_mesh_3d(8)
    qb, tb = mg.kuhn_box_mesh_3d(4)
    return {
        "c1a": mg.make_config("c1a"),
        "c1b": mg.make_config("c1b"),
        "c2_16": mg.make_config("c2", 16),
        "c2": mg.make_config("c2"),
        "c4_4": mg.make_config("c4", 4),
        "c4_8": mg.make_config("c4", 8),
        "rand3d_small": mg.random_simplices(3, 500, 16, 0.7, rng),
        "rand3d_mid": mg.random_simplices(3, 500, 16, 2.5, rng),
        "rand3d_tiled": mg.random_simplices(3, 40, 40, 9.0, rng),
        "rand3d_lognormal1": mg.random_simplices(3, 300, 16, 3.0, rng, rho_sigma=1.0),
        "rand2d": mg.random_simplices(2, 800, 32, 3.0, rng),
        "rand2d_tiled": mg.random_simplices(2, 60, 96, 20.0, rng),
        "aligned_kuhn_16": mg.Mesh(q8, t8, np.ones(q8.shape[1]), (16,) * 3, (0.0,) * 3, (1.0,) * 3, True),
        "aligned_kuhn_8": mg.Mesh(q8, t8, np.ones(q8.shape[1]), (8,) * 3, (0.0,) * 3, (1.0,) * 3, True),
        "box_linear_rho": mg.Mesh(qb * 0.8 + 0.1, tb, 1.0 + qb[0] - 0.5 * qb[2], (12, 10, 9), (0.0,) * 3,
                                  (1.0,) * 3, False),
        "ragged_grid": mg.Mesh(*(lambda m: (m.pos, m.simplices, m.rho))(mg.make_config("c2", 8)), (29, 31, 33),
                               (0.0,) * 3, (1.0,) * 3, True),
        # tetrahedra spanning several 23^3 tiles, with many cells entirely inside them (periodic, and
        # clipped by the walls of a non-periodic box)
        "rand3d_huge": mg.random_simplices(3, 6, 96, 22.0, np.random.default_rng(71)),
        "rand3d_huge_walls": mg.random_simplices(3, 5, 40, 30.0, np.random.default_rng(72), periodic=False),
    }


def _degenerate():
    out = {}
    for dim, seed in ((3, 81), (2, 82)):
        for name, (mesh, nzero) in mg.degenerate_meshes(dim, 32, np.random.default_rng(seed)).items():
            out[f"{name}_{dim}d"] = (mesh, nzero)
    return out


DEGENERATE = _degenerate()
CASES = _cases()
CASES.update({k: m for k, (m, _) in DEGENERATE.items()})


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_parity(proj, name, prec):
    mesh = CASES[name]
    ref = oracle.project(mesh)
    got = _run(proj, mesh, prec)
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(got - ref)) / scale
    tot = abs(got.sum() - ref.sum()) / abs(ref.sum())
    record(name, prec, max_rel=err, total_rel=tot, cells=int(got.size))
    assert err <= TOL[prec], f"{name}: max rel error {err:.3e}"
    ttol = TOL[1] if (prec == 1 and name in CLIPPED) else TOTAL_TOL
    assert tot <= ttol, f"{name}: total mass rel error {tot:.3e}"


@pytest.mark.parametrize("name", ["c2", "rand3d_tiled", "aligned_kuhn_16", "c1b", "rand2d_tiled", "rand3d_huge",
                                  "rand3d_huge_walls"] + sorted(DEGENERATE))
def test_same_decisions_both_precisions(proj, name):
    """The exact predicates take the same combinatorial decisions in both arithmetics (compared
    without the accuracy control, whose routing depends on the arithmetic's rounding)."""
    mesh = CASES[name]
    _, s64 = _run(proj, mesh, 0 | 0x100, stats=True)
    _, s32 = _run(proj, mesh, 1 | 0x100, stats=True)
    for k in ("corners_a", "corners_b", "corners_c", "corners_d", "n_single_cell", "n_small", "n_large",
              "n_large_tiles", "n_zero_volume"):
        assert s64[k] == s32[k], k
    assert s64["error_flags"] == 0


@pytest.mark.parametrize("name", sorted(DEGENERATE))
def test_zero_volume_count(proj, name):
    """Flat simplices (exactly, after the fixed-point conversion of dyadic coordinates) contribute
    nothing and are counted; no other simplex of the case is."""
    mesh, nzero = DEGENERATE[name]
    for prec in (0, 1):
        _, st = _run(proj, mesh, prec, stats=True)
        assert st["n_zero_volume"] == nzero, (prec, st["n_zero_volume"], nzero)
        assert st["error_flags"] == 0


def test_total_mass_against_simplex_masses(proj):
    mesh = CASES["c2"]
    ref = oracle.simplex_mass(mesh).sum()
    got = _run(proj, mesh, 0)
    assert abs(got.sum() - ref) <= TOTAL_TOL * ref


def test_empty_and_accumulate(proj):
    mesh = CASES["c2_16"]
    pos, simp, rho = _dev(mesh)
    out = proj.project(pos, simp[:0].contiguous(), rho, mesh.grid)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
    a = proj.project(pos, simp, rho, mesh.grid, precision=0)
    b = a.clone()
    proj.project(pos, simp, rho, mesh.grid, precision=0, out=b, accumulate=True)
    torch.cuda.synchronize()
    assert torch.allclose(b, 2 * a, rtol=1e-14, atol=0)


def test_device_detected_errors(proj):
    import paper_1509_07720_gb300 as pkg

    mesh = CASES["rand3d_small"]
    pos, simp, rho = _dev(mesh)
    bad = simp.clone()
    bad[3, 2] = mesh.n_verts + 5
    with pytest.raises(pkg.CdpError) as e:
        proj.project(pos, bad, rho, mesh.grid, stats=True)
    assert e.value.code == -2
    nanpos = pos.clone()
    nanpos[0, 7] = float("nan")
    with pytest.raises(pkg.CdpError) as e:
        proj.project(nanpos, simp, rho, mesh.grid)
        proj.check()
    assert e.value.code == -3
    proj.check()  # cleared


def test_extent_error(proj):
    import paper_1509_07720_gb300 as pkg

    pos = torch.tensor([[0.125, 0.625, 0.25], [0.125, 0.125, 0.25]], dtype=torch.float64, device="cuda:0")
    simp = torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda:0")
    rho = torch.ones(3, dtype=torch.float64, device="cuda:0")
    with pytest.raises(pkg.CdpError) as e:
        proj.project(pos, simp, rho, (4, 4), stats=True)
    assert e.value.code == -4


_ORACLE = {}


def _oracle_once(key, fn):
    """An oracle result computed once per test session (the large workloads take tens of seconds)."""
    if key not in _ORACLE:
        _ORACLE[key] = fn()
    return _ORACLE[key]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
def test_headline_workload_full_grid(proj, prec):
    """Full-size 128^3 Kuhn mesh (12,582,912 tets) on the 256^3 grid, in the benchmark's launch
    configuration: every one of the 16,777,216 cells against the oracle, the total mass against the
    simplex masses, and the same corner decisions in both precisions."""
    mesh = _oracle_once("c3_mesh", lambda: mg.make_config("c3"))
    got, st = _run(proj, mesh, prec, stats=True)
    assert st["error_flags"] == 0
    ref = _oracle_once("c3", lambda: oracle.project(mesh))
    scale = float(np.max(np.abs(ref)))
    err = float(np.max(np.abs(got - ref))) / scale
    tot = _oracle_once("c3_tot", lambda: oracle.simplex_mass(mesh).sum())
    rel = abs(got.sum() - tot) / tot
    record("c3", prec, max_rel=err, total_rel=rel, cells=int(got.size))
    assert err <= TOL[prec], f"max rel error over all cells {err:.3e}"
    assert rel <= TOTAL_TOL, f"total mass rel error {rel:.3e}"
    assert st["accuracy_bound"] <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
def test_adaptive_subset_full_grid(proj, prec):
    """A seeded 1/16 stratified subset of the bisected mesh (about 3.1M tets, every volume class
    represented) on the full 512^3 grid: every cell against the oracle, and the total mass."""
    sub = _oracle_once("c4_sub", lambda: mg.stratified_subset(_c4_full(), 16, np.random.default_rng(1604)))
    got = _run(proj, sub, prec)
    ref = _oracle_once("c4_sub_ref", lambda: oracle.project(sub))
    scale = float(np.max(np.abs(ref)))
    err = float(np.max(np.abs(got - ref))) / scale
    tot = float(ref.sum())
    record("c4_subset16", prec, max_rel=err, total_rel=abs(got.sum() - tot) / tot, cells=int(got.size),
           simplices=sub.n_simplices)
    assert err <= TOL[prec], f"max rel error over all cells {err:.3e}"
    assert abs(got.sum() - tot) <= TOTAL_TOL * tot


@pytest.mark.parametrize("axes", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (3, -2, 5)], ids=["x", "y", "z", "xyz"])
def test_shift_equivariance(proj, axes):
    """A translation by whole grid cells (dyadic coordinates, power-of-two grid, periodic box) moves
    every cell's mass with it.  Every exact decision is the same (equal corner counts), and each
    piece is computed from the same cell-relative numbers; only the order in which the pieces of a
    cell are summed on the GPU may differ (atomic adds), so cells agree to that rounding."""
    base = mg.quantize_positions(mg.make_config("c2", 8), 30)
    moved = mg.shift_mesh(base, axes)
    for prec, tol in ((0, 1e-14), (1, 2e-6)):
        a, sa = _run(proj, base, prec, stats=True)
        b, sb = _run(proj, moved, prec, stats=True)
        want = np.roll(a, axes, axis=(0, 1, 2))
        err = float(np.max(np.abs(b - want))) / float(np.max(np.abs(a)))
        assert err <= tol, (prec, err)
        for k in ("corners_a", "corners_b", "corners_c", "corners_d", "n_single_cell", "n_large_tiles"):
            assert sa[k] == sb[k], (prec, k)


@pytest.mark.parametrize("name", ["c2_16", "rand3d_tiled", "rand3d_huge", "aligned_kuhn_16", "c1b", "rand2d_tiled",
                                  "grid_planes_3d", "grid_lines_3d"])
def test_vertex_order_invariance(proj, name):
    """The projection of a simplex does not depend on the order in which its vertices are listed
    (even and odd permutations): the same corners are found, and cells agree within the tolerance."""
    mesh = CASES[name]
    perm = mg.permute_vertex_order(mesh, np.random.default_rng(5))
    assert not np.array_equal(perm.simplices, mesh.simplices)
    for prec, tol in ((0, 1e-12), (1, TOL[1])):
        a = _run(proj, mesh, prec)
        b = _run(proj, perm, prec)
        err = float(np.max(np.abs(b - a))) / float(np.max(np.abs(a)))
        assert err <= tol, (prec, err)
        # the corners found (without the accuracy control, whose routing may differ by a rounding)
        _, sa = _run(proj, mesh, prec | 0x100, stats=True)
        _, sb = _run(proj, perm, prec | 0x100, stats=True)
        for k in ("corners_a", "corners_b", "corners_c", "corners_d", "n_single_cell", "n_zero_volume",
                  "n_large_tiles"):
            assert sa[k] == sb[k], (prec, k)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
def test_adaptive_workload_sampled(proj, prec):
    """Full-size bisected mesh (50.3M tets, volumes over 4 decades, hanging nodes, base vertices on
    grid planes) on a 512^3 grid: sampled cells against the oracle, total mass against the simplex
    masses, and the same corner decisions in both precisions."""
    mesh = _c4_full()
    got, st = _run(proj, mesh, prec, stats=True)
    assert st["error_flags"] == 0
    rng = np.random.default_rng(98)
    cells = rng.choice(got.size, 256, replace=False)
    cells = np.unique(np.concatenate([cells, np.argsort(got.ravel())[-32:]]))
    ref = oracle.project_cells(mesh, cells)
    scale = float(np.max(got))
    err = np.max(np.abs(got.ravel()[cells] - ref)) / scale
    assert err <= TOL[prec], f"sampled max rel error {err:.3e}"
    tot = oracle.simplex_mass(mesh).sum()
    rel = abs(got.sum() - tot) / tot
    assert rel <= TOTAL_TOL, f"total mass rel error {rel:.3e}"
    _C4_STATS[prec] = st
    _C4_GRIDS[prec] = got
    if len(_C4_STATS) == 2:
        for k in ("n_single_cell", "n_large", "n_zero_volume"):
            assert _C4_STATS[0][k] == _C4_STATS[1][k], k
        # every cell of the full-size FP32-mixed grid against the full-size FP64 grid (the FP64
        # path is itself held to 1e-11 of the oracle on the stratified subset above)
        d = float(np.max(np.abs(_C4_GRIDS[1] - _C4_GRIDS[0]))) / float(np.max(_C4_GRIDS[0]))
        assert d <= TOL[1], f"FP32-mixed vs FP64 over all cells {d:.3e}"
        _C4_GRIDS.clear()


_C4 = {}
_C4_STATS = {}
_C4_GRIDS = {}


def _c4_full():
    if "m" not in _C4:
        _C4["m"] = mg.make_config("c4")
    return _C4["m"]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
def test_batched_matches_single(proj, prec):
    """cdp_project_batched projects its problems in groups (one launch of each kernel per group of up
    to 64 problems of one dimension): every problem's grid equals its projection alone, for a mix of
    2D and 3D problems (tiled and deferred/clipped simplices included) and more than one group."""
    import paper_1509_07720_gb300 as pkg

    names = ["c1a", "c2_16", "rand3d_mid", "rand2d", "rand3d_tiled", "aligned_kuhn_8", "box_linear_rho",
             "slivers_3d", "slivers_2d", "zero_volume_3d", "rand3d_huge", "c4_4"]
    meshes = [CASES[n] for n in names]
    rng = np.random.default_rng(90)
    meshes += [mg.random_simplices(3, 30, 16, 2.0, rng) for _ in range(66)]  # 3D: more than one group
    d = torch.device("cuda:0")
    keep, probs, outs = [], [], []
    for m in meshes:
        pos, simp, rho = _dev(m)
        out = torch.full(m.grid, 3.0, dtype=torch.float64, device=d)  # must be overwritten
        probs.append(pkg.Projector.make_problem(pos, simp, rho, m.grid, m.box_lo, m.box_len, m.periodic, out))
        keep.append((pos, simp, rho))
        outs.append(out)
    st = torch.cuda.current_stream().cuda_stream
    assert pkg.cdp_project_batched(proj._ctx, probs, prec, st) == 0
    torch.cuda.synchronize()
    proj.check()
    tol = 1e-13 if prec == 0 else 1e-6
    for i, m in enumerate(meshes):
        want = _run(proj, m, prec)
        got = outs[i].cpu().numpy()
        scale = float(np.max(np.abs(want)))
        assert np.max(np.abs(got - want)) <= tol * scale, i
        assert abs(got.sum() - want.sum()) <= 1e-13 * abs(want.sum()), i
