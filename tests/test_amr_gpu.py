"""Parity of the projection through coarser levels with donor-cell gather (cdp_project_amr, Sect. 4.4,
calculation of the acceleration) with its oracle (``oracle.amr``), element by element.

A simplex whose smallest perpendicular height lies within rounding of a power of two may take
either of the two levels (the kernel computes it from fixed-point coordinates, the oracle from the
world coordinates): the cases leave such simplices out.  The tolerances are those of the exact
projection (FP64 1e-11, FP32-mixed 1e-5 of the largest cell mass; total mass 1e-12).
"""
import numpy as np
import pytest

import oracle
from oracle import amr
from paper_1509_07720_gb300 import meshgen as mg
from parity_report import record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 1e-5}
TOTAL_TOL = 1e-12


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


def _clear_of_boundaries(mesh, lmax):
    """The mesh without the simplices whose height is within 1e-9 (relative) of 2^1 .. 2^lmax."""
    eta = amr.simplex_heights(mesh)
    keep = np.ones(eta.shape, dtype=bool)
    for l in range(1, lmax + 1):
        keep &= np.abs(eta / float(1 << l) - 1.0) > 1e-9
    return mesh.subset(np.nonzero(keep)[0])


def _cases():
    rng = np.random.default_rng(31)
    out = {
        "mixed3d_32": (mg.mixed_size_simplices(3, 32, ((300, 0.8), (200, 3.0), (100, 7.0)), rng), 2),
        "mixed3d_64": (mg.mixed_size_simplices(3, 64, ((400, 1.0), (200, 4.0), (120, 9.0), (40, 15.0)), rng), 3),
        "mixed2d_128": (mg.mixed_size_simplices(2, 128, ((800, 1.0), (300, 5.0), (200, 12.0), (80, 30.0)), rng), 4),
        "c2_16": (mg.make_config("c2", 16), 2),
        "c4_8": (mg.make_config("c4", 8), 3),
        "c1b_32": (mg.make_config("c1b", 32), 3),
    }
    return {k: (_clear_of_boundaries(m, l), l) for k, (m, l) in out.items()}


CASES = _cases()


def _dev(mesh):
    d = torch.device("cuda:0")
    return (torch.from_numpy(np.ascontiguousarray(mesh.pos)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.simplices)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.rho)).to(d))


def _amr(proj, mesh, lmax, prec, **kw):
    pos, simp, rho = _dev(mesh)
    res = proj.project_amr(pos, simp, rho, mesh.grid, lmax, mesh.box_lo, mesh.box_len, mesh.periodic,
                           precision=prec, **kw)
    torch.cuda.synchronize()
    return res


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_amr_parity(proj, name, prec):
    mesh, lmax = CASES[name]
    assert len(set(amr.amr_levels(mesh, lmax).tolist())) >= 2  # more than one level in use
    ref = amr.project_amr(mesh, lmax)
    out, st = _amr(proj, mesh, lmax, prec, stats=True)
    got = out.cpu().numpy()
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(got - ref)) / scale
    tot = abs(got.sum() - ref.sum()) / abs(ref.sum())
    record(f"amr_{name}", prec, max_rel=err, total_rel=tot, cells=int(got.size))
    assert st["error_flags"] == 0
    assert err <= TOL[prec], f"{name}: max rel error {err:.3e}"
    assert tot <= TOTAL_TOL, f"{name}: total mass rel error {tot:.3e}"


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
def test_level_zero_is_the_projection(proj, prec):
    mesh, _ = CASES["mixed3d_32"]
    pos, simp, rho = _dev(mesh)
    a = proj.project(pos, simp, rho, mesh.grid, precision=prec)
    b = proj.project_amr(pos, simp, rho, mesh.grid, 0, precision=prec)
    torch.cuda.synchronize()
    # (two FP32-mixed projections of the same mesh differ by the order of their FP32 shared-memory
    # adds: a few FP32 ulps of a piece)
    assert float((a - b).abs().max()) <= {0: 1e-13, 1: 1e-6}[prec] * float(a.abs().max())


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
def test_block_sums_full_size(proj, prec):
    """At the full size of the 256^3 random-field workload: every sum over an aligned block of
    2^max_level cells per axis equals that of the exact projection (the projection onto a level's
    grid is exact), and the total mass is kept."""
    mesh = mg.make_config("c3")
    lmax = 3
    pos, simp, rho = _dev(mesh)
    exact = proj.project(pos, simp, rho, mesh.grid, precision=prec)
    got = proj.project_amr(pos, simp, rho, mesh.grid, lmax, precision=prec)
    torch.cuda.synchronize()
    proj.check()
    b = 1 << lmax
    n = mesh.grid[0] // b
    be = exact.reshape(n, b, n, b, n, b).sum(dim=(1, 3, 5))
    bg = got.reshape(n, b, n, b, n, b).sum(dim=(1, 3, 5))
    err = float((be - bg).abs().max()) / float(be.abs().max())
    tot = abs(float(got.sum()) - float(exact.sum())) / float(exact.sum())
    record("amr_c3_block_sums", prec, max_rel=err, total_rel=tot, cells=int(be.numel()))
    assert err <= TOL[prec] * b ** 3
    assert tot <= TOTAL_TOL


def test_accumulate_and_arguments(proj):
    import paper_1509_07720_gb300 as pkg

    mesh, lmax = CASES["mixed2d_128"]
    a = _amr(proj, mesh, lmax, 0)
    b = a.clone()
    _amr(proj, mesh, lmax, 0, out=b, accumulate=True)
    assert float((b - 2 * a).abs().max()) <= 1e-13 * float(a.abs().max())
    pos, simp, rho = _dev(mesh)
    for bad_level, grid in ((7, (128, 128)), (-1, (128, 128)), (6, (96, 96))):
        with pytest.raises(pkg.CdpError):
            proj.project_amr(pos, simp, rho, grid, bad_level, precision=0)
    # empty mesh
    out = proj.project_amr(pos, simp[:0].contiguous(), rho, mesh.grid, 3, precision=1)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
