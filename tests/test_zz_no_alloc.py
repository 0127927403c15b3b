"""cdp_project_noalloc (static device scratch, no allocation) against cdp_project, through the C ABI.

Both entry points launch the same kernels, so their grids agree to the parity tolerances of the
projection (FP64 1e-11, FP32-mixed 1e-5 of the largest cell, total mass 1e-12).  The file is
named to be collected last, so that it runs after every other GPU test as well as alone.
"""
import numpy as np
import pytest

from paper_1509_07720_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 1e-5}
TOTAL_TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    import paper_1509_07720_gb300 as pkg
    from paper_1509_07720_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build_library()
    torch.cuda.set_device(0)
    c = pkg.cdp_create(0)
    yield c
    pkg.cdp_destroy(c)


def _dev(mesh):
    d = torch.device("cuda:0")
    return (torch.from_numpy(np.ascontiguousarray(mesh.pos)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.simplices)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.rho)).to(d))


def _cases():
    rng = np.random.default_rng(31)
    return {
        "c2_16": mg.make_config("c2", 16),
        "rand3d_mid": mg.random_simplices(3, 400, 16, 2.5, rng),
        "rand2d": mg.random_simplices(2, 600, 32, 3.0, rng),
        # tetrahedra whose bounding boxes span several 23^3-cell tiles: the large-tetrahedron kernel,
        # which here keeps no pieces between its two FP32 passes (no tile store) and recomputes them
        "rand3d_large": mg.random_simplices(3, 4, 96, 20.0, np.random.default_rng(3)),
    }


CASES = _cases()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_matches_project(ctx, name, prec):
    import paper_1509_07720_gb300 as pkg

    mesh = CASES[name]
    pos, simp, rho = _dev(mesh)
    st = torch.cuda.current_stream().cuda_stream
    ref = torch.empty(mesh.grid, dtype=torch.float64, device="cuda:0")
    p_ref = pkg.Projector.make_problem(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, ref)
    assert pkg.cdp_project(ctx, p_ref, prec, 0, st) == 0
    torch.cuda.synchronize()
    assert pkg.cdp_check(ctx, st) == 0
    want = ref.cpu().numpy()
    scale = float(np.max(want))

    out = torch.full(mesh.grid, 7.0, dtype=torch.float64, device="cuda:0")  # must be overwritten
    flags = torch.full((1,), 0xFF, dtype=torch.int32, device="cuda:0")
    p = pkg.Projector.make_problem(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, out)
    for call in range(2):  # two calls in a row on the same static scratch
        assert pkg.cdp_project_noalloc(p, prec, 0, flags.data_ptr(), st) == 0
        torch.cuda.synchronize()
        assert int(flags.item()) == 0, f"call {call}: error flags {int(flags.item())}"
        got = out.cpu().numpy()
        err = np.max(np.abs(got - want)) / scale
        assert err <= TOL[prec], f"call {call}: max rel difference {err:.3e}"
        assert abs(got.sum() - want.sum()) <= TOTAL_TOL * abs(want.sum())


def test_noalloc_large_tetrahedra_are_tiled(ctx):
    """The large case really reaches the tiled kernel (its tetrahedra exceed the shared-memory box)."""
    import paper_1509_07720_gb300 as pkg

    mesh = CASES["rand3d_large"]
    pos, simp, rho = _dev(mesh)
    out = torch.empty(mesh.grid, dtype=torch.float64, device="cuda:0")
    p = pkg.Projector.make_problem(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, out)
    st = pkg.cdp_stats()
    assert pkg.cdp_project(ctx, p, pkg.CDP_FP32_MIXED, 0, 0, st) == 0
    assert st.n_large > 0 and st.n_large_tiles > 0


def test_noalloc_accumulate_and_errors(ctx):
    import paper_1509_07720_gb300 as pkg

    mesh = CASES["rand3d_mid"]
    pos, simp, rho = _dev(mesh)
    st = torch.cuda.current_stream().cuda_stream
    out = torch.zeros(mesh.grid, dtype=torch.float64, device="cuda:0")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    p = pkg.Projector.make_problem(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, out)
    assert pkg.cdp_project_noalloc(p, 0, 0, flags.data_ptr(), st) == 0
    torch.cuda.synchronize()
    once = out.cpu().numpy()
    assert pkg.cdp_project_noalloc(p, 0, 1, flags.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - 2 * once)) <= 1e-11 * np.max(once)

    # a simplex naming a vertex past the end is flagged by the kernels' own index check
    bad = simp.clone()
    bad[3, 2] = mesh.n_verts + 5
    pb = pkg.Projector.make_problem(pos, bad, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, out)
    assert pkg.cdp_project_noalloc(pb, 0, 0, flags.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert int(flags.item()) & 1
    # the next good call starts from clear counters
    assert pkg.cdp_project_noalloc(p, 1, 0, flags.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert int(flags.item()) == 0

    # more vertices than the static scratch holds: rejected on the host, nothing enqueued
    big = pkg.Projector.make_problem(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, out)
    big.n_verts = pkg.CDP_NOALLOC_MAX_VERTS + 1
    assert pkg.cdp_project_noalloc(big, 0, 0, 0, st) == -1
    assert pkg.cdp_project_noalloc(p, 7, 0, 0, st) == -1
