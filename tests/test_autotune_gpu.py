"""cdp_autotune: the launch-shape tuning (grid multiplier, size-class threshold, tile edge of the large
tetrahedra), its cache file, and projections made with the tuned shape (they agree with those of an
untuned context to the parity tolerances)."""
import numpy as np
import pytest

from paper_1509_07720_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 1e-5}


@pytest.fixture(scope="module")
def pkg():
    import paper_1509_07720_gb300 as p
    from paper_1509_07720_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build_library()
    return p


def _dev(mesh):
    d = torch.device("cuda:0")
    return (torch.from_numpy(np.ascontiguousarray(mesh.pos)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.simplices)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.rho)).to(d))


def _mesh(name):
    if name == "c2_16":
        return mg.make_config("c2", 16)
    if name == "rand3d_large":  # tetrahedra of a few to a hundred thousand cells: both size classes
        return mg.random_simplices(3, 60, 96, 12.0, np.random.default_rng(6))
    return mg.random_simplices(2, 600, 32, 3.0, np.random.default_rng(5))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
@pytest.mark.parametrize("name", ["c2_16", "rand3d_large", "rand2d"])
def test_autotune_then_project(pkg, tmp_path, name, prec):
    mesh = _mesh(name)
    pos, simp, rho = _dev(mesh)
    cache = tmp_path / "tune.txt"
    tuned = pkg.Projector(0)
    try:
        m = tuned.autotune(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, precision=prec,
                           cache_path=str(cache))
        assert m[0] in (1, 2, 4, 8)
        if mesh.dim == 3:
            assert m[1] in (960, 1920, 3840, 6144 if prec == 1 else 10240) and m[2] in (18, 23)
        lines = cache.read_text().splitlines()
        assert len(lines) == 1 and lines[0].endswith(" %d %d %d" % m) and f"dim{mesh.dim}" in lines[0]
        # a second context takes the cached choice without timing (the file is not appended to)
        other = pkg.Projector(0)
        try:
            assert other.autotune(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic,
                                  precision=prec, cache_path=str(cache)) == m
            assert len(cache.read_text().splitlines()) == 1
        finally:
            other.close()
        got = tuned.project(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, precision=prec)
        torch.cuda.synchronize()
        tuned.check()
    finally:
        tuned.close()
    plain = pkg.Projector(0)
    try:
        ref = plain.project(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, precision=prec)
        torch.cuda.synchronize()
    finally:
        plain.close()
    a, b = got.cpu().numpy(), ref.cpu().numpy()
    assert np.max(np.abs(a - b)) <= TOL[prec] * np.max(np.abs(b))
    assert abs(a.sum() - b.sum()) <= 1e-12 * abs(b.sum())


def test_autotune_argument_errors(pkg):
    mesh = mg.make_config("c2", 16)
    pos, simp, rho = _dev(mesh)
    out = torch.empty(mesh.grid, dtype=torch.float64, device="cuda:0")
    proj = pkg.Projector(0)
    try:
        prob = pkg.Projector.make_problem(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, mesh.periodic, out)
        assert pkg.cdp_autotune(proj._ctx, prob, 7)[0] == -1
        assert pkg.cdp_autotune(None, prob, 0)[0] == -1
    finally:
        proj.close()
