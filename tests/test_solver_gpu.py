"""GPU parity of the solver steps (C ABI) with the numpy oracle: Poisson, force, drift/kick,
vertex densities, and batched projection against one-by-one projections.

Tolerances: FP64 arithmetic on both sides; the FFT and the summation orders differ, so the
bound is 1e-12 of the largest value (Poisson, force) and 1e-13 (elementwise steps)."""
import numpy as np
import pytest

import oracle
from oracle import solver
from paper_1509_07720_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1509_07720_gb300 as pkg
    from paper_1509_07720_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build_library()
    c = pkg.cdp_create(0)
    yield c
    pkg.cdp_destroy(c)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _ok(rc):
    assert rc == 0, rc


@pytest.mark.parametrize("shape,box", [((32, 32), (1.0, 1.0)), ((24, 20, 16), (1.0, 1.2, 0.9)),
                                       ((64, 64, 64), (1.0, 1.0, 1.0)), ((17, 9), (2.0, 1.0))])
def test_poisson(ctx, shape, box):
    import paper_1509_07720_gb300 as pkg

    rng = np.random.default_rng(sum(shape))
    mass = rng.random(shape)
    ref = solver.poisson(mass, box, 1.3)
    m = _t(mass)
    phi = torch.empty_like(m)
    dim = len(shape)
    _ok(pkg.cdp_poisson(ctx, dim, list(shape) + [1] * (3 - dim), list(box) + [1.0] * (3 - dim), 1.3,
                        m.data_ptr(), phi.data_ptr(), torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    got = phi.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("dim", [2, 3])
def test_force(ctx, dim):
    import paper_1509_07720_gb300 as pkg

    shape = (16, 20, 12)[:dim]
    box = (1.0, 1.25, 0.75)[:dim]
    lo = (0.1, -0.2, 0.3)[:dim]
    rng = np.random.default_rng(5 + dim)
    phi = rng.standard_normal(shape)
    n = 3000
    pos = np.stack([lo[a] + box[a] * rng.random(n) for a in range(dim)])
    ref = solver.force(phi, lo, box, pos)
    dp = _t(phi)
    tp = [_t(pos[a]) for a in range(dim)]
    ta = [torch.empty(n, dtype=torch.float64, device="cuda:0") for _ in range(dim)]
    _ok(pkg.cdp_force(ctx, dim, list(shape) + [1] * (3 - dim), list(lo) + [0.0] * (3 - dim),
                      list(box) + [1.0] * (3 - dim), dp.data_ptr(), n, tp, ta, torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    got = np.stack([t.cpu().numpy() for t in ta])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_drift_kick(ctx):
    import paper_1509_07720_gb300 as pkg

    rng = np.random.default_rng(9)
    n = 5000
    pos = rng.random((3, n))
    vel = rng.standard_normal((3, n))
    acc = rng.standard_normal((3, n))
    tp = [_t(pos[a]) for a in range(3)]
    tv = [_t(vel[a]) for a in range(3)]
    ta = [_t(acc[a]) for a in range(3)]
    st = torch.cuda.current_stream().cuda_stream
    _ok(pkg.cdp_drift(ctx, 3, n, tp, tv, 0.07, (0.0,) * 3, (1.0,) * 3, 1, st))
    _ok(pkg.cdp_kick(ctx, 3, n, tv, ta, 0.05, st))
    torch.cuda.synchronize()
    p_ref = solver.drift(pos, vel, 0.07, (0.0,) * 3, (1.0,) * 3)
    v_ref = solver.kick(vel, acc, 0.05)
    gp = np.stack([t.cpu().numpy() for t in tp])
    gv = np.stack([t.cpu().numpy() for t in tv])
    d = np.abs(gp - p_ref)
    d = np.minimum(d, 1.0 - d)  # a point on the wrap boundary may land on either side
    assert d.max() < 1e-14 and np.max(np.abs(gv - v_ref)) < 1e-14
    assert gp.min() >= 0.0 and gp.max() < 1.0


@pytest.mark.parametrize("name", ["c2_16", "c1b"])
def test_vertex_density(ctx, name):
    import paper_1509_07720_gb300 as pkg

    mesh = mg.make_config("c2", 16) if name == "c2_16" else mg.make_config("c1b")
    rng = np.random.default_rng(4)
    masses = rng.random(mesh.n_simplices) * 1e-4
    ref = solver.vertex_density(mesh.pos, mesh.simplices, masses, mesh.box_len)
    pos = _t(mesh.pos)
    simp = _t(mesh.simplices)
    rho = _t(mesh.rho)
    out = torch.empty(mesh.grid, dtype=torch.float64, device="cuda:0")
    prob = pkg.Projector.make_problem(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, True, out)
    rout = torch.empty(mesh.n_verts, dtype=torch.float64, device="cuda:0")
    _ok(pkg.cdp_vertex_density(ctx, prob, _t(masses).data_ptr(), rout.data_ptr(),
                               torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert np.max(np.abs(rout.cpu().numpy() - ref)) <= 1e-12 * np.max(ref)


def test_batched_equals_single(ctx):
    import paper_1509_07720_gb300 as pkg

    meshes = [mg.make_config("c2", 8), mg.make_config("c1a", 16), mg.random_simplices(3, 200, 24, 4.0,
                                                                                      np.random.default_rng(2))]
    keep, probs, outs = [], [], []
    for m in meshes:
        pos, simp, rho = _t(m.pos), _t(m.simplices), _t(m.rho)
        out = torch.empty(m.grid, dtype=torch.float64, device="cuda:0")
        keep += [pos, simp, rho]
        outs.append(out)
        probs.append(pkg.Projector.make_problem(pos, simp, rho, m.grid, m.box_lo, m.box_len, m.periodic, out))
    for prec, tol in ((0, 1e-11), (1, 1e-5)):
        _ok(pkg.cdp_project_batched(ctx, probs, prec, torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        for m, o in zip(meshes, outs):
            ref = oracle.project(m)
            assert np.max(np.abs(o.cpu().numpy() - ref)) <= tol * np.max(ref)
