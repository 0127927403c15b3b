"""A batched time step (drift, vertex density, projection, Poisson, force, kick, drift) through the
C ABI against the oracle composition of the same steps; the CUDA-graph replay against eager
execution."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import solver
from paper_1509_07720_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FPG = 1.0


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


def _problems():
    rng = np.random.default_rng(12)
    out = []
    m2 = mg.make_config("c1a", 16)
    m3 = mg.make_config("c2", 8)
    for m in (m2, m3):
        vel = 0.05 * rng.standard_normal(m.pos.shape)
        p = m.pos[:, m.simplices]
        e = p[:, :, 1:] - p[:, :, :1]
        e -= np.round(e)
        if m.dim == 3:
            vol = np.abs(np.einsum("ij,ij->j", e[:, :, 0], np.cross(e[:, :, 1].T, e[:, :, 2].T).T)) / 6
        else:
            vol = np.abs(e[0, :, 0] * e[1, :, 1] - e[1, :, 0] * e[0, :, 1]) / 2
        masses = vol * (1.0 + 0.3 * rng.random(m.n_simplices))
        out.append((m, vel, masses))
    return out


def _oracle_step(m, vel, masses, dt):
    pos = solver.drift(m.pos, vel, 0.5 * dt, m.box_lo, m.box_len)
    rho = solver.vertex_density(pos, m.simplices, masses, m.box_len)
    cm = oracle.project(mg.Mesh(pos, m.simplices, rho, m.grid, m.box_lo, m.box_len, True))
    phi = solver.poisson(cm, m.box_len, FPG)
    acc = solver.force(phi, m.box_lo, m.box_len, pos)
    v2 = solver.kick(vel, acc, dt)
    p2 = solver.drift(pos, v2, 0.5 * dt, m.box_lo, m.box_len)
    return p2, v2, rho, cm, phi, acc


class _Dev:
    def __init__(self, m, vel, masses):
        import paper_1509_07720_gb300 as pkg

        d = torch.device("cuda:0")
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)
        self.m = m
        self.pos = [t(m.pos[a]) for a in range(m.dim)]
        self.vel = [t(vel[a]) for a in range(m.dim)]
        self.acc = [torch.zeros(m.n_verts, dtype=torch.float64, device=d) for _ in range(m.dim)]
        self.simp = t(m.simplices)
        self.mass = t(masses)
        self.rho = torch.zeros(m.n_verts, dtype=torch.float64, device=d)
        self.cm = torch.zeros(m.grid, dtype=torch.float64, device=d)
        self.phi = torch.zeros(m.grid, dtype=torch.float64, device=d)
        sp = pkg.cdp_step_problem()
        sp.mesh = pkg.Projector.make_problem(self.pos, self.simp, self.rho, m.grid, m.box_lo, m.box_len, True, self.cm)
        for a in range(m.dim):
            sp.vel[a] = self.vel[a].data_ptr()
            sp.acc[a] = self.acc[a].data_ptr()
        sp.simplex_mass = self.mass.data_ptr()
        sp.phi = self.phi.data_ptr()
        self.sp = sp

    def state(self):
        c = lambda ts: np.stack([x.cpu().numpy() for x in ts])
        return c(self.pos), c(self.vel), self.rho.cpu().numpy(), self.cm.cpu().numpy(), self.phi.cpu().numpy(), c(
            self.acc)


def _periodic_diff(a, b, L=1.0):
    d = np.abs(a - b)
    return np.minimum(d, L - d)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_step_matches_oracle(ctx, use_graph):
    import paper_1509_07720_gb300 as pkg

    probs = _problems()
    devs = [_Dev(*p) for p in probs]
    arr = (pkg.cdp_step_problem * len(devs))(*[d.sp for d in devs])
    dt = 0.01
    rc = pkg.cdp_step_batched(ctx, arr, pkg.CDP_FP64, dt, FPG, use_graph, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    for (m, vel, masses), d in zip(probs, devs):
        p2, v2, rho, cm, phi, acc = _oracle_step(m, vel, masses, dt)
        gp, gv, grho, gcm, gphi, gacc = d.state()
        assert np.max(np.abs(grho - rho)) <= 1e-12 * np.max(rho)
        assert np.max(np.abs(gcm - cm)) <= 1e-11 * np.max(cm)
        assert np.max(np.abs(gphi - phi)) <= 1e-10 * np.max(np.abs(phi))
        assert np.max(np.abs(gacc - acc)) <= 1e-9 * np.max(np.abs(acc))
        assert np.max(np.abs(gv - v2)) <= 1e-9 * np.max(np.abs(v2))
        assert np.max(_periodic_diff(gp, p2)) <= 1e-12


def test_graph_replay_matches_eager(ctx):
    import paper_1509_07720_gb300 as pkg

    probs = _problems()
    a = [_Dev(*p) for p in probs]
    b = [_Dev(*p) for p in probs]
    arr_a = (pkg.cdp_step_problem * len(a))(*[d.sp for d in a])
    arr_b = (pkg.cdp_step_problem * len(b))(*[d.sp for d in b])
    st = torch.cuda.current_stream().cuda_stream
    for k, dt in enumerate((0.01, 0.012, 0.008)):
        assert pkg.cdp_step_batched(ctx, arr_a, pkg.CDP_FP64, dt, FPG, 1, st) == 0  # capture, then replays
        assert pkg.cdp_step_batched(ctx, arr_b, pkg.CDP_FP64, dt, FPG, 0, st) == 0
    torch.cuda.synchronize()
    for da, db in zip(a, b):
        sa, sb = da.state(), db.state()
        assert np.max(_periodic_diff(sa[0], sb[0])) <= 1e-13
        for x, y in zip(sa[1:], sb[1:]):
            assert np.max(np.abs(x - y)) <= 1e-11 * max(1e-300, np.max(np.abs(y)))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
def test_batched_workload_c5(ctx, prec):
    """The batched workload (64 problems, 2D and 3D, 18.3M simplices, grids 64..256 per axis) in one
    graph-captured step.  Every problem: the projected total equals the simplex masses of the
    drifted mesh at the step's own vertex densities.  The six smallest problems: the whole step
    against the oracle composition (FP64 strictly, FP32-mixed to its projection tolerance)."""
    import paper_1509_07720_gb300 as pkg

    batch = mg.make_batch("c5")
    dt = mg.cfl_dt(batch)
    devs = [_Dev(p.mesh, p.vel, p.masses) for p in batch]
    arr = (pkg.cdp_step_problem * len(devs))(*[d.sp for d in devs])
    st = torch.cuda.current_stream().cuda_stream
    assert pkg.cdp_step_batched(ctx, arr, prec, dt, FPG, 1, st) == 0
    torch.cuda.synchronize()
    small = set(np.argsort([p.mesh.n_simplices for p in batch])[:6].tolist())
    for i, (p, d) in enumerate(zip(batch, devs)):
        m = p.mesh
        gp, gv, grho, gcm, gphi, gacc = d.state()
        pos_mid = solver.drift(m.pos, p.vel, 0.5 * dt, m.box_lo, m.box_len)
        want_tot = oracle.simplex_mass(mg.Mesh(pos_mid, m.simplices, grho, m.grid, m.box_lo, m.box_len, True)).sum()
        assert abs(gcm.sum() - want_tot) <= 1e-12 * want_tot, f"problem {i}"
        if i not in small:
            continue
        p2, v2, rho, cm, phi, acc = _oracle_step(m, p.vel, p.masses, dt)
        assert np.max(np.abs(grho - rho)) <= 1e-12 * np.max(rho), f"problem {i}"
        if prec == 0:
            assert np.max(np.abs(gcm - cm)) <= 1e-11 * np.max(cm), f"problem {i}"
            assert np.max(np.abs(gphi - phi)) <= 1e-10 * np.max(np.abs(phi)), f"problem {i}"
            assert np.max(np.abs(gacc - acc)) <= 1e-9 * np.max(np.abs(acc)), f"problem {i}"
            assert np.max(np.abs(gv - v2)) <= 1e-9 * np.max(np.abs(v2)), f"problem {i}"
        else:
            assert np.max(np.abs(gcm - cm)) <= 1e-5 * np.max(cm), f"problem {i}"
            assert np.max(np.abs(gphi - phi)) <= 1e-4 * np.max(np.abs(phi)), f"problem {i}"
        assert np.max(_periodic_diff(gp, p2)) <= 1e-9, f"problem {i}"
