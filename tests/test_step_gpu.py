"""A batched time step (drift, vertex density, projection, Poisson, force, kick, drift) through the
C ABI against the oracle composition of the same steps; the CUDA-graph replay against eager
execution."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import solver
from paper_1509_07720_gb300 import meshgen as mg
from parity_report import record

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


def test_step_more_meshes_than_one_group(ctx):
    """70 meshes: the per-vertex kernels and the FP32 Poisson conversions run over tables of at
    most 64 meshes, so the step takes two groups.  Graph replay against eager execution for all of
    them (to the run-to-run noise of the atomic sums, which the potential and the force amplify:
    2.3e-13 in the positions after one FP64 step was seen), and the two meshes of the second group
    against the oracle composition."""
    import paper_1509_07720_gb300 as pkg

    rng = np.random.default_rng(31)
    base = _problems()
    probs = []
    for i in range(70):
        m, vel, masses = base[i % 2]
        probs.append((m, 0.05 * rng.standard_normal(m.pos.shape), masses))
    a = [_Dev(*p) for p in probs]
    b = [_Dev(*p) for p in probs]
    arr_a = (pkg.cdp_step_problem * len(a))(*[d.sp for d in a])
    arr_b = (pkg.cdp_step_problem * len(b))(*[d.sp for d in b])
    st = torch.cuda.current_stream().cuda_stream
    dt = 0.01
    for prec in (pkg.CDP_FP64, pkg.CDP_FP32_MIXED):
        assert pkg.cdp_step_batched(ctx, arr_a, prec, dt, FPG, 1, st) == 0
        assert pkg.cdp_step_batched(ctx, arr_b, prec, dt, FPG, 0, st) == 0
        torch.cuda.synchronize()
        tol_pos, tol_rel = (1e-11, 1e-9) if prec == pkg.CDP_FP64 else (1e-8, 1e-4)
        for da, db in zip(a, b):
            sa, sb = da.state(), db.state()
            assert np.max(_periodic_diff(sa[0], sb[0])) <= tol_pos
            for x, y in zip(sa[1:], sb[1:]):
                assert np.max(np.abs(x - y)) <= tol_rel * max(1e-300, np.max(np.abs(y)))
        if prec == pkg.CDP_FP64:
            # one FP64 step from the initial state: the second group against the oracle
            for i in (64, 69):
                m, vel, masses = probs[i]
                p2, v2, rho, cm, phi, acc = _oracle_step(m, vel, masses, dt)
                gp, gv, grho, gcm, gphi, gacc = a[i].state()
                assert np.max(np.abs(grho - rho)) <= 1e-12 * np.max(rho), f"mesh {i}"
                assert np.max(np.abs(gcm - cm)) <= 1e-11 * np.max(cm), f"mesh {i}"
                assert np.max(np.abs(gphi - phi)) <= 1e-10 * np.max(np.abs(phi)), f"mesh {i}"
                assert np.max(np.abs(gacc - acc)) <= 1e-9 * np.max(np.abs(acc)), f"mesh {i}"
                assert np.max(_periodic_diff(gp, p2)) <= 1e-12, f"mesh {i}"


def test_graph_recorded_again_after_scratch_moves(ctx):
    """A graph holds the addresses of the context's scratch.  Projecting a larger mesh and computing
    a larger vertex density on the same context reallocates that scratch; the next call with the
    graph's arguments must record the step again (not replay stale addresses) and still equal
    eager execution."""
    import paper_1509_07720_gb300 as pkg

    probs = _problems()
    a = [_Dev(*p) for p in probs]
    b = [_Dev(*p) for p in probs]
    arr_a = (pkg.cdp_step_problem * len(a))(*[d.sp for d in a])
    arr_b = (pkg.cdp_step_problem * len(b))(*[d.sp for d in b])
    st = torch.cuda.current_stream().cuda_stream
    assert pkg.cdp_step_batched(ctx, arr_a, pkg.CDP_FP64, 0.01, FPG, 1, st) == 0
    assert pkg.cdp_step_batched(ctx, arr_b, pkg.CDP_FP64, 0.01, FPG, 0, st) == 0
    # a mesh with more vertices and simplices than any the context has seen in this module
    big = mg.make_config("c2", 40)
    d = torch.device("cuda:0")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(d)
    pos = [t(big.pos[k]) for k in range(3)]
    simp, rho = t(big.simplices), t(big.rho)
    out = torch.empty(big.grid, dtype=torch.float64, device=d)
    prob = pkg.Projector.make_problem(pos, simp, rho, big.grid, big.box_lo, big.box_len, big.periodic, out)
    assert pkg.cdp_project(ctx, prob, pkg.CDP_FP32_MIXED, 0, st) == 0
    rout = torch.empty(big.n_verts, dtype=torch.float64, device=d)
    masses = t(np.full(big.n_simplices, 1e-5))
    assert pkg.cdp_vertex_density(ctx, prob, masses.data_ptr(), rout.data_ptr(), st) == 0
    torch.cuda.synchronize()
    del pos, simp, rho, out, rout, masses
    for dt in (0.012, 0.008):
        assert pkg.cdp_step_batched(ctx, arr_a, pkg.CDP_FP64, dt, FPG, 1, st) == 0
        assert pkg.cdp_step_batched(ctx, arr_b, pkg.CDP_FP64, dt, FPG, 0, st) == 0
    torch.cuda.synchronize()
    for da, db in zip(a, b):
        sa, sb = da.state(), db.state()
        assert np.max(_periodic_diff(sa[0], sb[0])) <= 1e-13
        for x, y in zip(sa[1:], sb[1:]):
            assert np.max(np.abs(x - y)) <= 1e-11 * max(1e-300, np.max(np.abs(y)))


_C5 = {}


def _c5_oracle(batch, dt):
    """The oracle composition up to the projection for every problem of the batch (drift dt/2,
    vertex densities, projection), computed once: the large 3D problems take the oracle minutes."""
    if "proj" not in _C5:
        res = []
        for p in batch:
            m = p.mesh
            pos = solver.drift(m.pos, p.vel, 0.5 * dt, m.box_lo, m.box_len)
            rho = solver.vertex_density(pos, m.simplices, p.masses, m.box_len)
            cm = oracle.project(mg.Mesh(pos, m.simplices, rho, m.grid, m.box_lo, m.box_len, True))
            res.append((pos, rho, cm))
        _C5["proj"] = res
    return _C5["proj"]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32mixed"])
def test_batched_workload_c5(ctx, prec):
    """The batched workload (64 problems, 2D and 3D, 18.3M simplices, grids 64..256 per axis) in one
    graph-captured step.  Every problem, every cell: the projected grid against the oracle's
    projection of the oracle's own drifted mesh and vertex densities (1e-11 FP64, 1e-5 FP32-mixed of
    the largest cell; this includes the 21 3D problems whose tetrahedra are tiled), and the total
    mass.  The six smallest problems: the rest of the step (potential, forces, kick, drift) too."""
    import paper_1509_07720_gb300 as pkg

    batch = mg.make_batch("c5")
    dt = mg.cfl_dt(batch)
    devs = [_Dev(p.mesh, p.vel, p.masses) for p in batch]
    arr = (pkg.cdp_step_problem * len(devs))(*[d.sp for d in devs])
    st = torch.cuda.current_stream().cuda_stream
    assert pkg.cdp_step_batched(ctx, arr, prec, dt, FPG, 1, st) == 0
    torch.cuda.synchronize()
    ref = _c5_oracle(batch, dt)
    small = set(np.argsort([p.mesh.n_simplices for p in batch])[:6].tolist())
    tol = 1e-11 if prec == 0 else 1e-5
    worst, worst_tot, cells, worst_phi, phi_cells = 0.0, 0.0, 0, 0.0, 0
    for i, (p, d, (pos_mid, rho_mid, cm_mid)) in enumerate(zip(batch, devs, ref)):
        gp, gv, grho, gcm, gphi, gacc = d.state()
        assert np.max(np.abs(grho - rho_mid)) <= 1e-12 * np.max(rho_mid), f"problem {i}"
        scale = float(np.max(np.abs(cm_mid)))
        err = float(np.max(np.abs(gcm - cm_mid))) / scale
        worst = max(worst, err)
        worst_tot = max(worst_tot, abs(gcm.sum() - cm_mid.sum()) / abs(cm_mid.sum()))
        cells += int(gcm.size)
        if i == len(batch) - 1:
            record("c5_step", prec, max_rel=worst, total_rel=worst_tot, cells=cells, problems=len(batch))
        assert err <= tol, f"problem {i} (dim {p.mesh.dim}, {p.mesh.n_simplices} simplices): {err:.3e}"
        assert abs(gcm.sum() - cm_mid.sum()) <= 1e-12 * abs(cm_mid.sum()), f"problem {i}"
        if i not in small:
            continue
        m = p.mesh
        p2, v2, rho, cm, phi, acc = _oracle_step(m, p.vel, p.masses, dt)
        phi_err = float(np.max(np.abs(gphi - phi)) / np.max(np.abs(phi)))
        worst_phi = max(worst_phi, phi_err)
        phi_cells += int(gphi.size)
        record("c5_step_potential", prec, max_rel=worst_phi, total_rel=0.0, cells=phi_cells, problems=len(small))
        if prec == 0:
            assert np.max(np.abs(gphi - phi)) <= 1e-10 * np.max(np.abs(phi)), f"problem {i}"
            assert np.max(np.abs(gacc - acc)) <= 1e-9 * np.max(np.abs(acc)), f"problem {i}"
            assert np.max(np.abs(gv - v2)) <= 1e-9 * np.max(np.abs(v2)), f"problem {i}"
        else:
            assert np.max(np.abs(gphi - phi)) <= 1e-4 * np.max(np.abs(phi)), f"problem {i}"
        assert np.max(_periodic_diff(gp, p2)) <= 1e-9, f"problem {i}"
