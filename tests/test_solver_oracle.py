"""Pins of the solver oracle (Poisson, force, kick-drift, vertex density) against closed forms."""
import numpy as np
import pytest

from oracle import solver
from paper_1509_07720_gb300 import meshgen as mg


@pytest.mark.parametrize("shape,box,axis,mode", [((32, 32), (1.0, 1.0), 0, 1), ((16, 24, 20), (1.0, 2.0, 1.5), 1, 2),
                                                 ((12, 10, 16), (1.0, 1.0, 2.0), 2, 3)])
def test_poisson_single_mode(shape, box, axis, mode):
    """rho = 1 + A sin(k x): laplacian(phi) = 4 pi G (rho - 1) gives phi = -4 pi G A sin(k x) / k^2."""
    d = len(shape)
    centres = [(np.arange(shape[a]) + 0.5) * box[a] / shape[a] for a in range(d)]
    X = np.meshgrid(*centres, indexing="ij")
    k = 2 * np.pi * mode / box[axis]
    A, fpg = 0.3, 1.7
    rho = 1.0 + A * np.sin(k * X[axis])
    cellvol = np.prod([box[a] / shape[a] for a in range(d)])
    phi = solver.poisson(rho * cellvol, box, fpg)
    expect = -fpg * A * np.sin(k * X[axis]) / k ** 2
    assert np.max(np.abs(phi - expect)) < 1e-13 * np.max(np.abs(expect)) + 1e-15


def test_poisson_mean_free_and_linear():
    rng = np.random.default_rng(1)
    m1 = rng.random((8, 12, 10))
    m2 = rng.random((8, 12, 10))
    box = (1.0, 1.5, 1.25)
    p1, p2 = solver.poisson(m1, box), solver.poisson(m2, box)
    p12 = solver.poisson(m1 + 3 * m2, box)
    assert abs(p1.mean()) < 1e-15
    assert np.max(np.abs(p12 - (p1 + 3 * p2))) < 1e-12 * np.max(np.abs(p12))


def test_grad4_closed_form_single_mode():
    """4-point difference of sin(kx) is cos(kx) (8 sin(kh) - sin(2kh)) / (6h)."""
    n, L = 24, 2.0
    h = L / n
    x = (np.arange(n) + 0.5) * h
    k = 2 * np.pi * 3 / L
    phi = np.sin(k * x)[:, None] * np.ones((1, 5))
    g = solver.grad4(phi, (L, 1.0))
    expect = np.cos(k * x) * (8 * np.sin(k * h) - np.sin(2 * k * h)) / (6 * h)
    assert np.max(np.abs(g[0][:, 0] - expect)) < 1e-12
    assert np.max(np.abs(g[1])) < 1e-12


def test_grad4_exact_for_cubics_in_the_interior():
    n = 40
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    phi = 2 * x ** 3 - x ** 2 + 0.5 * x
    g = solver.grad4(phi[:, None] * np.ones((1, 3)), (1.0, 1.0))[0][:, 0]
    exact = 6 * x ** 2 - 2 * x + 0.5
    assert np.max(np.abs(g[2:-2] - exact[2:-2])) < 1e-10


def test_tsc_constant_and_linear():
    rng = np.random.default_rng(2)
    n = 16
    field = np.full((n, n, n), 2.5)
    pos = rng.random((3, 200))
    assert np.max(np.abs(solver.tsc_interp(field, (0,) * 3, (1,) * 3, pos) - 2.5)) < 1e-14
    # linear in the cell index along x, probed away from the wrap-around
    i = np.arange(n, dtype=float)
    lin = (3.0 * i - 1.0)[:, None, None] * np.ones((1, n, n))
    p = np.stack([0.3 + 0.4 * rng.random(200), rng.random(200), rng.random(200)])
    got = solver.tsc_interp(lin, (0,) * 3, (1,) * 3, p)
    u = p[0] * n - 0.5
    assert np.max(np.abs(got - (3.0 * u - 1.0))) < 1e-12


def test_force_of_a_single_mode_at_cell_centres():
    """At a cell centre the TSC weights are (1/8, 3/4, 1/8)."""
    n, L = 32, 1.0
    h = L / n
    x = (np.arange(n) + 0.5) * h
    k = 2 * np.pi / L
    phi = np.sin(k * x)[:, None] * np.ones((1, 4))
    g = solver.grad4(phi, (L, L))[0][:, 0]
    pos = np.stack([x, np.full(n, 0.5 * h)])
    a = solver.force(phi, (0.0, 0.0), (L, L), pos)
    expect = -(0.125 * np.roll(g, 1) + 0.75 * g + 0.125 * np.roll(g, -1))
    assert np.max(np.abs(a[0] - expect)) < 1e-12 and np.max(np.abs(a[1])) < 1e-12


def test_vertex_density_recovers_uniform_density():
    q, t = mg.kuhn_mesh_3d(6)
    rng = np.random.default_rng(3)
    x = q + mg.grf_displacement(6, 3, 0.2, 2.0, rng)
    x -= np.floor(x)
    p = x[:, t]
    e = p[:, :, 1:] - p[:, :, :1]
    e -= np.round(e)
    vol = np.abs(np.einsum("ij,ij->j", e[:, :, 0], np.cross(e[:, :, 1].T, e[:, :, 2].T).T)) / 6
    rho = solver.vertex_density(x, t, 2.5 * vol, (1.0,) * 3)
    assert np.max(np.abs(rho - 2.5)) < 1e-12


def test_vertex_density_hand_case():
    pos = np.array([[0.0, 1.0, 0.0, 1.0], [0.0, 0.0, 1.0, 1.0]]) * 0.25
    simp = np.array([[0, 1, 2], [1, 3, 2]])
    rho = solver.vertex_density(pos, simp, np.array([1.0, 3.0]), (1.0, 1.0))
    area = 0.25 * 0.25 / 2
    assert np.allclose(rho, [1.0 / area, 4.0 / (2 * area), 4.0 / (2 * area), 3.0 / area], rtol=1e-14)


def test_leapfrog_energy_second_order():
    """Drift-kick-drift on a harmonic force conserves energy to O(dt^2)."""
    errs = []
    for dt in (0.02, 0.01):
        x = np.array([[1.0]])
        v = np.array([[0.0]])
        e0 = 0.5 * (x ** 2 + v ** 2)
        for _ in range(int(round(10 / dt))):
            x = x + 0.5 * dt * v
            v = solver.kick(v, -x, dt)
            x = x + 0.5 * dt * v
        errs.append(float(np.max(np.abs(0.5 * (x ** 2 + v ** 2) - e0))))
    assert errs[1] < 0.3 * errs[0]


def test_drift_wraps_into_box():
    pos = np.array([[0.95, 0.1]])
    vel = np.array([[1.0, -1.0]])
    out = solver.drift(pos, vel, 0.1, (0.0,), (1.0,))
    assert np.allclose(out, [[0.05, 0.0]], atol=1e-15)
