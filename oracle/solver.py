"""CPU oracle for the steps around the projection in one Vlasov-Poisson time step (TEST
INFRASTRUCTURE ONLY; only tests/, the smoke check and bench.py's CPU baseline use it).

Plain numpy restatements, in FP64, of what the paper's solver computes (Sect. 4, steps (ii)-(iv);
Sect. 4.4 calculation of the acceleration):

* vertex_density   rho_j = sum of M_i over simplices incident to j / sum of |V_i| over the same
                   simplices (Sect. 4.4, the formula for rho_j).
* poisson          periodic FFT solution of  laplacian(phi) = four_pi_G (rho - mean rho), with the
                   continuous Green function -1/k^2 (k = 2 pi n / L) and the zero mode removed
                   (Sect. 4.4: "Poisson equation is solved ... with FFTW"). numpy's FFT is the
                   library step.
* force            acceleration at a point = - sum over the 3^D nearest cell centres of the TSC
                   weight times the 4-point central difference of phi at that cell,
                   (8 (phi[i+1] - phi[i-1]) - (phi[i+2] - phi[i-2])) / (12 h)  (Sect. 4.4: 4-point
                   central difference combined with dual TSC interpolation).
* drift, kick      x += u dt ; u += a dt (eqs. drift1, kick, drift2).

Readings (the paper does not fix them): cell-centred grid (cell i centred at lo + (i + 1/2) h);
TSC weights 3/4 - d^2 and (1/2 +- d)^2 / 2 for the nearest cell and its two neighbours, d the
offset from the nearest centre in cells; positions wrapped into the periodic box after a drift.
"""
from __future__ import annotations

import numpy as np


def vertex_density(pos, simplices, masses, box_len, periodic=True):
    """rho_j = (sum_i M_i) / (sum_i |V_i|), the sums taken over the simplices i that have vertex j.

    pos [D, Nv], simplices [Ns, D+1], masses [Ns]. Vertices with no simplex get 0."""
    d = pos.shape[0]
    p = pos[:, simplices]  # [D, Ns, D+1]
    e = p[:, :, 1:] - p[:, :, :1]
    if periodic:
        L = np.asarray(box_len, dtype=np.float64).reshape(d, 1, 1)
        e = e - L * np.round(e / L)
    if d == 3:
        vol = np.abs(np.einsum("ij,ij->j", e[:, :, 0], np.cross(e[:, :, 1].T, e[:, :, 2].T).T)) / 6.0
    else:
        vol = np.abs(e[0, :, 0] * e[1, :, 1] - e[1, :, 0] * e[0, :, 1]) / 2.0
    nv = pos.shape[1]
    msum = np.zeros(nv)
    vsum = np.zeros(nv)
    for k in range(d + 1):
        np.add.at(msum, simplices[:, k], masses)
        np.add.at(vsum, simplices[:, k], vol)
    out = np.zeros(nv)
    nz = vsum > 0
    out[nz] = msum[nz] / vsum[nz]
    return out


def poisson(cell_mass, box_len, four_pi_G=1.0):
    """phi on the cell-centred periodic grid from cell masses."""
    shape = cell_mass.shape
    d = len(shape)
    cellvol = float(np.prod([box_len[a] / shape[a] for a in range(d)]))
    rho = cell_mass / cellvol
    rk = np.fft.rfftn(rho - rho.mean(), axes=tuple(range(d)))
    ks = [2 * np.pi * np.fft.fftfreq(shape[a], d=box_len[a] / shape[a]) for a in range(d - 1)]
    ks.append(2 * np.pi * np.fft.rfftfreq(shape[-1], d=box_len[-1] / shape[-1]))
    kk = np.meshgrid(*ks, indexing="ij")
    k2 = sum(k * k for k in kk)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(k2 > 0, -four_pi_G / k2, 0.0)
    return np.fft.irfftn(rk * g, s=shape, axes=tuple(range(d)))


def grad4(phi, box_len):
    """4-point central difference of phi along every axis (periodic): list of D arrays."""
    out = []
    for a in range(phi.ndim):
        h = box_len[a] / phi.shape[a]
        p1 = np.roll(phi, -1, axis=a)
        m1 = np.roll(phi, 1, axis=a)
        p2 = np.roll(phi, -2, axis=a)
        m2 = np.roll(phi, 2, axis=a)
        out.append((8.0 * (p1 - m1) - (p2 - m2)) / (12.0 * h))
    return out


def tsc_interp(field, box_lo, box_len, pos):
    """Triangular-shaped-cloud interpolation of a cell-centred periodic field at points [D, N]."""
    import itertools

    d = field.ndim
    n = pos.shape[1]
    centre, wts = [], []
    for a in range(d):
        h = box_len[a] / field.shape[a]
        u = (pos[a] - box_lo[a]) / h - 0.5
        i0 = np.floor(u + 0.5).astype(np.int64)
        dd = u - i0
        centre.append(i0)
        wts.append([0.5 * (0.5 - dd) ** 2, 0.75 - dd * dd, 0.5 * (0.5 + dd) ** 2])
    out = np.zeros(n)
    for offs in itertools.product((-1, 0, 1), repeat=d):
        w = np.ones(n)
        idx = []
        for a in range(d):
            w = w * wts[a][offs[a] + 1]
            idx.append((centre[a] + offs[a]) % field.shape[a])
        out += w * field[tuple(idx)]
    return out


def force(phi, box_lo, box_len, pos):
    """Acceleration -grad(phi) at points pos [D, N]: TSC interpolation of the 4-point gradient."""
    grads = grad4(phi, box_len)
    return np.stack([-tsc_interp(g, box_lo, box_len, pos) for g in grads])


def drift(pos, vel, dt, box_lo, box_len, periodic=True):
    out = pos + vel * dt
    if periodic:
        lo = np.asarray(box_lo, dtype=np.float64).reshape(-1, 1)
        L = np.asarray(box_len, dtype=np.float64).reshape(-1, 1)
        out = lo + np.mod(out - lo, L)
    return out


def kick(vel, acc, dt):
    return vel + acc * dt
