"""Oracle of the projection through coarser levels with donor-cell gather (TEST INFRASTRUCTURE ONLY).

Sect. 4.4 (calculation of the acceleration) projects the mesh exactly onto the cells of an AMR grid
that is refined while a cell is larger than the smallest perpendicular height of the simplices
crossing it, then gives the uniform grid of the Poisson solve the AMR masses by donor-cell
interpolation.  This module computes the per-simplex reading of that scheme, written out step by
step from its definition:

1. the smallest perpendicular height eta of every simplex, in cells of the output grid
   (D |volume| / largest facet measure: the height onto the largest facet);
2. its level l = min(max_level, floor(log2 eta)), and 0 when eta < 2 (cells of level l are 2^l
   output cells wide, so a level's cells are no wider than eta);
3. for every level, the exact projection (the oracle's ``project``) of the simplices of that level
   onto the grid with every axis divided by 2^l;
4. the donor-cell gather: every output cell takes its own level-0 mass plus, for each l >= 1, the
   mass of the level-l cell that contains it divided by 2^(D l).

Only ``tests/`` import this module.
"""
from __future__ import annotations

import numpy as np

from . import project


def simplex_heights(mesh) -> np.ndarray:
    """Smallest perpendicular height of every simplex in cells of ``mesh.grid`` (float64), taken at
    the minimal image of vertex 0 on a periodic box (vertex 0's displacement to the others)."""
    d = mesh.dim
    grid = np.asarray(mesh.grid, dtype=np.float64)
    ln = np.asarray(mesh.box_len, dtype=np.float64)
    x = mesh.pos.T[mesh.simplices] * (grid / ln)  # [ns, D+1, D] in cells
    e = x[:, 1:, :] - x[:, :1, :]
    if mesh.periodic:
        e = e - grid * np.round(e / grid)
    ns = mesh.simplices.shape[0]
    if d == 3:
        vol6 = np.abs(np.einsum("ni,ni->n", np.cross(e[:, 0], e[:, 1]), e[:, 2]))
        # the four facets: their normals are twice their areas
        p = np.concatenate([np.zeros((ns, 1, 3)), e], axis=1)
        amax = np.zeros(ns)
        for f in range(4):
            a, b, c = [k for k in range(4) if k != f]
            n = np.cross(p[:, b] - p[:, a], p[:, c] - p[:, a])
            amax = np.maximum(amax, np.sqrt(np.einsum("ni,ni->n", n, n)))
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(amax > 0, vol6 / amax, 0.0)
    area2 = np.abs(e[:, 0, 0] * e[:, 1, 1] - e[:, 0, 1] * e[:, 1, 0])
    p = np.concatenate([np.zeros((ns, 1, 2)), e], axis=1)
    lmax = np.zeros(ns)
    for k in range(3):
        a, b = (k + 1) % 3, (k + 2) % 3
        v = p[:, b] - p[:, a]
        lmax = np.maximum(lmax, np.sqrt(np.einsum("ni,ni->n", v, v)))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(lmax > 0, area2 / lmax, 0.0)


def amr_levels(mesh, max_level: int) -> np.ndarray:
    """Level of every simplex: min(max_level, floor(log2 eta)), 0 for eta < 2."""
    eta = simplex_heights(mesh)
    lev = np.zeros(eta.shape, dtype=np.int64)
    for l in range(1, max_level + 1):
        lev[eta >= float(1 << l)] = l
    return lev


def level_mesh(mesh, simplices_mask, level: int):
    """The simplices selected by the mask, on the grid of the given level."""
    from dataclasses import replace

    grid = tuple(int(n) >> level for n in mesh.grid)
    return replace(mesh, simplices=np.ascontiguousarray(mesh.simplices[simplices_mask]), grid=grid)


def donor_gather(level_masses, dim: int) -> np.ndarray:
    """Sum over the levels of every level's masses spread evenly over the output cells it covers:
    out[i] = sum_l m_l[i >> l] / 2^(D l)."""
    out = np.array(level_masses[0], dtype=np.float64, copy=True)
    for l, m in enumerate(level_masses):
        if l == 0:
            continue
        up = m
        for a in range(dim):
            up = np.repeat(up, 1 << l, axis=a)
        out += up / float(1 << (dim * l))
    return out


def project_amr(mesh, max_level: int, nthreads: int = 0):
    """Output-grid masses of the projection through the levels 0 .. max_level (steps 1-4 above)."""
    for n in mesh.grid:
        if n % (1 << max_level):
            raise ValueError("grid not divisible by 2^max_level")
    lev = amr_levels(mesh, max_level)
    masses = []
    for l in range(max_level + 1):
        sub = level_mesh(mesh, lev == l, l)
        masses.append(project(sub, nthreads=nthreads))
    return donor_gather(masses, mesh.dim)


def block_sums(m: np.ndarray, level: int) -> np.ndarray:
    """Masses summed over aligned blocks of 2^level cells per axis (the grid of that level)."""
    s = m
    for a in range(m.ndim):
        shp = list(s.shape)
        shp[a:a + 1] = [shp[a] >> level, 1 << level]
        s = s.reshape(shp).sum(axis=a + 1)
    return s

