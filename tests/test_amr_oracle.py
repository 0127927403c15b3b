"""Pins of the oracle of the projection through coarser levels with donor-cell gather (Sect. 4.4,
calculation of the acceleration), no GPU.

The pins fix each step to something other than the oracle itself:
  heights   closed forms of the smallest perpendicular height (Kuhn simplices: edge / sqrt 2;
            regular tetrahedron: edge sqrt(2/3); equilateral triangle: edge sqrt(3) / 2; right
            triangle: the altitude on the hypotenuse), invariance under a periodic wrap;
  levels    the definition floor(log2 eta) on simplices of chosen heights;
  gather    the projection onto a level's grid is the exact projection summed over blocks of
            2^l cells, so every block sum of the AMR result at the deepest level equals that of the
            exact projection; total mass; a mesh of one level gives masses constant on its blocks;
            max_level 0 is the exact projection.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import amr
from paper_1509_07720_gb300 import meshgen as mg


def _one(verts, grid, periodic=True):
    v = np.asarray(verts, dtype=np.float64)
    d = v.shape[1]
    return mg.Mesh(np.ascontiguousarray(v.T), np.arange(d + 1, dtype=np.int32)[None, :], np.ones(d + 1),
                   (grid,) * d, (0.0,) * d, (1.0,) * d, periodic)


def test_heights_kuhn_closed_form():
    for n, grid in ((4, 16), (4, 32), (8, 16)):
        q, t = mg.kuhn_mesh_3d(n)
        m = mg.Mesh(q, t, np.ones(q.shape[1]), (grid,) * 3, (0.0,) * 3, (1.0,) * 3, True)
        eta = amr.simplex_heights(m)
        assert np.allclose(eta, (grid / n) / math.sqrt(2.0), rtol=1e-12, atol=0)
        q, t = mg.square_mesh_2d(n)
        m = mg.Mesh(q, t, np.ones(q.shape[1]), (grid,) * 2, (0.0,) * 2, (1.0,) * 2, True)
        assert np.allclose(amr.simplex_heights(m), (grid / n) / math.sqrt(2.0), rtol=1e-12, atol=0)


def test_heights_regular_and_right_triangle():
    s = 0.25  # box lengths; grid 64 -> 16 cells
    reg = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    reg *= s / (2.0 * math.sqrt(2.0))  # edge s
    m = _one(reg + 0.5, 64)
    assert amr.simplex_heights(m)[0] == pytest.approx(16.0 * math.sqrt(2.0 / 3.0), rel=1e-12)
    tri = np.array([[0.0, 0.0], [s, 0.0], [s / 2, s * math.sqrt(3.0) / 2]]) + 0.3
    assert amr.simplex_heights(_one(tri, 64))[0] == pytest.approx(16.0 * math.sqrt(3.0) / 2, rel=1e-12)
    a, b = 3.0, 7.0  # legs in cells
    rt = np.array([[0.0, 0.0], [a, 0.0], [0.0, b]]) / 64 + 0.2
    assert amr.simplex_heights(_one(rt, 64))[0] == pytest.approx(a * b / math.hypot(a, b), rel=1e-12)


def test_heights_periodic_wrap():
    """A simplex across the periodic boundary has the height of its unwrapped copy."""
    tri = np.array([[0.0, 0.0], [5.0, 0.0], [1.0, 4.0]]) / 32
    inside = amr.simplex_heights(_one(tri + 0.4, 32))[0]
    wrapped = np.mod(tri - 0.02, 1.0)
    assert amr.simplex_heights(_one(wrapped, 32))[0] == pytest.approx(inside, rel=1e-12)


def test_levels_definition():
    # right triangles with legs a = b: eta = a / sqrt 2
    rng = np.random.default_rng(3)
    for a_cells, want in ((1.0, 0), (2.5, 0), (3.0, 1), (5.0, 1), (6.0, 2), (12.0, 3), (24.0, 4), (90.0, 4)):
        base = rng.uniform(0.2, 0.4, 2)
        tri = np.array([[0.0, 0.0], [a_cells, 0.0], [0.0, a_cells]]) / 256 + base
        lev = amr.amr_levels(_one(tri, 256), 4)[0]
        assert lev == want, (a_cells, lev, want)


def _mixed(dim, grid, seed):
    rng = np.random.default_rng(seed)
    # (offsets of at most `size` cells: spans below half the periodic box)
    sizes = ((60, 0.8), (40, 3.0), (40, 7.0)) if dim == 3 else ((200, 1.0), (100, 4.0), (60, 8.0), (40, 15.0))
    return mg.mixed_size_simplices(dim, grid, sizes, rng)


@pytest.mark.parametrize("dim,grid,lmax", [(3, 32, 2), (2, 64, 3)])
def test_block_sums_and_total(dim, grid, lmax):
    m = _mixed(dim, grid, 11 + dim)
    lev = amr.amr_levels(m, lmax)
    assert len(set(lev.tolist())) == lmax + 1  # every level is used
    got = amr.project_amr(m, lmax)
    ref = oracle.project(m)
    assert abs(got.sum() - ref.sum()) <= 1e-12 * abs(ref.sum())
    bs_got, bs_ref = amr.block_sums(got, lmax), amr.block_sums(ref, lmax)
    assert np.max(np.abs(bs_got - bs_ref)) <= 1e-12 * np.max(np.abs(bs_ref))
    # and the AMR result differs from the exact one (coarse levels are spread evenly)
    assert np.max(np.abs(got - ref)) > 1e-6 * np.max(np.abs(ref))


def test_one_level_is_blockwise_constant():
    q, t = mg.kuhn_mesh_3d(4)  # grid 16: edge 4 cells, eta 2.83 -> level 1
    rng = np.random.default_rng(5)
    m = mg.Mesh(q + 0.013, t, mg.lognormal_density(q.shape[1], 0.5, rng), (16,) * 3, (0.0,) * 3, (1.0,) * 3, True)
    assert np.all(amr.amr_levels(m, 3) == 1)
    got = amr.project_amr(m, 3)
    coarse = oracle.project(mg.Mesh(m.pos, m.simplices, m.rho, (8,) * 3, m.box_lo, m.box_len, True))
    want = np.repeat(np.repeat(np.repeat(coarse, 2, 0), 2, 1), 2, 2) / 8.0
    # (the oracle's threads add pieces in no fixed order: equal up to rounding)
    assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))
    blocks = got.reshape(8, 2, 8, 2, 8, 2)
    assert np.max(np.ptp(blocks, axis=(1, 3, 5))) <= 1e-14 * np.max(np.abs(want))


def test_level_zero_is_exact():
    m = _mixed(3, 32, 21)
    ref = oracle.project(m)
    assert np.max(np.abs(amr.project_amr(m, 0) - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_rejects_indivisible_grid():
    m = _mixed(2, 48, 2)
    with pytest.raises(ValueError):
        amr.project_amr(m, 5)
