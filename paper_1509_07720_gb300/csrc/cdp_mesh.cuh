// Vertex records and per-simplex canonicalisation (periodic unwrap, orientation, cells).
#pragma once

#include "cdp_franklin.cuh"

namespace cdp {

// Error bits raised by the kernels (combined with atomicOr into the context's flag word).
enum : unsigned {
    CDP_FLAG_INDEX = 1u,   // a simplex refers to a vertex outside [0, n_verts)
    CDP_FLAG_NAN = 2u,     // a non-finite coordinate or a coordinate out of the fixed-point range
    CDP_FLAG_EXTENT = 4u,  // a simplex spans half a periodic box, or more than CDP_MAX_EXTENT cells
};

// One vertex in the layout the projection reads: fixed-point grid coordinates (wrapped into
// [0, N) on periodic axes) and the density, 32 bytes so that one gather is one sector.
struct __align__(32) VertexRec {
    i64 x[3];
    double rho;
};

struct GridDesc {
    int dim;
    int n[3];
    double lo[3];
    double inv_h[3];    // cells per unit length
    double cell_volume; // world volume of one cell: densities are stored premultiplied by it, so
                        // every contribution (computed in cell units) is directly a world mass
    int periodic;
};

// World coordinates -> fixed point (grid units * 2^Q); returns 0 or an error flag.
CDP_HD unsigned vertex_to_fixed(const GridDesc& g, const double p[3], double rho, VertexRec& out) {
    unsigned flag = 0;
    for (int a = 0; a < 3; ++a) {
        if (a >= g.dim) {
            out.x[a] = 0;
            continue;
        }
        double u = (p[a] - g.lo[a]) * g.inv_h[a];
        if (!(u == u) || u > 1.0e6 || u < -1.0e6) {  // NaN / infinite / absurd
            flag |= CDP_FLAG_NAN;
            u = 0.0;
        }
        if (g.periodic) {
            // wrap into [0, N) (a coordinate already inside takes no division: the FP64 divide is
            // slow, and the fixed-point wrap below gives the same code either way)
            const double N = (double)g.n[a];
            if (!(u >= 0.0 && u < N)) u -= N * floor(u / N);
        }
        i64 X = (i64)llrint(ldexp(u, CDP_Q));
        if (g.periodic) {
            i64 NQ = (i64)g.n[a] << CDP_Q;
            if (X >= NQ) X -= NQ;
            if (X < 0) X += NQ;
        }
        out.x[a] = X;
    }
    out.rho = rho * g.cell_volume;
    if (!(rho == rho) || rho > 1.0e300 || rho < -1.0e300) flag |= CDP_FLAG_NAN;
    return flag;
}

// displacement of vertex coordinate d relative to vertex 0, minimal image on periodic axes
CDP_HD bool unwrap(i64& d, int n, int periodic) {
    if (!periodic) return true;
    i64 NQ = (i64)n << CDP_Q, half = (i64)n << (CDP_Q - 1);
    if (d > half) d -= NQ;
    if (d < -half) d += NQ;
    return d != half && d != -half;
}

// On a periodic axis the unwrapped simplex must span less than half the box: then every vertex is
// also the minimal image of every other one, so the simplex (and its projection) does not depend on
// which vertex is listed first.
CDP_HD bool extent_ok(i64 a, i64 b, i64 c, i64 d, int n, int periodic) {
    if (!periodic) return true;
    const i64 ab0 = a < b ? a : b, cd0 = c < d ? c : d, ab1 = a < b ? b : a, cd1 = c < d ? d : c;
    const i64 mn = ab0 < cd0 ? ab0 : cd0, mx = ab1 < cd1 ? cd1 : ab1;
    return mx - mn < ((i64)n << (CDP_Q - 1));
}

// Canonical tetrahedron from its 4 vertex records.  Returns 0 (ok), 1 (zero volume: contributes
// nothing) or an error flag.  COPY only gives a caller its own out-of-line instance.
template <int COPY = 0>
CDP_COLD unsigned canon_tet(const GridDesc& g, const VertexRec* v[4], Tet& S) {
    const i64 lim = (i64)CDP_MAX_EXTENT << CDP_Q;
    for (int a = 0; a < 3; ++a) {
        i64 X0 = v[0]->x[a];
        i64 A = X0 >> CDP_Q;  // floor
        S.anchor[a] = (int)A;
        i64 base = X0 - (A << CDP_Q);
        S.L[0][a] = base;
        for (int k = 1; k < 4; ++k) {
            i64 d = v[k]->x[a] - X0;
            if (!unwrap(d, g.n[a], g.periodic)) return CDP_FLAG_EXTENT;
            if (d > lim || d < -lim) return CDP_FLAG_EXTENT;
            S.L[k][a] = base + d;
        }
        if (!extent_ok(S.L[0][a], S.L[1][a], S.L[2][a], S.L[3][a], g.n[a], g.periodic)) return CDP_FLAG_EXTENT;
    }
    for (int k = 0; k < 4; ++k) S.rho[k] = v[k]->rho;
    // orientation: sign of (x3-x0) . ((x1-x0) x (x2-x0)); make it positive by swapping 2 and 3
    i64 e1[3], e2[3], e3[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = S.L[1][a] - S.L[0][a];
        e2[a] = S.L[2][a] - S.L[0][a];
        e3[a] = S.L[3][a] - S.L[0][a];
    }
    i128 n3[3];
    cross_exact(e1, e2, n3);
    int s = sgn_wide(dot3_wide(n3, e3));
    if (s == 0) return 1;
    if (s < 0) {
        for (int a = 0; a < 3; ++a) {
            i64 t = S.L[2][a];
            S.L[2][a] = S.L[3][a];
            S.L[3][a] = t;
        }
        double t = S.rho[2];
        S.rho[2] = S.rho[3];
        S.rho[3] = t;
    }
    for (int a = 0; a < 3; ++a) {
        S.lo[a] = 1 << 30;
        S.hi[a] = -(1 << 30);
        for (int k = 0; k < 4; ++k) {
            int c = (int)(S.L[k][a] >> CDP_Q);
            S.cell[k][a] = c;
            S.lo[a] = c < S.lo[a] ? c : S.lo[a];
            S.hi[a] = c > S.hi[a] ? c : S.hi[a];
        }
    }
    return 0;
}

CDP_COLD unsigned canon_tri(const GridDesc& g, const VertexRec* v[3], Tri& S) {
    const i64 lim = (i64)CDP_MAX_EXTENT << CDP_Q;
    for (int a = 0; a < 2; ++a) {
        i64 X0 = v[0]->x[a];
        i64 A = X0 >> CDP_Q;
        S.anchor[a] = (int)A;
        i64 base = X0 - (A << CDP_Q);
        S.L[0][a] = base;
        for (int k = 1; k < 3; ++k) {
            i64 d = v[k]->x[a] - X0;
            if (!unwrap(d, g.n[a], g.periodic)) return CDP_FLAG_EXTENT;
            if (d > lim || d < -lim) return CDP_FLAG_EXTENT;
            S.L[k][a] = base + d;
        }
        if (!extent_ok(S.L[0][a], S.L[1][a], S.L[2][a], S.L[2][a], g.n[a], g.periodic)) return CDP_FLAG_EXTENT;
    }
    for (int k = 0; k < 3; ++k) S.rho[k] = v[k]->rho;
    i128 D = mul64(S.L[1][0] - S.L[0][0], S.L[2][1] - S.L[0][1]) -
             mul64(S.L[1][1] - S.L[0][1], S.L[2][0] - S.L[0][0]);
    if (D == 0) return 1;
    if (D < 0) {
        for (int a = 0; a < 2; ++a) {
            i64 t = S.L[1][a];
            S.L[1][a] = S.L[2][a];
            S.L[2][a] = t;
        }
        double t = S.rho[1];
        S.rho[1] = S.rho[2];
        S.rho[2] = t;
    }
    for (int a = 0; a < 2; ++a) {
        S.lo[a] = 1 << 30;
        S.hi[a] = -(1 << 30);
        for (int k = 0; k < 3; ++k) {
            int c = (int)(S.L[k][a] >> CDP_Q);
            S.cell[k][a] = c;
            S.lo[a] = c < S.lo[a] ? c : S.lo[a];
            S.hi[a] = c > S.hi[a] ? c : S.hi[a];
        }
    }
    return 0;
}

// Exact mass of a tetrahedron, |V| mean(rho) (densities premultiplied by the cell volume), in double.
CDP_HD double tet_mass_cells(const Tet& S) {
    i64 e1[3], e2[3], e3[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = S.L[1][a] - S.L[0][a];
        e2[a] = S.L[2][a] - S.L[0][a];
        e3[a] = S.L[3][a] - S.L[0][a];
    }
    i128 n3[3];
    cross_exact(e1, e2, n3);
    double D = wide_to_double(dot3_wide(n3, e3), 3 * CDP_Q);
    return D * (1.0 / 6.0) * 0.25 * (S.rho[0] + S.rho[1] + S.rho[2] + S.rho[3]);
}

CDP_HD double tri_mass_cells(const Tri& S) {
    i128 D = mul64(S.L[1][0] - S.L[0][0], S.L[2][1] - S.L[0][1]) -
             mul64(S.L[1][1] - S.L[0][1], S.L[2][0] - S.L[0][0]);
    return i128_to_real<double>(D, 2 * CDP_Q) * 0.5 * (S.rho[0] + S.rho[1] + S.rho[2]) * (1.0 / 3.0);
}

// absolute cell -> flat output index (C order, axis 0 slowest); -1 when outside a non-periodic grid
CDP_HD long long flat_cell(const GridDesc& g, int cx, int cy, int cz) {
    int c[3] = {cx, cy, cz};
    long long idx = 0;
    for (int a = 0; a < g.dim; ++a) {
        int v = c[a], n = g.n[a];
        if (g.periodic) {
            v %= n;
            if (v < 0) v += n;
        } else if (v < 0 || v >= n) {
            return -1;
        }
        idx = idx * n + v;
    }
    return idx;
}

}  // namespace cdp
