// Exact projection of one simplex (or of one tile of its bounding box) onto the grid cells, by
// enumerating the corners of every polyhedron (simplex intersect cell) and adding Franklin's
// (vertex, edge, facet) contributions (Sect. 3.1, eqs. firstOrder, contrib, E0, E1; Appendix C).
//
// For a corner at position P (relative to an origin O chosen per (simplex, cell) piece) and one
// incident (vertex, edge, facet) triple with unit vectors T (along the edge, leaving the corner),
// N (in the facet, normal to T, pointing into the facet) and B (normal to the facet, pointing into
// the polyhedron), the contribution in 3D is
//     C = E0 [rho(O) + E1 . grad rho],  E0 = -1/6 (P.T)(P.N)(P.B),
//     E1 = 1/4 ((P.T) T + 2 (P.N) N + 3 (P.B) B),
// and in 2D E0 = 1/2 (P.T)(P.N), E1 = 1/3 ((P.T) T + 2 (P.N) N).  With rho(O) = rho(X) - grad.P
// and T, N, B orthonormal the bracket becomes rho(X) - 3/4 (P.T)(T.g) - 1/2 (P.N)(N.g)
// - 1/4 (P.B)(B.g) in 3D and rho(X) - 2/3 (P.T)(T.g) - 1/3 (P.N)(N.g) in 2D, which is what is
// evaluated (rho(X) is the density at the corner itself, g = grad rho).
//
// The four corner types of Sect. 3.2 (Fig. cubeTetInter):
//   A  a grid node inside the simplex: 6 triples (2 in 2D) with axis-aligned T, N, B; the sum
//      over them is the closed form  sigma * prod_a P_a * (rho(X) - grad.P / 2), sigma = product
//      of the signs telling on which side of the cell the node is;
//   B  a simplex vertex: its 3 edges x 2 incident facets (2 triples in 2D);
//   C  a simplex edge crossing a cell face: 6 triples (2 in 2D) for each of the 2 cells;
//   D  a simplex facet crossing a cell edge (3D only): 6 triples for each of the 4 cells.
// Every edge direction and in-facet normal is oriented by an exact sign (vertex order, exact
// normal components, fixed parities of the vertex labels), never by a rounded dot product, and
// every facet normal is converted from its exact integer value component by component, so that
// nearly parallel planes do not lose the direction of their intersection line (Sect. 3.4: the
// triplets need care in nearly degenerate configurations).
//
// Origin of each piece (reading of Sect. 3.1, which extrapolates rho to "the origin of
// coordinates"): Franklin's sum over the corners of one closed polyhedron does not depend on the
// origin, so every (simplex, cell) piece uses its own origin O = the simplex centroid clamped
// into the cell.  Then |P| is bounded by both the cell diagonal and twice the simplex size,
// which keeps the FP32 evaluation accurate.
#pragma once

#include "cdp_exact.cuh"

namespace cdp {

template <typename R>
struct Eps;
template <>
struct Eps<float> {
    // semi-static filter bounds (multiples of the unit roundoff 2^-24, see setup)
    static constexpr float k2 = 3.814697265625e-06f;   // 2^-18
    static constexpr float k3 = 3.814697265625e-06f;   // 2^-18
};
template <>
struct Eps<double> {
    static constexpr double k2 = 7.105427357601002e-15;  // 2^-47
    static constexpr double k3 = 7.105427357601002e-15;  // 2^-47
};

template <typename R>
CDP_HD R rsqrt_r(R v);
template <>
CDP_HD float rsqrt_r<float>(float v) {
#ifdef __CUDA_ARCH__
    return rsqrtf(v);
#else
    return 1.0f / sqrtf(v);
#endif
}
template <>
CDP_HD double rsqrt_r<double>(double v) {
#ifdef __CUDA_ARCH__
    return rsqrt(v);
#else
    return 1.0 / sqrt(v);
#endif
}

// a / b where the quotient only seeds a guess that exact predicates then confirm or correct
template <typename R>
CDP_HD R div_guess(R a, R b) { return a / b; }
template <>
CDP_HD float div_guess<float>(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

// 1 / x for the FP32 contributions: the hardware reciprocal (relative error ~1e-7, far below the
// FP32-mixed tolerance); FP64 keeps the correctly rounded quotient
template <typename R>
CDP_HD R rcp_fast(R x) { return R(1) / x; }
template <>
CDP_HD float rcp_fast<float>(float x) {
#ifdef __CUDA_ARCH__
    return __fdividef(1.0f, x);
#else
    return 1.0f / x;
#endif
}

template <typename R>
CDP_HD R floor_r(R v);
template <>
CDP_HD float floor_r<float>(float v) { return floorf(v); }
template <>
CDP_HD double floor_r<double>(double v) { return floor(v); }

template <typename R>
CDP_HD R dot3(const R a[3], const R b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

template <typename R>
CDP_HD void cross3(const R a[3], const R b[3], R o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename R>
CDP_HD R clamp_r(R v, R lo, R hi) { return v < lo ? lo : (v > hi ? hi : v); }

// One 3D (vertex, edge, facet) triple; the caller multiplies the sum by -1/6.
template <typename R>
CDP_HD R trip3(const R P[3], const R T[3], const R N[3], const R B[3], R rhoX, const R g[3]) {
    R pt = dot3(P, T), pn = dot3(P, N), pb = dot3(P, B);
    R gt = dot3(g, T), gn = dot3(g, N), gb = dot3(g, B);
    return pt * pn * pb * (rhoX - R(0.75) * pt * gt - R(0.5) * pn * gn - R(0.25) * pb * gb);
}

// One 2D (vertex, edge) pair; the caller multiplies the sum by 1/2.
template <typename R>
CDP_HD R trip2(const R P[2], const R T[2], const R N[2], R rhoX, const R g[2]) {
    R pt = P[0] * T[0] + P[1] * T[1], pn = P[0] * N[0] + P[1] * N[1];
    R gt = g[0] * T[0] + g[1] * T[1], gn = g[0] * N[0] + g[1] * N[1];
    return pt * pn * (rhoX - R(2.0 / 3.0) * pt * gt - R(1.0 / 3.0) * pn * gn);
}

// Counters of one projection (all optional, gathered only when requested).
struct UnitCounts {
    unsigned long long a, b, c, d, exact;
};

// ==========================================================================================
// 3D
// ==========================================================================================

// A tetrahedron after canonicalisation: vertex coordinates in fixed point relative to the
// integer cell `anchor` (absolute cell index of the frame origin), positively oriented.
struct Tet {
    i64 L[4][3];
    double rho[4];
    int cell[4][3];  // cell of every vertex, relative to the anchor
    int lo[3], hi[3];
    int anchor[3];
};

// the vertices of the edge e (a < b) and the two others (p < q)
CDP_HD void tet_edge(int e, int& a, int& b, int& p, int& q) {
    // (0,1),(0,2),(0,3),(1,2),(1,3),(2,3); nibble e of each constant
    a = (0x211000 >> (4 * e)) & 15;
    b = (0x332321 >> (4 * e)) & 15;
    p = (0x000112 >> (4 * e)) & 15;
    q = (0x123233 >> (4 * e)) & 15;
}

// Bit e set when the permutation (a, b, p, q) of edge e (tet_edge order) is odd, computed at
// compile time from the same nibble tables.
constexpr unsigned tet_edge_odd_mask() {
    unsigned m = 0;
    for (int e = 0; e < 6; ++e) {
        const int v[4] = {(0x211000 >> (4 * e)) & 15, (0x332321 >> (4 * e)) & 15, (0x000112 >> (4 * e)) & 15,
                          (0x123233 >> (4 * e)) & 15};
        int inv = 0;
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j) inv += v[i] > v[j];
        if (inv & 1) m |= 1u << e;
    }
    return m;
}

// parity4(a, b, p, q) of edge e: +1 even, -1 odd
CDP_HD int tet_edge_parity(int e) { return ((tet_edge_odd_mask() >> e) & 1u) ? -1 : 1; }

CDP_HD constexpr int tet_edge_index(int i, int j) {
    int a = i < j ? i : j, b = i < j ? j : i;
    return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

// Register-friendly access to 3-vectors with a run-time index (a runtime-indexed local array
// would be placed in local memory).
template <typename T>
CDP_HD T pick3(T a0, T a1, T a2, int i) { return i == 0 ? a0 : (i == 1 ? a1 : a2); }

// Per-unit working set of a tetrahedron: coordinates relative to the unit's tile origin.
template <typename R>
struct TetGeo {
    i64 Lt[4][3];          // exact, relative to the tile origin
    R x[4][3];             // rounded copies (high part)
    R xl[4][3];            // low part: x + xl is the exact coordinate to twice the precision of R
    R n[4][3];             // unit inward normals of the facets (facet f is opposite vertex f)
    R g[3];                // grad rho (per cell length)
    R rho[4];
    R c[3], rhoc;          // centroid and density there
    R B2, B3;              // filter bounds for side2 / side3
    int cell[4][3];        // vertex cells relative to the tile origin
    int lo[3], hi[3];      // bounding box relative to the tile origin
    int anchor[3];         // absolute cell of the tile origin
    signed char ns[4][3];  // signs of the exact normal components
    int prob;              // the problem of the batch the tetrahedron belongs to
    double mexact;         // |V| mean(rho) in FP64 (closed form, for the mass closure)
    float mexact_hi;       // (float)mexact
    float mexact_lo;       // mexact - mexact_hi: mexact as an unevaluated sum of two floats
};

// exact inward normal of facet f (the facet opposite vertex f) of a positively oriented tetrahedron
CDP_COLD void facet_normal_exact(const i64 L[4][3], int f, i128 out[3]) {
    int o = f == 0 ? 1 : 0;  // reference vertex of the facet
    int u, v;                // the normal is (x_u - x_o) x (x_v - x_o)
    if (f == 0) { u = 3; v = 2; }
    else if (f == 1) { u = 2; v = 3; }
    else if (f == 2) { u = 3; v = 1; }
    else { u = 1; v = 2; }
    i64 d1[3], d2[3];
    for (int a = 0; a < 3; ++a) {
        d1[a] = L[u][a] - L[o][a];
        d2[a] = L[v][a] - L[o][a];
    }
    cross_exact(d1, d2, out);
}

template <typename R>
CDP_HD R low_part(i64 L, R hi);
template <>
CDP_HD float low_part<float>(i64 L, float hi) {
    i64 Lhi = (i64)llrintf(ldexpf(hi, CDP_Q));  // exact: hi has 24 bits and |hi| < 2^13
    return ldexpf((float)(L - Lhi), -CDP_Q);
}
template <>
CDP_HD double low_part<double>(i64, double) { return 0.0; }

// Rounded coordinates of the working set from its exact ones (Lt).
template <typename R>
CDP_HD void tet_round_coords(TetGeo<R>& G) {
    for (int k = 0; k < 4; ++k)
        for (int a = 0; a < 3; ++a) {
            G.x[k][a] = i64_to_real<R>(G.Lt[k][a], CDP_Q);
            G.xl[k][a] = low_part<R>(G.Lt[k][a], G.x[k][a]);
        }
}

// Fields of the working set that depend on the tile's frame besides the coordinates: the centroid
// and the filter bounds (from the largest coordinate magnitude in cells).
template <typename R>
CDP_HD void tet_frame_bounds(TetGeo<R>& G) {
    for (int a = 0; a < 3; ++a) G.c[a] = R(0.25) * (G.x[0][a] + G.x[1][a] + G.x[2][a] + G.x[3][a]);
    int m = 1;
    for (int a = 0; a < 3; ++a) {
        int v = G.lo[a] < 0 ? -G.lo[a] : G.lo[a];
        int w = G.hi[a] + 1 < 0 ? -(G.hi[a] + 1) : G.hi[a] + 1;
        m = v > m ? v : m;
        m = w > m ? w : m;
    }
    R Rm = R(m + 1);
    G.B2 = Eps<R>::k2 * Rm * Rm;
    G.B3 = Eps<R>::k3 * Rm;
}

// Fill the working set for the tile whose lowest cell is T (relative to the anchor).  COPY only
// gives a caller its own out-of-line instance (register allocation of its own).
template <typename R, int COPY = 0>
CDP_COLD void tet_setup(const Tet& S, const int T[3], TetGeo<R>& G) {
    for (int k = 0; k < 4; ++k)
        for (int a = 0; a < 3; ++a) {
            G.Lt[k][a] = S.L[k][a] - ((i64)T[a] << CDP_Q);
            G.cell[k][a] = S.cell[k][a] - T[a];
        }
    tet_round_coords(G);
    for (int a = 0; a < 3; ++a) {
        G.lo[a] = S.lo[a] - T[a];
        G.hi[a] = S.hi[a] - T[a];
    }
    i64 e3[3];
    for (int a = 0; a < 3; ++a) e3[a] = G.Lt[3][a] - G.Lt[0][a];
    R nr[4][3];
    i128 n3[3];
    for (int f = 0; f < 4; ++f) {
        i128 nE[3];
        facet_normal_exact(G.Lt, f, nE);
        for (int a = 0; a < 3; ++a) {
            nr[f][a] = i128_to_real<R>(nE[a], 2 * CDP_Q);
            G.ns[f][a] = (signed char)sgn_i128(nE[a]);
            if (f == 3) n3[a] = nE[a];
        }
        R inv = rsqrt_r<R>(dot3(nr[f], nr[f]));
        for (int a = 0; a < 3; ++a) G.n[f][a] = nr[f][a] * inv;
    }
    // 6 |V| = e3 . (e1 x e2), exact, then rounded
    double D = wide_to_double(dot3_wide(n3, e3), 3 * CDP_Q);
    R invD = R(1) / R(D);
    G.mexact = D * (1.0 / 6.0) * 0.25 * (S.rho[0] + S.rho[1] + S.rho[2] + S.rho[3]);
    G.mexact_hi = (float)G.mexact;
    G.mexact_lo = (float)(G.mexact - (double)G.mexact_hi);
    for (int a = 0; a < 3; ++a) G.anchor[a] = S.anchor[a] + T[a];
    for (int k = 0; k < 4; ++k) G.rho[k] = (R)S.rho[k];
    R d1 = G.rho[1] - G.rho[0], d2 = G.rho[2] - G.rho[0], d3 = G.rho[3] - G.rho[0];
    for (int a = 0; a < 3; ++a) G.g[a] = (d1 * nr[1][a] + d2 * nr[2][a] + d3 * nr[3][a]) * invD;
    G.rhoc = R(0.25) * (G.rho[0] + G.rho[1] + G.rho[2] + G.rho[3]);
    tet_frame_bounds(G);
}

// ------------------------------------------------------------------------------------------
// exact stages of the two predicates (Sect. 3.3, with SoS): the orient2d of a grid point against
// a projected edge (side2) and the orient3d of a grid node against a facet (side3).  The kernels
// evaluate a floating-point filter (bounds B2, B3 of the working set) and take these only when it
// is inconclusive (out of line: rarely reached, and kept out of the hot loops' instruction
// footprint).
// ------------------------------------------------------------------------------------------

template <typename R>
CDP_COLD int tet_side2_exact(const TetGeo<R>& G, int i, int j, int u, int v, int pu, int pv) {
    return side2_exact(G.Lt[i][u], G.Lt[i][v], G.Lt[j][u], G.Lt[j][v], (i64)pu << CDP_Q, (i64)pv << CDP_Q);
}

template <typename R>
CDP_COLD int tet_side3_exact(const TetGeo<R>& G, int f, int g0, int g1, int g2) {
    int a = f == 0 ? 1 : 0;
    i64 gp[3] = {(i64)g0 << CDP_Q, (i64)g1 << CDP_Q, (i64)g2 << CDP_Q};
    i128 nE[3];
    facet_normal_exact(G.Lt, f, nE);
    return side3_exact(nE, G.Lt[a], gp);
}

// ------------------------------------------------------------------------------------------
// contributions of one (corner, cell) incidence; P = corner - O with O the piece's origin
// ------------------------------------------------------------------------------------------

// origin of the piece in cell (v0, v1, v2): the centroid clamped into the central half of the
// cell, so that |P| stays below both twice the simplex size plus half a cell and 3/4 of a cell
// per axis (small simplices keep a nearby origin, large ones get one near the cell centre)
template <typename R>
CDP_HD void piece_origin(const TetGeo<R>& G, int v0, int v1, int v2, R O[3]) {
    O[0] = clamp_r(G.c[0], R(v0) + R(0.25), R(v0) + R(0.75));
    O[1] = clamp_r(G.c[1], R(v1) + R(0.25), R(v1) + R(0.75));
    O[2] = clamp_r(G.c[2], R(v2) + R(0.25), R(v2) + R(0.75));
}

// The per-simplex values that every (corner, cell) evaluation reads (centroid, density there and
// gradient), copied to registers once before a loop over cells.
template <typename R>
struct TetFrame {
    R c[3], rhoc, g[3];
};

template <typename R>
CDP_HD TetFrame<R> tet_frame(const TetGeo<R>& G) {
    TetFrame<R> F;
    for (int a = 0; a < 3; ++a) {
        F.c[a] = G.c[a];
        F.g[a] = G.g[a];
    }
    F.rhoc = G.rhoc;
    return F;
}

template <typename R>
CDP_HD void piece_origin(const TetFrame<R>& F, int v0, int v1, int v2, R O[3]) {
    O[0] = clamp_r(F.c[0], R(v0) + R(0.25), R(v0) + R(0.75));
    O[1] = clamp_r(F.c[1], R(v1) + R(0.25), R(v1) + R(0.75));
    O[2] = clamp_r(F.c[2], R(v2) + R(0.25), R(v2) + R(0.75));
}

// B: simplex vertex i; P = x_i - O
template <typename R>
CDP_COLD R tet_corner_B(const TetGeo<R>& G, int i, const R P[3]) {
    R s = 0;
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        if (j == i) continue;
        int a = i < j ? i : j, b = i < j ? j : i;
        R ev[3];
        for (int t = 0; t < 3; ++t) ev[t] = (G.x[b][t] - G.x[a][t]) + (G.xl[b][t] - G.xl[a][t]);
        R inv = rsqrt_r<R>(dot3(ev, ev));
        for (int t = 0; t < 3; ++t) ev[t] *= inv;
        R sg = i == a ? R(1) : R(-1);
        R T[3] = {sg * ev[0], sg * ev[1], sg * ev[2]};
        for (int f = 0; f < 4; ++f) {
            if (f == i || f == j) continue;
            int r = 6 - i - j - f;  // third vertex of facet f
            const R nf[3] = {G.n[f][0], G.n[f][1], G.n[f][2]};
            R N[3];
            cross3(nf, ev, N);
            R ps = R(parity4(a, b, r, f));
            for (int t = 0; t < 3; ++t) N[t] *= ps;
            s += trip3(P, T, N, nf, G.rho[i], G.g);
        }
    }
    return R(-1.0 / 6.0) * s;
}

// A: grid node inside the simplex; cell on side s (sgn = product of s_a, s_a = +1 when the node is
// the cell's upper corner along a)
template <typename R>
CDP_HD R tet_corner_A(const TetGeo<R>& G, const R P[3], R rhoX, R sgn) {
    return sgn * P[0] * P[1] * P[2] * (rhoX - R(0.5) * dot3(G.g, P));
}

// density at the corner whose offset from the origin O of its piece is P
template <typename R>
CDP_HD R rho_from_P(const TetGeo<R>& G, const R P[3], const R O[3]) {
    return G.rhoc + G.g[0] * (P[0] + (O[0] - G.c[0])) + G.g[1] * (P[1] + (O[1] - G.c[1])) +
           G.g[2] * (P[2] + (O[2] - G.c[2]));
}

template <typename R>
CDP_HD R rho_from_P(const TetFrame<R>& F, const R P[3], const R O[3]) {
    return F.rhoc + F.g[0] * (P[0] + (O[0] - F.c[0])) + F.g[1] * (P[1] + (O[1] - F.c[1])) +
           F.g[2] * (P[2] + (O[2] - F.c[2]));
}

template <typename R>
CDP_HD R tet_corner_A(const TetFrame<R>& F, const R P[3], R rhoX, R sgn) {
    return sgn * P[0] * P[1] * P[2] * (rhoX - R(0.5) * dot3(F.g, P));
}

// Facets pierced by a grid line, from the signs of the 6 projected edges against the line point
// (bit e of sgn set when positive, tet_edge order): bit f set when the projection of facet f
// contains the point, i.e. its three edges, oriented around it, have one sign.
CDP_HD constexpr unsigned tet_pierced(unsigned sgn) {
    unsigned hits = 0;
    for (int f = 0; f < 4; ++f) {
        int a = f == 0 ? 1 : 0, b = f <= 1 ? 2 : 1, cc = f == 3 ? 2 : 3;
        unsigned sab = (sgn >> tet_edge_index(a, b)) & 1u, sbc = (sgn >> tet_edge_index(b, cc)) & 1u,
                 sac = (sgn >> tet_edge_index(a, cc)) & 1u;
        // orient(a,b), orient(b,c), orient(c,a) = -orient(a,c) all of one sign
        if (sab == sbc && sbc != sac) hits |= 1u << f;
    }
    return hits;
}

// ------------------------------------------------------------------------------------------
// Closed forms of the C and D corners for all the cells around the corner at once.  The six
// (vertex, edge, facet) triples of such a corner are built from the unit normal(s) of the
// simplex facet(s) and the cell faces; expanding them gives short polynomials in P (the corner
// relative to its piece's origin) whose coefficients depend only on the corner, so they are
// computed once for the 4 (D) or 2 (C) cells.
// ------------------------------------------------------------------------------------------

// (a x b) component i
template <typename R>
CDP_HD R cross_comp(const R a[3], const R b[3], int i) {
    R c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
    return pick3(c0, c1, c2, i);
}

// Facet-face triples: a simplex facet (unit normal n) meets the cell face normal to axis a along a
// line, oriented by su, on the side sigma of the cell.  With Pn = P.n, gn = g.n, h = (g x n)_a,
// ir2 = 1 / (1 - n_a^2), c = (P x n)_a, d3 = P_a - n_a Pn, d4 = Pn - n_a P_a, e3 = g_a - n_a gn,
// e4 = gn - n_a g_a and b = rho(X) - (3/4) c h ir2, its two triples sum (times -6) to
//   su sigma c ir2 [d3 Pn (b - d3 e3 ir2 / 2 - Pn gn / 4) + d4 P_a (b - d4 e4 ir2 / 2 - P_a g_a / 4)].
// tet_eval_D4 and tet_eval_C2 write this out with the factors their cells share taken out.

// D corner (facet f pierced by the grid line along l at (dj, dk), in cell column m): the values
// of the 4 cells (oj, ok) = (0,0), (0,1), (1,0), (1,1), passed to acc(cell, value).  The cells
// share the slab m along l and, pairwise, their columns along j and k, so their piece origins (and
// the corner's offsets P from them) take 1 + 2 + 2 values; the density at the corner is the same for
// all four.
template <typename R, class Acc>
CDP_HD void tet_eval_D4(const TetGeo<R>& G, int f, int l, int dj, int dk, int m, Acc& acc) {
    int j = l == 0 ? 1 : 0, k = l == 2 ? 1 : 2;
    int va = f == 0 ? 1 : 0;
    const R n[3] = {G.n[f][0], G.n[f][1], G.n[f][2]};
    R nj = pick3(n[0], n[1], n[2], j), nk = pick3(n[0], n[1], n[2], k), nl = pick3(n[0], n[1], n[2], l);
    R tau = G.ns[f][l] > 0 ? R(1) : R(-1);
    R eps = (l == 1) ? R(-1) : R(1);
    R off = -(nj * ((R(dj) - G.x[va][j]) - G.xl[va][j]) + nk * ((R(dk) - G.x[va][k]) - G.xl[va][k])) * rcp_fast(nl);
    const R g[3] = {G.g[0], G.g[1], G.g[2]};
    R gn = dot3(g, n);
    R hj = cross_comp(g, n, j), hk = cross_comp(g, n, k);
    R irj2 = rcp_fast(nk * nk + nl * nl), irk2 = rcp_fast(nj * nj + nl * nl);
    R gj = pick3(g[0], g[1], g[2], j), gk = pick3(g[0], g[1], g[2], k), gl = pick3(g[0], g[1], g[2], l);
    const TetFrame<R> F = tet_frame(G);
    const R cl = pick3(F.c[0], F.c[1], F.c[2], l), cj = pick3(F.c[0], F.c[1], F.c[2], j),
            ck = pick3(F.c[0], F.c[1], F.c[2], k);
    // piece origins (the centroid clamped into the central half of each cell) and offsets of the
    // corner from them, along l (shared) and along j, k (two values each)
    const R Ol = clamp_r(cl, R(m) + R(0.25), R(m) + R(0.75));
    const R Pl = (G.x[va][l] - Ol) + (G.xl[va][l] + off);
    const R Oj0 = clamp_r(cj, R(dj - 1) + R(0.25), R(dj - 1) + R(0.75)), Oj1 = clamp_r(cj, R(dj) + R(0.25), R(dj) + R(0.75));
    const R Ok0 = clamp_r(ck, R(dk - 1) + R(0.25), R(dk - 1) + R(0.75)), Ok1 = clamp_r(ck, R(dk) + R(0.25), R(dk) + R(0.75));
    const R Pj0 = R(dj) - Oj0, Pj1 = R(dj) - Oj1, Pk0 = R(dk) - Ok0, Pk1 = R(dk) - Ok1;
    // the density at the corner
    const R rhoX = F.rhoc + gl * (Pl + (Ol - cl)) + gj * (Pj0 + (Oj0 - cj)) + gk * (Pk0 + (Ok0 - ck));
    const R PnL = Pl * nl;
    // the facet-face triples of the two cell faces through the line (normal to j and to k): their
    // per-record factors, and the cross-product components
    // (P x n)_j = eps (Pk nl - Pl nk), (P x n)_k = eps (Pl nj - Pj nl), whose sign eps cancels
    // against the orientation of the facet/face lines
    const R Lj = R(0.75) * eps * hj * irj2, Lk = R(0.75) * eps * hk * irk2;
    const R hj3 = R(0.5) * (gj - nj * gn) * irj2, hj4 = R(0.5) * (gn - nj * gj) * irj2;
    const R hk3 = R(0.5) * (gk - nk * gn) * irk2, hk4 = R(0.5) * (gn - nk * gk) * irk2;
    const R qgn = R(0.25) * gn, qgj = R(0.25) * gj, qgk = R(0.25) * gk;
    const R T0 = R(2) * rhoX - R(1.5) * Pl * gl;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        const int oj = q >> 1, ok = q & 1;
        const int vj = dj - 1 + oj, vk = dk - 1 + ok;
        const int v0 = l == 0 ? m : vj;
        const int v1 = l == 1 ? m : (l == 0 ? vj : vk);
        const int v2 = l == 2 ? m : vk;
        const R Pj = oj ? Pj1 : Pj0, Pk = ok ? Pk1 : Pk0;
        const R Pn = PnL + Pj * nj + Pk * nk;
        // the facet with the two faces' line
        const R s12 = Pj * Pk * Pl * (T0 - R(0.75) * (Pj * gj + Pk * gk));
        // facet / face normal to j
        const R Cj = Pk * nl - Pl * nk;
        const R d3j = Pj - nj * Pn, d4j = Pn - nj * Pj, b0j = rhoX - Lj * Cj;
        const R Fj = d3j * Pn * (b0j - d3j * hj3 - Pn * qgn) + d4j * Pj * (b0j - d4j * hj4 - Pj * qgj);
        // facet / face normal to k
        const R Ck = Pl * nj - Pj * nl;
        const R d3k = Pk - nk * Pn, d4k = Pn - nk * Pk, b0k = rhoX - Lk * Ck;
        const R Fk = d3k * Pn * (b0k - d3k * hk3 - Pn * qgn) + d4k * Pk * (b0k - d4k * hk4 - Pk * qgk);
        const R sgn = (oj == ok ? tau : -tau) * R(-1.0 / 6.0);
        acc(v0, v1, v2, sgn * (s12 + Cj * irj2 * Fj - Ck * irk2 * Fk));
    }
}

// C corner (edge e crossing the plane x_k = c): the values of the 2 cells (below, above), passed to
// acc(cell, value)
template <typename R, class Acc>
CDP_HD void tet_eval_C2(const TetGeo<R>& G, int e, int k, int c, int cj1, int cj2, Acc& acc) {
    int a, b, p, q;
    tet_edge(e, a, b, p, q);
    int dirk = G.cell[b][k] > G.cell[a][k] ? 1 : -1;
    int j1 = k == 0 ? 1 : 0;
    R ev[3];
    for (int w = 0; w < 3; ++w) ev[w] = (G.x[b][w] - G.x[a][w]) + (G.xl[b][w] - G.xl[a][w]);
    R evk = pick3(ev[0], ev[1], ev[2], k);
    R t = ((R(c) - G.x[a][k]) - G.xl[a][k]) * rcp_fast(evk);
    R rhoX = G.rho[a] + t * (G.rho[b] - G.rho[a]);
    R inv = rsqrt_r<R>(dot3(ev, ev));
    const R eu[3] = {ev[0] * inv, ev[1] * inv, ev[2] * inv};
    const R g[3] = {G.g[0], G.g[1], G.g[2]};
    const R np_[3] = {G.n[p][0], G.n[p][1], G.n[p][2]};
    const R nq_[3] = {G.n[q][0], G.n[q][1], G.n[q][2]};
    // in-facet normals of the edge: m_p in facet p (towards q), m_q in facet q (towards p); the
    // orientations are the parities of (a, b, q, p) = -(a, b, p, q) and of (a, b, p, q)
    const R pq = R(tet_edge_parity(e)), pp = -pq;
    R mp[3], mq[3];
    cross3(np_, eu, mp);
    cross3(nq_, eu, mq);
    for (int w = 0; w < 3; ++w) {
        mp[w] *= pp;
        mq[w] *= pq;
    }
    R ge = dot3(g, eu), gmp = dot3(g, mp), gmq = dot3(g, mq), gnp = dot3(g, np_), gnq = dot3(g, nq_);
    R hp = cross_comp(g, np_, k), hq = cross_comp(g, nq_, k);
    // 1 / (1 - n_k^2) from the other two components (no cancellation when n_k is near 1)
    R a0 = pick3(np_[1], np_[0], np_[0], k), a1 = pick3(np_[2], np_[2], np_[1], k);
    R b0 = pick3(nq_[1], nq_[0], nq_[0], k), b1 = pick3(nq_[2], nq_[2], nq_[1], k);
    R irp2 = rcp_fast(a0 * a0 + a1 * a1), irq2 = rcp_fast(b0 * b0 + b1 * b1);
    R lam = -pq * R(dirk);
    // the crossing point as vertex a (high part) plus a small offset
    const R xa[3] = {G.x[a][0], G.x[a][1], G.x[a][2]};
    const R dx[3] = {G.xl[a][0] + t * ev[0], G.xl[a][1] + t * ev[1], G.xl[a][2] + t * ev[2]};
    const TetFrame<R> F = tet_frame(G);
    // the two cells differ only along k: the piece origins share their other components, and so do
    // the corner's offsets P from them; the dot products with P share those terms
    R P[3];
    {
        const int vv0 = j1 == 0 ? cj1 : cj2, vv1 = j1 == 1 ? cj1 : cj2, vv2 = j1 == 2 ? cj1 : cj2;
        R O[3];
        piece_origin(F, vv0, vv1, vv2, O);  // (its k component is replaced below)
        for (int w = 0; w < 3; ++w) P[w] = (xa[w] - O[w]) + dx[w];
    }
    P[0] = k == 0 ? R(0) : P[0];
    P[1] = k == 1 ? R(0) : P[1];
    P[2] = k == 2 ? R(0) : P[2];
    const R ek = pick3(eu[0], eu[1], eu[2], k), mpk = pick3(mp[0], mp[1], mp[2], k),
            mqk = pick3(mq[0], mq[1], mq[2], k), npk = pick3(np_[0], np_[1], np_[2], k),
            nqk = pick3(nq_[0], nq_[1], nq_[2], k);
    const R Pe0 = dot3(P, eu), Pmp0 = dot3(P, mp), Pmq0 = dot3(P, mq), Pnp0 = dot3(P, np_), Pnq0 = dot3(P, nq_);
    const R ckc = pick3(F.c[0], F.c[1], F.c[2], k);
    // the facet-face triples of the two facets with the face normal to k: (P x n)_k has no P_k in
    // it, so it and the bracket's lead b are the same for both cells
    const R gkk = pick3(g[0], g[1], g[2], k), qgk = R(0.25) * gkk;
    const R cpp = cross_comp(P, np_, k), cpq = cross_comp(P, nq_, k);
    const R bp = rhoX - R(0.75) * cpp * hp * irp2, bq = rhoX - R(0.75) * cpq * hq * irq2;
    const R hp3 = R(0.5) * (gkk - npk * gnp) * irp2, hp4 = R(0.5) * (gnp - npk * gkk) * irp2;
    const R hq3 = R(0.5) * (gkk - nqk * gnq) * irq2, hq4 = R(0.5) * (gnq - nqk * gkk) * irq2;
    const R qgnp = R(0.25) * gnp, qgnq = R(0.25) * gnq;
    const R Wp = lam * cpp * irp2, Wq = -lam * cpq * irq2;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        int vk = side ? c : c - 1;
        int v0 = k == 0 ? vk : (j1 == 0 ? cj1 : cj2);
        int v1 = k == 1 ? vk : (j1 == 1 ? cj1 : cj2);
        int v2 = k == 2 ? vk : (j1 == 2 ? cj1 : cj2);
        const R Pk = R(c) - clamp_r(ckc, R(vk) + R(0.25), R(vk) + R(0.75));
        R sigma = side ? R(1) : R(-1);
        R so = sigma * R(dirk);
        R Pe = Pe0 + Pk * ek, Pmp = Pmp0 + Pk * mpk, Pmq = Pmq0 + Pk * mqk, Pnp = Pnp0 + Pk * npk,
          Pnq = Pnq0 + Pk * nqk;
        // the simplex edge with its two facets
        R s12 = so * Pe *
                (Pmp * Pnp * (rhoX - R(0.75) * Pe * ge - R(0.5) * Pmp * gmp - R(0.25) * Pnp * gnp) +
                 Pmq * Pnq * (rhoX - R(0.75) * Pe * ge - R(0.5) * Pmq * gmq - R(0.25) * Pnq * gnq));
        const R d3p = Pk - npk * Pnp, d4p = Pnp - npk * Pk, d3q = Pk - nqk * Pnq, d4q = Pnq - nqk * Pk;
        const R s34 = sigma * Wp * (d3p * Pnp * (bp - d3p * hp3 - Pnp * qgnp) + d4p * Pk * (bp - d4p * hp4 - Pk * qgk));
        const R s56 = sigma * Wq * (d3q * Pnq * (bq - d3q * hq3 - Pnq * qgnq) + d4q * Pk * (bq - d4q * hq4 - Pk * qgk));
        acc(v0, v1, v2, R(-1.0 / 6.0) * (s12 + s34 + s56));
    }
}

// ------------------------------------------------------------------------------------------
// Split form for a work queue: the locate step of a crossing / a line yields compact records of
// corners, and the evaluate step (tet_eval_C2 / tet_eval_D4) turns one record into the
// contributions of all the cells around it, so that the (costly) evaluations of a warp can run in
// full batches of identical work.  The records assume the tile is the whole bounding box (every
// cell around an interior crossing or line lies in it).
//   C record: bits 0-10 c, 11-21 cj1, 22-32 cj2, 34-35 k, 36-38 e
//   D record: bits 0-10 m, 11-21 dj, 22-32 dk, 35-36 l, 37-38 f
// (coordinates in the tile frame, 0 <= value < 2048).  Bits 40 and up are left to the caller.
// ------------------------------------------------------------------------------------------
typedef unsigned long long Rec;

CDP_HD void decode_C(Rec r, int& e, int& k, int& c, int& cj1, int& cj2) {
    c = (int)(r & 2047);
    cj1 = (int)((r >> 11) & 2047);
    cj2 = (int)((r >> 22) & 2047);
    k = (int)((r >> 34) & 3);
    e = (int)((r >> 36) & 7);
}

CDP_HD void decode_D(Rec r, int& f, int& l, int& dj, int& dk, int& m) {
    m = (int)(r & 2047);
    dj = (int)((r >> 11) & 2047);
    dk = (int)((r >> 22) & 2047);
    l = (int)((r >> 35) & 3);
    f = (int)((r >> 37) & 3);
}

// ==========================================================================================
// 2D
// ==========================================================================================

struct Tri {
    i64 L[3][2];
    double rho[3];
    int cell[3][2];
    int lo[2], hi[2];
    int anchor[2];
};

template <typename R>
struct TriGeo {
    i64 Lt[3][2];
    R x[3][2];
    R xl[3][2];   // low parts (x + xl exact to twice the precision of R)
    R n[3][2];    // unit inward normal of the edge opposite vertex k
    i64 nE[3][2]; // exact normals
    R g[2];
    R rho[3];
    R c[2], rhoc;
    R B2;
    int cell[3][2];
    int lo[2], hi[2];
    int anchor[3];  // absolute cell of the tile origin (third entry 0)
    int prob;       // the problem of the batch the triangle belongs to
    double mexact;  // |V| mean(rho) in FP64
};

template <typename R>
CDP_COLD void tri_setup(const Tri& S, const int T[2], TriGeo<R>& G) {
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a) {
            G.Lt[k][a] = S.L[k][a] - ((i64)T[a] << CDP_Q);
            G.x[k][a] = i64_to_real<R>(G.Lt[k][a], CDP_Q);
            G.xl[k][a] = low_part<R>(G.Lt[k][a], G.x[k][a]);
            G.cell[k][a] = S.cell[k][a] - T[a];
        }
    for (int a = 0; a < 2; ++a) {
        G.lo[a] = S.lo[a] - T[a];
        G.hi[a] = S.hi[a] - T[a];
    }
    // n_k = perp(x_{k+2} - x_{k+1}), perp(v) = (-v_y, v_x), for a positively oriented triangle
    for (int k = 0; k < 3; ++k) {
        int i1 = (k + 1) % 3, i2 = (k + 2) % 3;
        i64 dx = G.Lt[i2][0] - G.Lt[i1][0], dy = G.Lt[i2][1] - G.Lt[i1][1];
        G.nE[k][0] = -dy;
        G.nE[k][1] = dx;
        R nx = i64_to_real<R>(-dy, CDP_Q), ny = i64_to_real<R>(dx, CDP_Q);
        R inv = rsqrt_r<R>(nx * nx + ny * ny);
        G.n[k][0] = nx * inv;
        G.n[k][1] = ny * inv;
    }
    i64 e1x = G.Lt[1][0] - G.Lt[0][0], e1y = G.Lt[1][1] - G.Lt[0][1];
    i64 e2x = G.Lt[2][0] - G.Lt[0][0], e2y = G.Lt[2][1] - G.Lt[0][1];
    i128 Dq = mul64(e1x, e2y) - mul64(e1y, e2x);
    double D = i128_to_real<double>(Dq, 2 * CDP_Q);
    G.mexact = D * 0.5 * (S.rho[0] + S.rho[1] + S.rho[2]) * (1.0 / 3.0);
    G.anchor[0] = S.anchor[0] + T[0];
    G.anchor[1] = S.anchor[1] + T[1];
    G.anchor[2] = 0;
    for (int k = 0; k < 3; ++k) G.rho[k] = (R)S.rho[k];
    R d1 = G.rho[1] - G.rho[0], d2 = G.rho[2] - G.rho[0];
    R ex1 = i64_to_real<R>(e1x, CDP_Q), ey1 = i64_to_real<R>(e1y, CDP_Q);
    R ex2 = i64_to_real<R>(e2x, CDP_Q), ey2 = i64_to_real<R>(e2y, CDP_Q);
    R invD = R(1) / R(D);
    G.g[0] = (d1 * ey2 - d2 * ey1) * invD;
    G.g[1] = (d2 * ex1 - d1 * ex2) * invD;
    for (int a = 0; a < 2; ++a) G.c[a] = (G.x[0][a] + G.x[1][a] + G.x[2][a]) * R(1.0 / 3.0);
    G.rhoc = (G.rho[0] + G.rho[1] + G.rho[2]) * R(1.0 / 3.0);
    int m = 1;
    for (int a = 0; a < 2; ++a) {
        int v = G.lo[a] < 0 ? -G.lo[a] : G.lo[a];
        int w = G.hi[a] + 1 < 0 ? -(G.hi[a] + 1) : G.hi[a] + 1;
        m = v > m ? v : m;
        m = w > m ? w : m;
    }
    R Rm = R(m + 1);
    G.B2 = Eps<R>::k2 * Rm * Rm;
}

template <typename R>
CDP_HD int tri_side2(const TriGeo<R>& G, int i, int j, int pu, int pv, UnitCounts* cnt) {
    R du = G.x[j][0] - G.x[i][0], dv = G.x[j][1] - G.x[i][1];
    R val = du * (R(pv) - G.x[i][1]) - dv * (R(pu) - G.x[i][0]);
    if (val > G.B2) return 1;
    if (val < -G.B2) return -1;
    if (cnt) cnt->exact++;
    return side2_exact(G.Lt[i][0], G.Lt[i][1], G.Lt[j][0], G.Lt[j][1], (i64)pu << CDP_Q, (i64)pv << CDP_Q);
}

// sign(X_j - d) for the crossing of edge (a -> b) with the line x_k = c (j = 1 - k)
template <typename R>
CDP_HD int tri_cross_side(const TriGeo<R>& G, int a, int b, int k, int c, int d, int dirk, UnitCounts* cnt) {
    // j < k: orient2d(a, b, (d, c)); j > k: -orient2d(a, b, (c, d)) in (x, y) order
    int s = k == 1 ? tri_side2(G, a, b, d, c, cnt) : -tri_side2(G, a, b, c, d, cnt);
    return dirk * s;
}

template <typename R>
CDP_HD int tri_cross_cell(const TriGeo<R>& G, int a, int b, int k, int c, int guess, int dirk, UnitCounts* cnt) {
    int j = 1 - k;
    int lo = G.cell[a][j] < G.cell[b][j] ? G.cell[a][j] : G.cell[b][j];
    int hi = G.cell[a][j] < G.cell[b][j] ? G.cell[b][j] : G.cell[a][j];
    int d = guess < lo ? lo : (guess > hi ? hi : guess);
    for (int it = 0; it <= hi - lo + 1; ++it) {
        if (d > lo && tri_cross_side(G, a, b, k, c, d, dirk, cnt) < 0) {
            --d;
            continue;
        }
        if (d < hi && tri_cross_side(G, a, b, k, c, d + 1, dirk, cnt) > 0) {
            ++d;
            continue;
        }
        break;
    }
    return d;
}

template <typename R>
CDP_HD void tri_origin(const TriGeo<R>& G, int v0, int v1, R O[2]) {
    O[0] = clamp_r(G.c[0], R(v0) + R(0.25), R(v0) + R(0.75));
    O[1] = clamp_r(G.c[1], R(v1) + R(0.25), R(v1) + R(0.75));
}

// B: vertex i; P = x_i - O
template <typename R>
CDP_COLD R tri_corner_B(const TriGeo<R>& G, int i, const R P[2]) {
    R s = 0;
    for (int j = 0; j < 3; ++j) {
        if (j == i) continue;
        int k = 3 - i - j;  // edge (i, j) is opposite vertex k
        R T[2] = {(G.x[j][0] - G.x[i][0]) + (G.xl[j][0] - G.xl[i][0]),
                  (G.x[j][1] - G.x[i][1]) + (G.xl[j][1] - G.xl[i][1])};
        R inv = rsqrt_r<R>(T[0] * T[0] + T[1] * T[1]);
        T[0] *= inv;
        T[1] *= inv;
        const R N[2] = {G.n[k][0], G.n[k][1]};
        s += trip2(P, T, N, G.rho[i], G.g);
    }
    return R(0.5) * s;
}

// C: edge (a, b) (opposite o) crossing the grid line x_k = c; cell on side sigma; eu = unit (a -> b)
template <typename R>
CDP_HD R tri_corner_C(const TriGeo<R>& G, int o, int k, int dirk, R sigma, const R eu[2], const R P[2], R rhoX) {
    R so = sigma * R(dirk);
    const R T[2] = {so * eu[0], so * eu[1]};
    const R N[2] = {G.n[o][0], G.n[o][1]};
    R s = trip2(P, T, N, rhoX, G.g);
    // along the grid line (axis j = 1 - k), into the triangle; inward normal of the cell side
    R tj = (k == 1 ? G.nE[o][0] : G.nE[o][1]) > 0 ? R(1) : R(-1);
    const R T2[2] = {k == 1 ? tj : R(0), k == 0 ? tj : R(0)};
    const R N2[2] = {k == 0 ? sigma : R(0), k == 1 ? sigma : R(0)};
    s += trip2(P, T2, N2, rhoX, G.g);
    return R(0.5) * s;
}

template <typename R, class Acc>
CDP_HD void tri_item_vertex(const TriGeo<R>& G, int i, const int td[2], Acc& acc, UnitCounts* cnt) {
    const int v0 = G.cell[i][0], v1 = G.cell[i][1];
    if (v0 >= 0 && v0 < td[0] && v1 >= 0 && v1 < td[1]) {
        R O[2];
        tri_origin(G, v0, v1, O);
        const R P[2] = {(G.x[i][0] - O[0]) + G.xl[i][0], (G.x[i][1] - O[1]) + G.xl[i][1]};
        acc(v0, v1, 0, tri_corner_B(G, i, P));
        if (cnt) cnt->b++;
    }
}

// edge opposite vertex o as (a < b)
CDP_HD void tri_edge(int o, int& a, int& b) {
    a = o == 0 ? 1 : 0;
    b = o == 2 ? 1 : 2;
}

template <typename R>
CDP_HD int tri_crossings(const TriGeo<R>& G, int o, int k, const int td[2], int& c0) {
    int a, b;
    tri_edge(o, a, b);
    int ca = G.cell[a][k], cb = G.cell[b][k];
    c0 = (ca < cb ? ca : cb) + 1;
    int c1 = ca < cb ? cb : ca;
    if (c0 < 0) c0 = 0;
    int tk = k == 0 ? td[0] : td[1];
    if (c1 > tk) c1 = tk;
    return c1 >= c0 ? c1 - c0 + 1 : 0;
}

template <typename R, class Acc>
CDP_HD void tri_item_crossing(const TriGeo<R>& G, int o, int k, int c, const int td[2], Acc& acc, UnitCounts* cnt) {
    int a, b;
    tri_edge(o, a, b);
    int j = 1 - k;
    int dirk = G.cell[b][k] > G.cell[a][k] ? 1 : -1;
    R ev[2] = {(G.x[b][0] - G.x[a][0]) + (G.xl[b][0] - G.xl[a][0]),
               (G.x[b][1] - G.x[a][1]) + (G.xl[b][1] - G.xl[a][1])};
    R evk = k == 0 ? ev[0] : ev[1], evj = k == 0 ? ev[1] : ev[0];
    R t = ((R(c) - G.x[a][k]) - G.xl[a][k]) / evk;
    R dj = t * evj;
    R Xj = G.x[a][j] + dj;
    int cj = tri_cross_cell(G, a, b, k, c, (int)floor_r(Xj), dirk, cnt);
    int tj = j == 0 ? td[0] : td[1], tk = k == 0 ? td[0] : td[1];
    if (cj < 0 || cj >= tj) return;
    R rhoX = G.rho[a] + t * (G.rho[b] - G.rho[a]);
    R inv = rsqrt_r<R>(ev[0] * ev[0] + ev[1] * ev[1]);
    const R eu[2] = {ev[0] * inv, ev[1] * inv};
    for (int side = 0; side < 2; ++side) {
        int vk = side == 0 ? c - 1 : c;
        if (vk < 0 || vk >= tk) continue;
        int v0 = k == 0 ? vk : cj, v1 = k == 1 ? vk : cj;
        R O[2];
        tri_origin(G, v0, v1, O);
        R Pk = R(c) - (k == 0 ? O[0] : O[1]);
        R Pj = (G.x[a][j] - (j == 0 ? O[0] : O[1])) + (G.xl[a][j] + dj);
        const R P[2] = {k == 0 ? Pk : Pj, k == 1 ? Pk : Pj};
        acc(v0, v1, 0, tri_corner_C(G, o, k, dirk, side == 0 ? R(-1) : R(1), eu, P, rhoX));
        if (cnt) cnt->c++;
    }
}

// rows of grid nodes along x inside the tile: y = dy0 .. dy0 + n - 1
template <typename R>
CDP_HD int tri_rows(const TriGeo<R>& G, const int td[2], int& dy0) {
    dy0 = G.lo[1] + 1 > 0 ? G.lo[1] + 1 : 0;
    int dy1 = G.hi[1] < td[1] ? G.hi[1] : td[1];
    return dy1 >= dy0 ? dy1 - dy0 + 1 : 0;
}

// A: the grid nodes of row y = dy inside the triangle (between the two crossing edges)
template <typename R, class Acc>
CDP_HD void tri_item_row(const TriGeo<R>& G, int dy, const int td[2], Acc& acc, UnitCounts* cnt) {
    int mlo = 0, mhi = -1, nhit = 0;
    for (int o = 0; o < 3; ++o) {
        int a, b;
        tri_edge(o, a, b);
        int ca = G.cell[a][1], cb = G.cell[b][1];
        int c0 = (ca < cb ? ca : cb) + 1, c1 = ca < cb ? cb : ca;
        if (dy < c0 || dy > c1) continue;
        int dirk = cb > ca ? 1 : -1;
        R t = (R(dy) - G.x[a][1]) / (G.x[b][1] - G.x[a][1]);
        R xx = G.x[a][0] + t * (G.x[b][0] - G.x[a][0]);
        int m = tri_cross_cell(G, a, b, 1, dy, (int)floor_r(xx), dirk, cnt);
        ++nhit;
        if (G.nE[o][0] > 0)
            mlo = m;
        else
            mhi = m;
    }
    if (nhit != 2) return;
    int n0 = mlo + 1 > 0 ? mlo + 1 : 0, n1 = mhi < td[0] ? mhi : td[0];
    for (int cx = n0; cx <= n1; ++cx) {
        for (int o = 0; o < 4; ++o) {
            int v0 = cx - 1 + (o & 1), v1 = dy - 1 + ((o >> 1) & 1);
            if (v0 < 0 || v0 >= td[0] || v1 < 0 || v1 >= td[1]) continue;
            R sg = ((o & 1) ? -1 : 1) * (((o >> 1) & 1) ? -1 : 1);
            R O[2];
            tri_origin(G, v0, v1, O);
            R P0 = R(cx) - O[0], P1 = R(dy) - O[1];
            R rhoX = G.rhoc + G.g[0] * (P0 + (O[0] - G.c[0])) + G.g[1] * (P1 + (O[1] - G.c[1]));
            acc(v0, v1, 0, sg * P0 * P1 * (rhoX - R(0.5) * (G.g[0] * P0 + G.g[1] * P1)));
            if (cnt) cnt->a++;
        }
    }
}

// Split form of a 2D crossing for a work queue.
//   C record: bits 0-10 c, 11-21 cj, 22 side, 23 k, 24-25 o (edge opposite vertex o)
template <typename R, class Push>
CDP_HD void tri_locate_crossing(const TriGeo<R>& G, int o, int k, int c, const int td[2], Push& push,
                                UnitCounts* cnt) {
    int a, b;
    tri_edge(o, a, b);
    int j = 1 - k;
    int dirk = G.cell[b][k] > G.cell[a][k] ? 1 : -1;
    R evk = (G.x[b][k] - G.x[a][k]) + (G.xl[b][k] - G.xl[a][k]);
    R evj = (G.x[b][j] - G.x[a][j]) + (G.xl[b][j] - G.xl[a][j]);
    R t = ((R(c) - G.x[a][k]) - G.xl[a][k]) / evk;
    int cj = tri_cross_cell(G, a, b, k, c, (int)floor_r(G.x[a][j] + t * evj), dirk, cnt);
    int tj = j == 0 ? td[0] : td[1], tk = k == 0 ? td[0] : td[1];
    if (cj < 0 || cj >= tj) return;
    unsigned long long base = (unsigned long long)c | ((unsigned long long)cj << 11) | ((unsigned long long)k << 23) |
                              ((unsigned long long)o << 24);
    if (c - 1 >= 0 && c - 1 < tk) push(base);
    if (c < tk) push(base | (1ull << 22));
}

template <typename R>
CDP_HD R tri_eval_crossing(const TriGeo<R>& G, unsigned long long r, int& v0, int& v1, int& v2) {
    int c = (int)(r & 2047), cj = (int)((r >> 11) & 2047), side = (int)((r >> 22) & 1), k = (int)((r >> 23) & 1),
        o = (int)((r >> 24) & 3);
    int a, b;
    tri_edge(o, a, b);
    int j = 1 - k;
    int dirk = G.cell[b][k] > G.cell[a][k] ? 1 : -1;
    R ev[2] = {(G.x[b][0] - G.x[a][0]) + (G.xl[b][0] - G.xl[a][0]),
               (G.x[b][1] - G.x[a][1]) + (G.xl[b][1] - G.xl[a][1])};
    R evk = k == 0 ? ev[0] : ev[1], evj = k == 0 ? ev[1] : ev[0];
    R t = ((R(c) - G.x[a][k]) - G.xl[a][k]) / evk;
    int vk = side ? c : c - 1;
    v0 = k == 0 ? vk : cj;
    v1 = k == 1 ? vk : cj;
    v2 = 0;
    R O[2];
    tri_origin(G, v0, v1, O);
    R Pk = R(c) - (k == 0 ? O[0] : O[1]);
    R Pj = (G.x[a][j] - (j == 0 ? O[0] : O[1])) + (G.xl[a][j] + t * evj);
    const R P[2] = {k == 0 ? Pk : Pj, k == 1 ? Pk : Pj};
    R inv = rsqrt_r<R>(ev[0] * ev[0] + ev[1] * ev[1]);
    const R eu[2] = {ev[0] * inv, ev[1] * inv};
    return tri_corner_C(G, o, k, dirk, side ? R(1) : R(-1), eu, P, G.rho[a] + t * (G.rho[b] - G.rho[a]));
}

template <typename R, class Acc>
CDP_HD void tri_unit(const TriGeo<R>& G, const int td[2], Acc& acc, UnitCounts* cnt) {
    for (int i = 0; i < 3; ++i) tri_item_vertex(G, i, td, acc, cnt);
    for (int o = 0; o < 3; ++o)
        for (int k = 0; k < 2; ++k) {
            int c0, n = tri_crossings(G, o, k, td, c0);
            for (int c = c0; c < c0 + n; ++c) tri_item_crossing(G, o, k, c, td, acc, cnt);
        }
    int dy0, n = tri_rows(G, td, dy0);
    for (int t = 0; t < n; ++t) tri_item_row(G, dy0 + t, td, acc, cnt);
}

}  // namespace cdp
