// Projection kernel of tetrahedral meshes (Sect. 3; Algorithm 2 organised per simplex).
//
// k_tet_setup: one thread per tetrahedron canonicalises it (exact orientation, periodic unwrap,
// cells), deposits a tetrahedron inside one cell at once (Algorithm 2, step 1), lists one whose
// bounding box exceeds TB_MAX_CELLS as large, and writes the geometry record of every other one to
// HBM.
//
// k_project_tet<R> is a persistent block-cooperative kernel.  A block takes TB_NT consecutive
// tetrahedra, copies their records into shared memory and gives each a dense box of per-cell
// accumulators, one slot per cell of its bounding box; the tetrahedra are packed, in order, into
// rounds whose boxes fit the block's slots together.  The work of a round is split into three
// phases of independent items -- the vertices (corners B), the (edge, axis, plane) crossings
// (corners C) and the grid lines (corners D, and along x the grid nodes between the two pierced
// facets, corners A) -- whose items of all tetrahedra of the round are numbered consecutively and
// dealt to the block's warps 32 at a time (the three item counts of every unit scanned once per
// round; a warp goes from one phase to the next without waiting for the others), so that the items
// are balanced over the warps.  Locating a corner costs a few exact-sign predicates; evaluating it
// (all the cells around it at once) costs most of the arithmetic, so each warp queues the corners
// it locates as compact records and evaluates them in full batches of 32 identical evaluations.
// Every (corner, cell) contribution is one shared-memory add into the box of its tetrahedron.  At
// the end of the round the boxes are flushed with one FP64 global atomic per non-zero
// (tetrahedron, cell) piece.
//
// k_project_big, launched after it, takes the large tetrahedra of the list one at a time per block
// and projects each in tiles of TB_TE^3 cells: one unit per tile, its record in the tile's frame, its
// items (planes, lines, vertices) clipped to the tile, its box flushed by the whole block.  A
// corner on a tile face is evaluated in both tiles, each keeping the cells of its own.  Tiles
// outside a facet plane are skipped; the x lines leave their runs of inside grid nodes in a table,
// from which a last phase takes the tile's cells column by column (a cell with all eight corners
// inside gets its closed-form mass).
//
// FP32-mixed path only: the mass closure (not in the paper).  The FP64 closed-form masses of the
// tetrahedra of a round minus the (two-float, exact enough) sum of their FP32 pieces is spread over
// those pieces in proportion to their magnitude, so the total mass is exact to FP64 rounding and
// no piece moves by more than about the FP32 rounding of the pieces themselves.  A tiled
// tetrahedron is closed on its own, in two passes over its tiles: the first only sums the pieces,
// the second flushes them with the closure scale and adds what its rounded pieces still miss, in
// FP64, to the cell of vertex 0.
#include <cuda_runtime.h>

#include "cdp_mesh.cuh"
#include "cdp_project.h"

namespace cdp {

namespace {

constexpr int TB_WARPS = 8;                 // warps per block
constexpr int TB_THREADS = 32 * TB_WARPS;   // threads per block
constexpr int TB_NT = 8 * TB_WARPS;         // tetrahedra per block chunk (power of two, <= TB_THREADS)
constexpr int TB_QCAP = 128;                // C / D corner records awaiting evaluation, per warp
constexpr int TB_ACAP = 64;                 // runs of A nodes awaiting evaluation, per warp
constexpr int TB_PCAP = 64;                 // pierced grid lines awaiting their facet searches, per warp
constexpr int TB_OWN_BITS = 7;              // tetrahedron-of-chunk index in a queued record
constexpr unsigned FULL = 0xffffffffu;
static_assert(TB_NT <= (1 << TB_OWN_BITS) && TB_NT <= TB_THREADS && TB_NT % 32 == 0, "chunk index does not fit");

// default largest bounding box (cells) projected by the main kernel (the size-class threshold; the
// launch may choose another up to the block's box slots), and the block's box slots (FP32: sized
// with the rest of the block's shared memory for three resident blocks per SM)
constexpr int TB_MAX_CELLS = 1920;
// largest tile edge (cells) of a tetrahedron whose bounding box exceeds the threshold (the launch
// chooses its edge up to this; both precisions take the same default, so that they take the same
// decisions tile by tile), and the cells of one tile of that edge.  The large-tetrahedron kernel
// has a shared-memory layout of its own (one unit, no chunk records) whose box holds such a tile:
// the work of a tile grows with its surface (its grid lines), its cells with its volume, so the
// largest tile that leaves three FP32 blocks per SM is the fastest.
constexpr int TB_TE = 23;
constexpr int TB_TILE_CELLS = TB_TE * TB_TE * TB_TE;

template <typename R>
struct BoxCap {
    static constexpr int value = sizeof(R) == 4 ? 6144 : 10240;
};
static_assert(BoxCap<float>::value >= TB_MAX_CELLS, "one tetrahedron's box must fit the block's slots");

// Tiling state of a block's current large tetrahedron: uniform over the block, written by thread 0
// only, between barriers.
struct BigState {
    int te;             // tile edge (cells) of this launch
    int ext[3], nt[3];  // bounding-box extent (cells) and tiles along each axis
    int ntiles, tile;   // tiles, next tile; ntiles < 0: the list is exhausted
    int live;           // tiles set up so far in this pass (those the tetrahedron may meet)
    int pass;           // FP32 path: 0 sums the tiles' pieces, 1 flushes them (FP64 path: always 1)
    float scale;        // closure scale of the flush pass
    float s[3];         // sum of the pieces as two floats (hi, lo) and the sum of their magnitudes
};

// The pass of the large-tetrahedron kernel and the lists of the accuracy control.
struct BigPass {
    AccCtl acc;
    int second;
    int te;             // tile edge (cells), at most TB_TE
    int* defer_list;
    long long defer_cap;
    int* clip_list;
    long long clip_cap;
};

// The block's shared memory: NT units of a round (their records, box placements and item counts), a
// box of BOXN slots, the warps' queues, and for the tile rounds a run table of tiles of edge up to TE.
template <typename R, int NT, int BOXN, int TE>
struct TetSharedT {
    using Real = R;
    static constexpr int kNT = NT;                     // units of a round
    static constexpr int kScan = NT < 32 ? 32 : NT;    // entries of the round's item-count scan
    static constexpr int kBox = BOXN;                  // box slots
    static constexpr int kTE = TE;                     // largest tile edge of the run table
    static constexpr int kRuns = (TE + 1) * (TE + 1);  // its x lines
    TetGeo<R> geo[NT];
    R box[BOXN];
    Rec q[TB_WARPS][TB_QCAP];
    unsigned long long aq[TB_WARPS][TB_ACAP];
    unsigned long long pq[TB_WARPS][TB_PCAP];  // pierced lines awaiting their facet searches
    unsigned short xcum[NT][18];     // running count of the crossings of the (edge, axis) pairs
    int boff[NT];                    // first box slot of each tetrahedron of the round
    int lr[NT][6];                   // grid-line ranges of each unit (unit_line_ranges: r0[3], n[3])
    int td[NT][3];                   // box (tile) dimensions of each unit: its bounding box, or one tile
                                     // of a tetrahedron whose bounding box exceeds TB_MAX_CELLS
    TetGeo<R> big0;                  // the large tetrahedron being tiled, in the frame of its tile 0
    short2 runs[kRuns];              // tile rounds: grid nodes inside the tetrahedron on the x line
                                     // through (y, z) = (j, k) of the tile, entry j + (TE + 1) k:
                                     // the node range [x, y] clipped to the tile (empty: x > y)
    BigState bs;                     // its tiling state
    int wsum[TB_WARPS];              // block-scan scratch
    int wsum3[kScan / 32][3];        // the three phases' item counts of each scanning warp's 32 units
    int pre3[3][kScan];              // inclusive prefixes of the three phases' item counts
    float red[3][TB_WARPS];          // block-reduction scratch of the mass closure
};
// the chunk kernel's layout (no tile rounds) and the large-tetrahedron kernel's (one unit per round)
template <typename R>
using TetShared = TetSharedT<R, TB_NT, BoxCap<R>::value, 1>;
template <typename R>
using TetSharedBig = TetSharedT<R, 1, TB_TILE_CELLS, TB_TE>;

// ------------------------------------------------------------------------------------------
// accumulation into the box of tetrahedron `own` (cell (x, y, z) of its bounding box)
// ------------------------------------------------------------------------------------------
// The box of unit `own` with its dimensions read once: add(x, y, z, v) accumulates v into cell
// (x, y, z) of the unit's box (bounds-checked; cells outside the box, which a tile clips, are
// dropped).
template <typename R>
struct BoxAcc {
    R* box;
    int ex, ey, ez;
    template <class SH>
    __device__ __forceinline__ BoxAcc(SH* sh, int own)
        : box(sh->box + sh->boff[own]), ex(sh->td[own][0]), ey(sh->td[own][1]), ez(sh->td[own][2]) {}
    __device__ __forceinline__ void operator()(int x, int y, int z, R v) const {
        if ((unsigned)x < (unsigned)ex && (unsigned)y < (unsigned)ey && (unsigned)z < (unsigned)ez)
            atomicAdd(&box[x + ex * (y + ey * z)], v);
    }
};

// ------------------------------------------------------------------------------------------
// items
// ------------------------------------------------------------------------------------------

// The facets pierced by a grid line (tet_pierced) for every sign mask of the 6 projected edges,
// packed 4 bits per mask into four 64-bit words at compile time.
constexpr unsigned long long pierced_word(int w) {
    unsigned long long v = 0;
    for (int i = 0; i < 16; ++i) v |= (unsigned long long)tet_pierced((unsigned)(w * 16 + i)) << (4 * i);
    return v;
}

__device__ __forceinline__ unsigned pierced_lut(unsigned sgn) {
    constexpr unsigned long long w0 = pierced_word(0), w1 = pierced_word(1), w2 = pierced_word(2),
                                 w3 = pierced_word(3);
    const unsigned hi = sgn >> 4;
    const unsigned long long w = hi == 0 ? w0 : (hi == 1 ? w1 : (hi == 2 ? w2 : w3));
    return (unsigned)(w >> ((sgn & 15u) * 4u)) & 15u;
}

// Exact stage of the crossing-side predicate: sign(X_j - d) (before the dirk orientation) for the
// crossing X of edge a -> b with the grid plane x_k = c: the orient2d, in the axes (j, k), of the
// grid point (d, c) against the projected edge (tet_side2_exact's argument order: axes ascending).
template <typename R>
CDP_COLD int cross_side_exact(const TetGeo<R>& G, int a, int b, int j, int k, int c, int d) {
    return j < k ? tet_side2_exact(G, a, b, j, k, d, c) : -tet_side2_exact(G, a, b, k, j, c, d);
}

// Exact stage of the line signs: bit e of `amb` marks an edge whose filtered orient2d was not
// conclusive; its exact sign replaces bit e of sgn.
template <typename R>
CDP_COLD unsigned line_signs_exact(const TetGeo<R>& G, int j, int k, int dj, int dk, unsigned sgn, unsigned amb) {
    for (int e = 0; e < 6; ++e) {
        if (!((amb >> e) & 1u)) continue;
        int a, b, p, q;
        tet_edge(e, a, b, p, q);
        if (tet_side2_exact(G, a, b, j, k, dj, dk) > 0)
            sgn |= 1u << e;
        else
            sgn &= ~(1u << e);
    }
    return sgn;
}

// Cell along axis j of the crossing of edge a -> b (coordinates in registers: xa_j, xa_k, xb_j, xb_k)
// with the grid plane x_k = c: the d in [lo, hi] with the crossing above plane d and below plane
// d + 1, found from `guess` by an exact-sign search (one predicate per step: the filtered orient2d of
// the grid point (plane, c) against the projected edge, else its exact stage).
template <typename R>
__device__ __forceinline__ int cross_cell_regs(const TetGeo<R>& G, int a, int b, int j, int k, int c, R xaj, R xak,
                                               R xbj, R xbk, int lo, int hi, int guess, int dirk, R B2,
                                               UnitCounts* cnt) {
    int d = guess < lo ? lo : (guess > hi ? hi : guess);
    const R du = xbj - xaj, dv = xbk - xak;
    const R A = du * (R(c) - xak);
    {
        // the common case: both planes around the guess decided by the filter, the crossing
        // between them (the same expressions and decisions as the search below)
        const R v0 = A - dv * (R(d) - xaj), v1 = A - dv * (R(d + 1) - xaj);
        const R s0 = dirk > 0 ? v0 : -v0, s1 = dirk > 0 ? v1 : -v1;
        if ((d == lo || s0 > B2) && (d == hi || s1 < -B2)) return d;
    }
    bool upper = false;  // false: checking plane d (want the crossing above it), true: plane d + 1
#pragma unroll 1
    for (int it = 0; it < 2 * (hi - lo) + 4; ++it) {
        if (!upper && d == lo) {
            upper = true;
            continue;
        }
        if (upper && d == hi) break;
        const int dd = upper ? d + 1 : d;
        // orient2d of the grid point (dd, c) against the projected edge, filtered by B2
        const R val = A - dv * (R(dd) - xaj);
        int sd;
        if (val > B2) {
            sd = 1;
        } else if (val < -B2) {
            sd = -1;
        } else {
            if (cnt) cnt->exact++;
            sd = cross_side_exact(G, a, b, j, k, c, dd);
        }
        sd *= dirk;
        if (!upper) {
            if (sd < 0)
                --d;
            else
                upper = true;
        } else {
            if (sd > 0)
                ++d;
            else
                break;
        }
    }
    return d;
}

// Cell along l of the crossing of facet f (unit normal nf, reference vertex xf) with the grid line
// along l through (dj, dk): the m in [lo, hi] with node m on the near side and node m + 1 on the
// far side, found from `guess` by an exact-sign search (one predicate per step: the filtered
// orient3d of the node against the facet, else its exact stage).
template <typename R>
__device__ __forceinline__ int facet_line_cell_regs(const TetGeo<R>& G, int f, int l, int dj, int dk, int guess,
                                                    int lo, int hi, int up, const R nf[3], const R xf[3], R B3,
                                                    UnitCounts* cnt) {
    int m = guess < lo ? lo : (guess > hi ? hi : guess);
    {
        // the common case: the nodes m and m + 1 decided by the filter, on either side of the
        // facet (the same expressions and decisions as the search below)
        const int g00 = l == 0 ? m : dj, g01 = l == 1 ? m : (l == 0 ? dj : dk), g02 = l == 2 ? m : dk;
        const int g10 = l == 0 ? m + 1 : dj, g11 = l == 1 ? m + 1 : (l == 0 ? dj : dk), g12 = l == 2 ? m + 1 : dk;
        const R v0 = nf[0] * (R(g00) - xf[0]) + nf[1] * (R(g01) - xf[1]) + nf[2] * (R(g02) - xf[2]);
        const R v1 = nf[0] * (R(g10) - xf[0]) + nf[1] * (R(g11) - xf[1]) + nf[2] * (R(g12) - xf[2]);
        const R s0 = up > 0 ? v0 : -v0, s1 = up > 0 ? v1 : -v1;
        if ((m == lo || s0 < -B3) && (m == hi || s1 > B3)) return m;
    }
    bool upper = false;
#pragma unroll 1
    for (int it = 0; it < 2 * (hi - lo) + 4; ++it) {
        if (!upper && m == lo) {
            upper = true;
            continue;
        }
        if (upper && m == hi) break;
        const int t = upper ? m + 1 : m;
        // node (t along l, dj, dk) in axis order against the facet's plane, filtered by B3
        const int g0 = l == 0 ? t : dj, g1 = l == 1 ? t : (l == 0 ? dj : dk), g2 = l == 2 ? t : dk;
        const R val = nf[0] * (R(g0) - xf[0]) + nf[1] * (R(g1) - xf[1]) + nf[2] * (R(g2) - xf[2]);
        int st;
        if (val > B3) {
            st = 1;
        } else if (val < -B3) {
            st = -1;
        } else {
            if (cnt) cnt->exact++;
            st = tet_side3_exact(G, f, g0, g1, g2);
        }
        if (!upper) {
            if (st == up)
                --m;  // node m already past the crossing
            else
                upper = true;
        } else {
            if (st == -up)
                ++m;
            else
                break;
        }
    }
    return m;
}

// Grid lines of a unit: along every axis a, the grid points strictly inside the bounding box
// (lo_a, hi_a] clipped to the unit's box [0, td_a]: first point r0[a], count n[a].
template <typename R>
__device__ __forceinline__ void unit_line_ranges(const TetGeo<R>& G, const int td[3], int r0[3], int n[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int lo = G.lo[a] + 1 > 0 ? G.lo[a] + 1 : 0;
        const int hi = G.hi[a] < td[a] ? G.hi[a] : td[a];
        r0[a] = lo;
        n[a] = hi >= lo ? hi - lo + 1 : 0;
    }
}

// Item counts of a unit (its crossings per (edge, axis) pair, as running counts in xcum, and its
// grid lines, whose ranges go to lr), with the planes and lines clipped to the unit's box.
template <class SH>
__device__ __forceinline__ void unit_prepare(SH* sh, int u, int& n_cross, int& n_lines) {
    using R = typename SH::Real;
    const TetGeo<R>& G = sh->geo[u];
    const int* td = sh->td[u];
    int run = 0;
#pragma unroll 1
    for (int p = 0; p < 18; ++p) {
        const int e = p / 3, k = p - 3 * e;
        int a, b, pp, qq;
        tet_edge(e, a, b, pp, qq);
        const int ca = G.cell[a][k], cb = G.cell[b][k];
        const int lo = (ca < cb ? ca : cb) + 1, hi = ca < cb ? cb : ca;
        const int c0 = lo > 0 ? lo : 0, c1 = hi < td[k] ? hi : td[k];
        run += c1 >= c0 ? c1 - c0 + 1 : 0;
        sh->xcum[u][p] = (unsigned short)run;
    }
    n_cross = run;
    int r0[3], n[3];
    unit_line_ranges(G, td, r0, n);
    for (int a = 0; a < 3; ++a) {
        sh->lr[u][a] = r0[a];
        sh->lr[u][3 + a] = n[a];
    }
    n_lines = n[1] * n[2] + n[0] * n[2] + n[0] * n[1];
}

// B: vertex i of tetrahedron own
template <class SH>
__device__ __forceinline__ void item_vertex(SH* sh, int own, int i) {
    using R = typename SH::Real;
    const TetGeo<R>& G = sh->geo[own];
    const int v0 = G.cell[i][0], v1 = G.cell[i][1], v2 = G.cell[i][2];
    if ((unsigned)v0 >= (unsigned)sh->td[own][0] || (unsigned)v1 >= (unsigned)sh->td[own][1] ||
        (unsigned)v2 >= (unsigned)sh->td[own][2])
        return;  // the vertex lies in another tile
    R O[3], P[3];
    piece_origin(G, v0, v1, v2, O);
    for (int a = 0; a < 3; ++a) P[a] = (G.x[i][a] - O[a]) + G.xl[i][a];
    BoxAcc<R> acc(sh, own);
    acc(v0, v1, v2, tet_corner_B(G, i, P));
}

// crossing t of tetrahedron own: its C record (the crossing point's cells along the two other axes
// located with the exact-sign search, vertex coordinates read once into registers)
template <class SH>
__device__ __forceinline__ Rec item_crossing(const SH* sh, int own, int t, UnitCounts* cnt) {
    using R = typename SH::Real;
    const unsigned short* cum = sh->xcum[own];
    // first (edge, axis) pair whose running count exceeds t
    int p = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (p + step <= 17 && (int)cum[p + step - 1] <= t) p += step;
    const int before = p > 0 ? (int)cum[p - 1] : 0;
    const int e = p / 3, k = p - 3 * e;
    const TetGeo<R>& G = sh->geo[own];
    int a, b, pp, qq;
    tet_edge(e, a, b, pp, qq);
    const R xa0 = G.x[a][0], xa1 = G.x[a][1], xa2 = G.x[a][2];
    const R xb0 = G.x[b][0], xb1 = G.x[b][1], xb2 = G.x[b][2];
    const int ca0 = G.cell[a][0], ca1 = G.cell[a][1], ca2 = G.cell[a][2];
    const int cb0 = G.cell[b][0], cb1 = G.cell[b][1], cb2 = G.cell[b][2];
    const int cak = pick3(ca0, ca1, ca2, k), cbk = pick3(cb0, cb1, cb2, k);
    const int c0 = (cak < cbk ? cak : cbk) + 1;
    const int c = (c0 > 0 ? c0 : 0) + (t - before);  // planes clipped to the unit's box
    const int dirk = cbk > cak ? 1 : -1;
    const R B2 = G.B2;
    // rounded crossing point: guesses of its cells
    const R xak = pick3(xa0, xa1, xa2, k), xbk = pick3(xb0, xb1, xb2, k);
    const R evk = (xbk - xak) + (G.xl[b][k] - G.xl[a][k]);
    const R tt = div_guess((R(c) - xak) - G.xl[a][k], evk);
    const int j1 = k == 0 ? 1 : 0, j2 = k == 2 ? 1 : 2;
    // the cells along the two other axes: both rounded guesses decided by the filter side by side
    // (the common case), else the search of cross_cell_regs for the undecided one(s)
    int cjw[2];
    bool okw[2];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const int j = w == 0 ? j1 : j2;
        const R xaj = pick3(xa0, xa1, xa2, j), xbj = pick3(xb0, xb1, xb2, j);
        const R evj = (xbj - xaj) + (G.xl[b][j] - G.xl[a][j]);
        const int caj = pick3(ca0, ca1, ca2, j), cbj = pick3(cb0, cb1, cb2, j);
        const int lo = caj < cbj ? caj : cbj, hi = caj < cbj ? cbj : caj;
        const int guess = (int)floor_r(xaj + tt * evj);
        const int d = guess < lo ? lo : (guess > hi ? hi : guess);
        const R du = xbj - xaj, dv = xbk - xak;
        const R A = du * (R(c) - xak);
        const R v0 = A - dv * (R(d) - xaj), v1 = A - dv * (R(d + 1) - xaj);
        const R s0 = dirk > 0 ? v0 : -v0, s1 = dirk > 0 ? v1 : -v1;
        cjw[w] = d;
        okw[w] = (d == lo || s0 > B2) && (d == hi || s1 < -B2);
    }
    if (!(okw[0] && okw[1])) {
#pragma unroll 1
        for (int w = 0; w < 2; ++w) {
            if (okw[w]) continue;
            const int j = w == 0 ? j1 : j2;
            const R xaj = pick3(xa0, xa1, xa2, j), xbj = pick3(xb0, xb1, xb2, j);
            const R evj = (xbj - xaj) + (G.xl[b][j] - G.xl[a][j]);
            const int caj = pick3(ca0, ca1, ca2, j), cbj = pick3(cb0, cb1, cb2, j);
            const int lo = caj < cbj ? caj : cbj, hi = caj < cbj ? cbj : caj;
            cjw[w] = cross_cell_regs(G, a, b, j, k, c, xaj, xak, xbj, xbk, lo, hi, (int)floor_r(xaj + tt * evj), dirk,
                                     B2, cnt);
        }
    }
    const int cj0 = cjw[0], cj1 = cjw[1];
    if ((unsigned)cj0 >= (unsigned)sh->td[own][j1] || (unsigned)cj1 >= (unsigned)sh->td[own][j2]) return 0;
    // bit 39 marks the record as present (every field may be 0 in a tile)
    return (Rec)c | ((Rec)cj0 << 11) | ((Rec)cj1 << 22) | ((Rec)k << 34) | ((Rec)e << 36) | (1ull << 39);
}

// Line t of tetrahedron own: which facets the grid line pierces.  Returns the pierced-line record
// (facet mask in bits 0-3, l in 4-5, dj in 6-16, dk in 17-27; 0 when the line misses).
template <class SH>
__device__ __forceinline__ unsigned long long item_line_test(const SH* sh, int own, int t,
                                                             UnitCounts* cnt) {
    using R = typename SH::Real;
    const TetGeo<R>& G = sh->geo[own];
    // lines along l through the grid points (dj, dk) inside the bounding box and the unit's box
    const int* lr = sh->lr[own];
    const int r0[3] = {lr[0], lr[1], lr[2]}, n[3] = {lr[3], lr[4], lr[5]};
    int l, nj;
    if (t < n[1] * n[2]) {
        l = 0;
        nj = n[1];
    } else if ((t -= n[1] * n[2]) < n[0] * n[2]) {
        l = 1;
        nj = n[0];
    } else {
        t -= n[0] * n[2];
        l = 2;
        nj = n[0];
    }
    const int j = l == 0 ? 1 : 0, k = l == 2 ? 1 : 2;
    const int tq = t / nj;
    const int dj = pick3(r0[0], r0[1], r0[2], j) + t - tq * nj, dk = pick3(r0[0], r0[1], r0[2], k) + tq;
    // signs of the 6 projected edges against (dj, dk) (the filtered orient2d of the edge, from the
    // projected vertices read once; inconclusive ones settled exactly)
    unsigned sgn = 0, amb = 0;
    {
        const R B2 = G.B2;
        R pj[4], pk[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            pj[v] = G.x[v][j];
            pk[v] = G.x[v][k];
        }
        const R fj = R(dj), fk = R(dk);
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const int a = e < 3 ? 0 : (e < 5 ? 1 : 2), b = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
            const R du = pj[b] - pj[a], dv = pk[b] - pk[a];
            const R val = du * (fk - pk[a]) - dv * (fj - pj[a]);
            sgn |= (val > R(0) ? 1u : 0u) << e;
            amb |= (val <= B2 && val >= -B2 ? 1u : 0u) << e;
        }
    }
    if (amb) {
        if (cnt) cnt->exact += __popc(amb);
        sgn = line_signs_exact(G, j, k, dj, dk, sgn, amb);
    }
    const unsigned hits = pierced_lut(sgn);
    if (!hits) return 0ull;
    return (unsigned long long)hits | ((unsigned long long)l << 4) | ((unsigned long long)dj << 6) |
           ((unsigned long long)dk << 17);
}

// A pierced line (record of item_line_test): its D records (one per pierced facet, the cell along
// the line located with the exact-sign search) and the run of A nodes between them (x lines only).
template <bool TILE, class SH>
__device__ __forceinline__ int item_line_facets(SH* sh, int own, unsigned long long pr, Rec& r0,
                                                Rec& r1, unsigned long long& arun, UnitCounts* cnt) {
    using R = typename SH::Real;
    const TetGeo<R>& G = sh->geo[own];
    const unsigned hits = (unsigned)(pr & 15u);
    const int l = (int)((pr >> 4) & 3u), dj = (int)((pr >> 6) & 2047u), dk = (int)((pr >> 17) & 2047u);
    const int j = l == 0 ? 1 : 0, k = l == 2 ? 1 : 2;
    int nr = 0, npierced = 0;
    arun = 0;
    int mlo = 0, mhi = -1;
    const int lol = pick3(G.lo[0], G.lo[1], G.lo[2], l), hil = pick3(G.hi[0], G.hi[1], G.hi[2], l);
    const R B3 = G.B3;
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        if (!((hits >> f) & 1u)) continue;
        const int va = f == 0 ? 1 : 0;
        const R nf[3] = {G.n[f][0], G.n[f][1], G.n[f][2]};
        const R xf[3] = {G.x[va][0], G.x[va][1], G.x[va][2]};
        const R fj = pick3(nf[0], nf[1], nf[2], j), fk = pick3(nf[0], nf[1], nf[2], k),
                fl = pick3(nf[0], nf[1], nf[2], l);
        const R off = div_guess(-(fj * ((R(dj) - pick3(xf[0], xf[1], xf[2], j)) - G.xl[va][j]) +
                                  fk * ((R(dk) - pick3(xf[0], xf[1], xf[2], k)) - G.xl[va][k])),
                                fl);
        const int up = G.ns[f][l] > 0 ? 1 : -1;
        const int m = facet_line_cell_regs(G, f, l, dj, dk, (int)floor_r(pick3(xf[0], xf[1], xf[2], l) + off), lol,
                                           hil, up, nf, xf, B3, cnt);
        if (up > 0)
            mlo = m;
        else
            mhi = m;
        ++npierced;
        if ((unsigned)m >= (unsigned)pick3(sh->td[own][0], sh->td[own][1], sh->td[own][2], l)) continue;
        const Rec r = (Rec)m | ((Rec)dj << 11) | ((Rec)dk << 22) | ((Rec)l << 35) | ((Rec)f << 37);
        if (nr == 0)
            r0 = r;
        else
            r1 = r;
        ++nr;
    }
    // grid nodes strictly inside: (cx, dj, dk) for cx in [mlo + 1, mhi] within the unit's box
    // [0, td_0] (x lines only): a run of A nodes (bit 51 marks the record as present), or in a tile
    // round the line's entry of the run table
    const int cx0 = mlo + 1 > 0 ? mlo + 1 : 0, cx1 = mhi < sh->td[own][0] ? mhi : sh->td[own][0];
    if (l == 0 && npierced == 2 && cx1 >= cx0) {
        if (TILE)
            sh->runs[dj + (SH::kTE + 1) * dk] = make_short2((short)cx0, (short)cx1);
        else
            arun = (unsigned long long)cx0 | ((unsigned long long)cx1 << 11) | ((unsigned long long)dj << 22) |
                   ((unsigned long long)dk << 33) | (1ull << 51);
    }
    return nr;
}

// ------------------------------------------------------------------------------------------
// evaluation of queued corners
// ------------------------------------------------------------------------------------------

template <bool STATS, class SH>
__device__ __forceinline__ void eval_CD(SH* sh, Rec r, bool is_c, UnitCounts& cnt) {
    using R = typename SH::Real;
    const int own = (int)((r >> 40) & ((1 << TB_OWN_BITS) - 1));
    const TetGeo<R>& G = sh->geo[own];
    BoxAcc<R> acc(sh, own);
    if (is_c) {
        int e, k, c, cj1, cj2;
        decode_C(r, e, k, c, cj1, cj2);
        tet_eval_C2(G, e, k, c, cj1, cj2, acc);
        if (STATS) cnt.c += 2;
    } else {
        int f, l, dj, dk, m;
        decode_D(r, f, l, dj, dk, m);
        tet_eval_D4(G, f, l, dj, dk, m, acc);
        if (STATS) cnt.d += 4;
    }
}

// a run of A nodes (grid nodes inside the tetrahedron on one x line): the 8 cells of each node
template <bool STATS, class SH>
__device__ __forceinline__ void eval_A(SH* sh, unsigned long long r, UnitCounts& cnt) {
    using R = typename SH::Real;
    const int own = (int)((r >> 44) & ((1 << TB_OWN_BITS) - 1));
    const int cx0 = (int)(r & 2047), cx1 = (int)((r >> 11) & 2047);
    const int dj = (int)((r >> 22) & 2047), dk = (int)((r >> 33) & 2047);
    const TetFrame<R> F = tet_frame(sh->geo[own]);
    BoxAcc<R> acc(sh, own);
    // the cells of the run's nodes share their columns along y and z: two piece-origin components
    // along each (the centroid clamped into the central half of the cell), and the offsets of the
    // nodes from them; the density at a node is the same for its 8 cells
    const R Py0 = R(dj) - clamp_r(F.c[1], R(dj - 1) + R(0.25), R(dj - 1) + R(0.75)),
            Py1 = R(dj) - clamp_r(F.c[1], R(dj) + R(0.25), R(dj) + R(0.75));
    const R Pz0 = R(dk) - clamp_r(F.c[2], R(dk - 1) + R(0.25), R(dk - 1) + R(0.75)),
            Pz1 = R(dk) - clamp_r(F.c[2], R(dk) + R(0.25), R(dk) + R(0.75));
    const R ryz = F.rhoc + F.g[1] * (R(dj) - F.c[1]) + F.g[2] * (R(dk) - F.c[2]);
#pragma unroll 1
    for (int cx = cx0; cx <= cx1; ++cx) {
        const R Px0 = R(cx) - clamp_r(F.c[0], R(cx - 1) + R(0.25), R(cx - 1) + R(0.75)),
                Px1 = R(cx) - clamp_r(F.c[0], R(cx) + R(0.25), R(cx) + R(0.75));
        const R rhoX = ryz + F.g[0] * (R(cx) - F.c[0]);
#pragma unroll 1
        for (int o = 0; o < 8; ++o) {
            const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
            const R P[3] = {ox ? Px1 : Px0, oy ? Py1 : Py0, oz ? Pz1 : Pz0};
            // the node is the cell's upper corner along a when the cell index is node - 1
            const R sg = R((ox ? -1 : 1) * (oy ? -1 : 1) * (oz ? -1 : 1));
            acc(cx - 1 + ox, dj - 1 + oy, dk - 1 + oz, tet_corner_A(F, P, rhoX, sg));
        }
        if (STATS) cnt.a += 8;
    }
}

// Column t = y + td_1 z of the tile (unit 0, tile rounds): the cells (x, y, z), x in [0, td_0), with
// their A corners from the run table.  A cell whose eight corners are all inside the tetrahedron
// lies inside it: its piece is the integral of rho over the cell, rho at its centre (the eight A
// terms sum to exactly that).  Otherwise the A terms of its inside corners are summed with the
// cell's piece origin.  Columns are disjoint and the round's other phases are done, so the box
// entries are updated without atomics.  Returns the number of (A corner, cell) incidences.
template <class SH>
__device__ __noinline__ unsigned item_column(SH* sh, int t) {
    using R = typename SH::Real;
    const int ex = sh->td[0][0], ey = sh->td[0][1];
    const int z = t / ey, y = t - z * ey;
    short2 run[4];
    int amin = 1 << 20, bmax = -(1 << 20), amax = -(1 << 20), bmin = 1 << 20;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        run[w] = sh->runs[(y + (w & 1)) + (SH::kTE + 1) * (z + (w >> 1))];
        if (run[w].x <= run[w].y) {
            amin = min(amin, (int)run[w].x);
            bmax = max(bmax, (int)run[w].y);
        }
        amax = max(amax, (int)run[w].x);  // (an empty run, (1, 0), leaves no cell entirely inside)
        bmin = min(bmin, (int)run[w].y);
    }
    if (amin > bmax) return 0u;
    const int x0 = max(amin - 1, 0), x1 = min(bmax, ex - 1);
    const int flo = amax, fhi = bmin - 1;  // the cells with all eight corners inside
    const TetFrame<R> F = tet_frame(sh->geo[0]);
    const R ryz = F.rhoc + F.g[1] * ((R(y) + R(0.5)) - F.c[1]) + F.g[2] * ((R(z) + R(0.5)) - F.c[2]);
    R* col = sh->box + sh->boff[0] + ex * (y + ey * z);
    unsigned n = 0;
#pragma unroll 1
    for (int x = x0; x <= x1; ++x) {
        R v;
        if (x >= flo && x <= fhi) {
            v = ryz + F.g[0] * ((R(x) + R(0.5)) - F.c[0]);
            n += 8u;
        } else {
            // bit 2 w + o: corner x + o on the line (y + (w & 1), z + (w >> 1))
            unsigned mask = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                mask |= (run[w].x <= x && x <= run[w].y ? 1u : 0u) << (2 * w);
                mask |= (run[w].x <= x + 1 && x + 1 <= run[w].y ? 1u : 0u) << (2 * w + 1);
            }
            if (!mask) continue;
            R O[3];
            piece_origin(F, x, y, z, O);
            v = R(0);
#pragma unroll 1
            for (int b = 0; b < 8; ++b) {
                if (!((mask >> b) & 1u)) continue;
                // the corner is the cell's upper one along an axis where its offset is 1
                const int ox = b & 1, oy = (b >> 1) & 1, oz = b >> 2;
                const R P[3] = {R(x + ox) - O[0], R(y + oy) - O[1], R(z + oz) - O[2]};
                const R sg = R((ox ? 1 : -1) * (oy ? 1 : -1) * (oz ? 1 : -1));
                v += tet_corner_A(F, P, rho_from_P(F, P, O), sg);
            }
            n += __popc(mask);
        }
        col[x] += v;
    }
    return n;
}

// absolute cell index along one axis (periodic wrap without a division in the common case)
__device__ __forceinline__ int wrap_axis(int v, int n, int periodic, bool& ok) {
    if (!periodic) {
        ok = ok && v >= 0 && v < n;
        return v;
    }
    if (v >= n) v -= n;
    if (v < 0) v += n;
    if ((unsigned)v >= (unsigned)n) {
        v %= n;
        if (v < 0) v += n;
    }
    return v;
}

// The FP64 value of a float, assembled from its bits with integer operations (this GPU's FP64
// pipe, which also converts, runs at a small fraction of the FP32 rate); zero, subnormal and
// non-finite inputs take the converting instruction.
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(e + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// (hi, lo) += v with the rounding error of hi + v kept in lo (Knuth's two-sum, FP32 only)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bv = s - hi;
    const float err = (hi - (s - bv)) + (v - bv);
    hi = s;
    lo += err;
}

// inclusive prefix sum over the block of one value per thread (thread order)
__device__ __forceinline__ int block_scan(int v, int* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    __syncthreads();  // wsum free
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    return v + off;
}

// first index t of the non-decreasing pre[0, TB_NT) with pre[t] > u (u < pre[TB_NT - 1])
template <int N>
__device__ __forceinline__ int upper_index(const int* pre, int u) {
    int pos = 0;
#pragma unroll
    for (int step = N / 2; step > 0; step >>= 1)
        if (pre[pos + step - 1] <= u) pos += step;
    return pos;
}

// The three phases of one round over the units of the block's shared records whose thread (index
// < TB_NT) has `in` set: items dealt to the warps 32 at a time, located corners queued per warp and
// evaluated in full batches into the units' boxes.  Every thread of the block calls it.
template <bool STATS, bool TILE, class SH>
__device__ __forceinline__ void round_phases(SH* sh, bool in, int n_cross, int n_lines, UnitCounts& cnt,
                                             UnitCounts* pc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Rec* const q = sh->q[warp];
    unsigned long long* const aq = sh->aq[warp];
    unsigned long long* const pq = sh->pq[warp];
    const unsigned lt_mask = (1u << lane) - 1u;
    // the item counts of the three phases of the round's units (threads 0 .. TB_NT - 1), scanned at once
    // (a tile round's one unit: its counts are in pre3 already, written by the warp that set it up)
    if (!TILE) {
        constexpr int SW = SH::kScan / 32;  // the warps that scan, one unit per thread
        int m0 = in ? 4 : 0, m1 = in ? n_cross : 0, m2 = in ? n_lines : 0;
        if (warp < SW) {
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t0 = __shfl_up_sync(FULL, m0, o), t1 = __shfl_up_sync(FULL, m1, o),
                          t2 = __shfl_up_sync(FULL, m2, o);
                if (lane >= o) {
                    m0 += t0;
                    m1 += t1;
                    m2 += t2;
                }
            }
            if (lane == 31) {
                sh->wsum3[warp][0] = m0;
                sh->wsum3[warp][1] = m1;
                sh->wsum3[warp][2] = m2;
            }
        }
        __syncthreads();
        if (warp < SW) {
            for (int w = 0; w < warp; ++w) {
                m0 += sh->wsum3[w][0];
                m1 += sh->wsum3[w][1];
                m2 += sh->wsum3[w][2];
            }
            sh->pre3[0][tid] = m0;
            sh->pre3[1][tid] = m1;
            sh->pre3[2][tid] = m2;
        }
        __syncthreads();
    }
#pragma unroll 1
    for (int ph = 0; ph < 3; ++ph) {
        const int* const pre_ph = sh->pre3[ph];
        const int tot = pre_ph[SH::kScan - 1];
        // item rounds of 32 dealt to the warps in turn; each warp queues and evaluates its own
        // located corners
        const int nrounds = (tot + 31) >> 5;
        const int my_rounds = nrounds > warp ? (nrounds - warp + TB_WARPS - 1) / TB_WARPS : 0;
        unsigned head = 0, tail = 0, ahead = 0, atail = 0, phead = 0, ptail = 0;
#pragma unroll 1
        for (int i = 0; i < my_rounds; ++i) {
            const int u = ((warp + i * TB_WARPS) << 5) + lane;
            Rec r0 = 0;
            unsigned long long pline = 0;
            int own = 0;
            if (u < tot) {
                own = upper_index<SH::kScan>(pre_ph, u);
                const int t = u - (own > 0 ? pre_ph[own - 1] : 0);
                if (ph == 0) {
                    item_vertex(sh, own, t);
                    if (STATS) cnt.b++;
                } else if (ph == 1) {
                    r0 = item_crossing(sh, own, t, pc);
                } else {
                    pline = item_line_test(sh, own, t, pc);
                }
            }
            // append located corners (C) or pierced lines to the warp's queues (warp-aggregated,
            // no atomics)
            {
                const unsigned bc = __ballot_sync(FULL, r0 != 0);
                if (r0) q[(tail + __popc(bc & lt_mask)) & (TB_QCAP - 1)] = r0 | ((Rec)own << 40);
                tail += __popc(bc);
                const unsigned bp = __ballot_sync(FULL, pline != 0);
                if (pline) pq[(ptail + __popc(bp & lt_mask)) & (TB_PCAP - 1)] = pline | ((unsigned long long)own << 28);
                ptail += __popc(bp);
            }
            __syncwarp();
            const bool last_round = i + 1 == my_rounds;
            // Work off the queues in full batches of 32 (after the warp's last items, down to empty):
            // facet searches of pierced lines (which feed the D and A queues, when they have room),
            // then C / D corners, then runs of A nodes.  One call site each.
#pragma unroll 1
            for (;;) {
                const unsigned pav = ptail - phead, cav = tail - head, aav = atail - ahead;
                const bool p_ready = pav >= 32u || (last_round && pav > 0u);
                if (p_ready && cav <= TB_QCAP - 64u && aav <= TB_ACAP - 32u) {
                    Rec d0 = 0, d1 = 0;
                    unsigned long long arun = 0;
                    int nr = 0, lown = 0;
                    if ((unsigned)lane < pav) {
                        const unsigned long long pr = pq[(phead + lane) & (TB_PCAP - 1)];
                        lown = (int)((pr >> 28) & ((1u << TB_OWN_BITS) - 1u));
                        nr = item_line_facets<TILE>(sh, lown, pr, d0, d1, arun, pc);
                    }
                    phead += pav < 32u ? pav : 32u;
                    const Rec ob = (Rec)lown << 40;
                    const unsigned b0 = __ballot_sync(FULL, nr >= 1), b1 = __ballot_sync(FULL, nr >= 2);
                    const unsigned off = __popc(b0 & lt_mask) + __popc(b1 & lt_mask);
                    if (nr >= 1) q[(tail + off) & (TB_QCAP - 1)] = d0 | ob;
                    if (nr >= 2) q[(tail + off + 1) & (TB_QCAP - 1)] = d1 | ob;
                    tail += __popc(b0) + __popc(b1);
                    const unsigned ba = __ballot_sync(FULL, arun != 0);
                    if (arun) aq[(atail + __popc(ba & lt_mask)) & (TB_ACAP - 1)] = arun | ((unsigned long long)lown << 44);
                    atail += __popc(ba);
                    __syncwarp();
                    continue;
                }
                const bool drain = last_round && pav == 0u;
                if (cav >= 32u || (drain && cav > 0u)) {
                    if ((unsigned)lane < cav) eval_CD<STATS>(sh, q[(head + lane) & (TB_QCAP - 1)], ph == 1, cnt);
                    head += cav < 32u ? cav : 32u;
                    __syncwarp();
                    continue;
                }
                if (aav >= 32u || (drain && aav > 0u)) {
                    if ((unsigned)lane < aav) eval_A<STATS>(sh, aq[(ahead + lane) & (TB_ACAP - 1)], cnt);
                    ahead += aav < 32u ? aav : 32u;
                    __syncwarp();
                    continue;
                }
                break;
            }
        }
        // (no barrier: a warp goes on to the next phase at once)
    }
    __syncthreads();  // every warp has finished the line phase: the boxes are complete
}

// How a round's boxes are flushed.  FLUSH_CLOSE_ROUND: the round's own mass closure (FP32 path:
// the closed-form masses of its tetrahedra minus the sum of their pieces, spread over the pieces;
// the accuracy control keeps tetrahedra whose pieces may carry a large rounding error out of the
// rounds, so the round's residual is a few FP32 ulps of its pieces).  FLUSH_SUM_ONLY: the pieces are
// only summed into (s_hi, s_lo, s_abs) and cleared (first pass over the tiles of a large
// tetrahedron).  FLUSH_SCALED: the pieces are flushed with the given closure scale, and summed as
// well (second pass).
// FLUSH_CLOSE_UNITS: every tetrahedron's own closure (its residual spread over its own pieces), for
// the second pass, whose rounds hold only the deferred tetrahedra: their pieces may carry the
// larger rounding the accuracy control accepted, which a round's closure would spread over the
// round's other tetrahedra.
enum FlushMode { FLUSH_CLOSE_ROUND = 0, FLUSH_SUM_ONLY = 1, FLUSH_SCALED = 2, FLUSH_CLOSE_UNITS = 3 };

// (hi, lo) as a two-float sum and asum summed over the block; every thread gets the totals
__device__ __forceinline__ void block_sum2(float& hi, float& lo, float& asum, float (*red)[TB_WARPS]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(FULL, hi, o), olo = __shfl_xor_sync(FULL, lo, o);
        lo += olo;
        two_sum_acc(hi, lo, ohi);
        asum += __shfl_xor_sync(FULL, asum, o);
    }
    __syncthreads();  // red is free
    if (lane == 0) {
        red[0][warp] = hi;
        red[1][warp] = lo;
        red[2][warp] = asum;
    }
    __syncthreads();
    hi = 0.f;
    lo = 0.f;
    asum = 0.f;
    for (int w = 0; w < TB_WARPS; ++w) {
        lo += red[1][w];
        two_sum_acc(hi, lo, red[0][w]);
        asum += red[2][w];
    }
}

// The quantities of the accuracy control of one simplex (AccCtl): its largest |density| and the
// norm of its density gradient (both premultiplied by the cell volume; gradient per cell).
template <typename R>
__device__ __forceinline__ void acc_terms(const TetGeo<R>& G, float& rmax, float& gn) {
    rmax = fmaxf(fmaxf(fabsf((float)G.rho[0]), fabsf((float)G.rho[1])), fmaxf(fabsf((float)G.rho[2]), fabsf((float)G.rho[3])));
    const float g0 = (float)G.g[0], g1 = (float)G.g[1], g2 = (float)G.g[2];
    gn = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
}

// The largest |cell mass| of problem p after the first pass (0 before it has been taken).
__device__ __forceinline__ double first_pass_max(const Counters* ctr, int p) {
    return __longlong_as_double((long long)*(volatile const unsigned long long*)&ctr->mmax_bits[p]);
}

// Where the set-up sends a simplex whose box fits the chunks: 0 the chunks (Franklin's sum in this
// pass), 1 the deferred list (first pass: its gradient is steep), 2 the clip list (second pass: its
// cancellation bound exceeds the accepted error).
template <typename R>
__device__ __forceinline__ int acc_route(const TetGeo<R>& G, const AccCtl& acc, bool second, const Counters* ctr) {
    float rmax, gn;
    acc_terms(G, rmax, gn);
    if (!second) return gn > acc.defer_ratio * rmax ? 1 : 0;
    return acc.eps_k_grad * (double)gn > acc.tau * first_pass_max(ctr, G.prob) ? 2 : 0;
}

__device__ __forceinline__ void list_append(int* list, long long cap, unsigned* count, int s) {
    const unsigned at = atomicAdd(count, 1u);
    if ((long long)at < cap) list[at] = s;
}

// Flush every box of the round: one FP64 atomic per non-zero piece (FP32 path: and one more for its
// share of the mass-closure residual, `scale` |piece|).  Every thread of the block calls it; the
// piece sums of FLUSH_SUM_ONLY / FLUSH_SCALED are added into `sums` by thread 0, and FLUSH_SUM_ONLY
// also copies the box to `store` when it is given.  With
// `whole` (one unit, a tile) the whole block flushes that unit's box; otherwise each warp flushes
// the boxes of every TB_WARPS-th unit.  Each unit's grid is its problem's (T); the units of a round of
// the first pass belong to one problem (a problem's tetrahedra start a new chunk), so the round's
// closure keeps every problem's mass.
template <class SH>
__device__ __forceinline__ void round_flush(SH* sh, const ProbTable& T, bool in, int pre_box,
                                            int mode, float scale, bool whole, float* sums, float* store) {
    using R = typename SH::Real;
    constexpr bool fp32 = sizeof(R) == 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the round's units are a prefix of the box slots: the last one ends at the largest pre_box
    int used_slots = 0;
    if (whole) {
        // one unit, set up before the round's barriers
        used_slots = sh->boff[0] >= 0 ? sh->td[0][0] * sh->td[0][1] * sh->td[0][2] : 0;
    } else {
        int m = in ? pre_box : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
        if (lane == 0) sh->wsum[warp] = m;
        __syncthreads();
        for (int w = 0; w < TB_WARPS; ++w) used_slots = max(used_slots, sh->wsum[w]);
    }
    if (fp32 && mode != FLUSH_SCALED && mode != FLUSH_CLOSE_UNITS) {
        // FP32 pieces of the round minus the closed-form masses of its tetrahedra, summed as two
        // floats (exact enough, FP32 arithmetic only); the residual is then spread over the pieces
        // in proportion to their magnitude
        float hi = 0.f, lo = 0.f, asum = 0.f;
        if (in && mode == FLUSH_CLOSE_ROUND) {
            two_sum_acc(hi, lo, -sh->geo[tid].mexact_hi);
            lo -= sh->geo[tid].mexact_lo;
        }
        for (int e = tid; e < used_slots; e += TB_THREADS) {
            const float v = (float)sh->box[e];
            if (mode == FLUSH_SUM_ONLY) {
                sh->box[e] = R(0);
                if (store) store[e] = v;
            }
            two_sum_acc(hi, lo, v);
            asum += fabsf(v);
        }
        block_sum2(hi, lo, asum, sh->red);
        if (mode == FLUSH_SUM_ONLY) {
            if (tid == 0) {
                sums[1] += lo;
                two_sum_acc(sums[0], sums[1], hi);
                sums[2] += asum;
            }
            return;
        }
        const float resid = -(hi + lo);
        if (asum > 0.f) {
            scale = resid * __frcp_rn(asum);
        } else if (tid == 0) {
            // no piece to carry it: the cell of vertex 0 of the round's first unit
            int t = 0;
            while (t < SH::kNT - 1 && sh->boff[t] < 0) ++t;
            const TetGeo<R>& G = sh->geo[t];
            const ProbEntry& P = T.p[G.prob];
            const long long idx =
                flat_cell(P.g, G.anchor[0] + G.cell[0][0], G.anchor[1] + G.cell[0][1], G.anchor[2] + G.cell[0][2]);
            if (idx >= 0) atomicAdd(P.out + idx, (double)resid);
        }
    }
    const int gsize = whole ? TB_THREADS : 32, glane = whole ? tid : lane;
    float f_hi = 0.f, f_lo = 0.f, f_abs = 0.f;  // FLUSH_SCALED: the flushed pieces
#pragma unroll 1
    for (int t = whole ? 0 : warp; t < (whole ? 1 : SH::kNT); t += TB_WARPS) {
        const int base = sh->boff[t];
        if (base < 0) continue;
        const TetGeo<R>& G = sh->geo[t];
        const GridDesc& g = T.p[G.prob].g;
        double* const out = T.p[G.prob].out;
        const int ex = sh->td[t][0], ey = sh->td[t][1], ez = sh->td[t][2];
        const int size = ex * ey * ez;
        const int ax = G.anchor[0], ay = G.anchor[1], az = G.anchor[2];
        if (fp32 && mode == FLUSH_CLOSE_UNITS) {
            // this tetrahedron's closure: its closed-form mass minus the two-float sum of its pieces,
            // spread over them in proportion to their magnitude (the warp's lanes share the box)
            float hi = 0.f, lo = 0.f, asum = 0.f;
            if (lane == 0) {
                two_sum_acc(hi, lo, -G.mexact_hi);
                lo -= G.mexact_lo;
            }
            for (int e = lane; e < size; e += 32) {
                const float v = (float)sh->box[base + e];
                two_sum_acc(hi, lo, v);
                asum += fabsf(v);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ohi = __shfl_xor_sync(FULL, hi, o), olo = __shfl_xor_sync(FULL, lo, o);
                lo += olo;
                two_sum_acc(hi, lo, ohi);
                asum += __shfl_xor_sync(FULL, asum, o);
            }
            const float resid = -(hi + lo);
            scale = asum > 0.f ? resid * __frcp_rn(asum) : 0.f;
            if (!(asum > 0.f) && lane == 0) {
                const long long idx = flat_cell(g, ax + G.cell[0][0], ay + G.cell[0][1], az + G.cell[0][2]);
                if (idx >= 0) atomicAdd(out + idx, (double)resid);
            }
        }
        const float inv_ex = __frcp_rn((float)ex), inv_ey = __frcp_rn((float)ey);
        // a box inside the grid needs no wrap: flat index = base + (x n1 + y) n2 + z
        const bool inside =
            ax >= 0 && ay >= 0 && az >= 0 && ax + ex <= g.n[0] && ay + ey <= g.n[1] && az + ez <= g.n[2];
        const long long cbase = ((long long)ax * g.n[1] + ay) * g.n[2] + az;
#pragma unroll 1
        for (int e = glane; e < size; e += gsize) {
            const R v = sh->box[base + e];
            if (v == R(0)) continue;
            sh->box[base + e] = R(0);
            if (fp32 && mode == FLUSH_SCALED) {
                two_sum_acc(f_hi, f_lo, (float)v);
                f_abs += fabsf((float)v);
            }
            // e = x + ex (y + ey z): quotients from float reciprocals, corrected exactly
            int r = (int)((float)e * inv_ex);
            r += (r + 1) * ex <= e ? 1 : 0;
            r -= r * ex > e ? 1 : 0;
            const int x = e - r * ex;
            int z = (int)((float)r * inv_ey);
            z += (z + 1) * ey <= r ? 1 : 0;
            z -= z * ey > r ? 1 : 0;
            const int y = r - z * ey;
            double* cell;
            if (inside) {
                cell = out + cbase + ((long long)x * g.n[1] + y) * g.n[2] + z;
            } else {
                bool ok = true;
                const int cx = wrap_axis(ax + x, g.n[0], g.periodic, ok);
                const int cy = wrap_axis(ay + y, g.n[1], g.periodic, ok);
                const int cz = wrap_axis(az + z, g.n[2], g.periodic, ok);
                if (!ok) continue;
                cell = out + ((long long)cx * g.n[1] + cy) * g.n[2] + cz;
            }
            if constexpr (fp32) {
                atomicAdd(cell, f32_to_f64((float)v));
                // the piece's share of the closure residual (FP64 atomics are cheap here)
                atomicAdd(cell, f32_to_f64(scale * fabsf((float)v)));
            } else {
                atomicAdd(cell, (double)v);
            }
        }
    }
    if (fp32 && mode == FLUSH_SCALED) {
        block_sum2(f_hi, f_lo, f_abs, sh->red);
        if (tid == 0) {
            sums[1] += f_lo;
            two_sum_acc(sums[0], sums[1], f_hi);
            sums[2] += f_abs;
        }
    }
    // (the next round's barriers order the flush before new box writes)
}

}  // namespace

// One pass of the set-up over the tetrahedra of one batch (thread i < nb for the batch's tetrahedron
// i):
// Indices are in the group's simplex numbering (T: each problem's simplices from its s_off, a
// multiple of TB_NT; the indices between two problems are no simplex and get need = 0).
//  first pass  (list == null) the batch is [s0, s0 + nb) of the numbering.  Canonicalise (exact
//              orientation, periodic unwrap, cells); a tetrahedron inside one cell deposits its
//              mass at once (Algorithm 2, step 1); one whose bounding box exceeds TB_MAX_CELLS is
//              listed as large (k_project_big); one with a steep gradient is deferred; every other
//              one gets its geometry record geo[i] and need[i] = its bounding-box cell count.
//  second pass (list = the deferred list) the batch is entries [s0, s0 + nb) of the list, nb
//              capped by the list's count on the device.  A large one is listed again (the list was
//              emptied between the passes); the others get their record, or are sent to the clip
//              list when their cancellation bound exceeds the accepted error (AccCtl).
// need[i] = 0 for every tetrahedron with nothing left for the chunks.
template <typename R>
__global__ void __launch_bounds__(128) k_tet_setup(const __grid_constant__ ProbTable T, long long s0, long long nb,
                                                   const VertexRec* __restrict__ V, Counters* __restrict__ ctr,
                                                   TetGeo<R>* __restrict__ geo, int* __restrict__ need,
                                                   int* __restrict__ big_list, long long big_cap, int count,
                                                   int max_cells, const unsigned char* __restrict__ levels,
                                                   const int* __restrict__ list, AccCtl acc,
                                                   int* __restrict__ defer_list,
                                                   long long defer_cap, int* __restrict__ clip_list, long long clip_cap) {
    // the block's records are assembled in shared memory and written out with coalesced stores
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TetGeo<R>* stage = reinterpret_cast<TetGeo<R>*>(smem_raw);
    const bool second = list != nullptr;
    if (second) {
        const long long listed = (long long)*(volatile const unsigned*)&ctr->defer_count;
        const long long avail = (listed < defer_cap ? listed : defer_cap) - s0;
        nb = avail < 0 ? 0 : (avail < nb ? avail : nb);
    }
    int n_zero = 0, n_single = 0, n_box = 0;
    double ebm = 0.0;  // the largest error bound (AccCtl) of the tetrahedra sent to the chunks
    // groups of 128 consecutive tetrahedra, one per block in turn
#pragma unroll 1
    for (long long first = (long long)blockIdx.x * blockDim.x; first < nb; first += (long long)gridDim.x * blockDim.x) {
    const long long i = first + threadIdx.x;
    __syncthreads();  // the stage is free
    if (i < nb) {
        const long long sg = second ? (long long)list[s0 + i] : s0 + i;  // in the group's numbering
        const int prob = find_simplex(T, sg);
        const ProbEntry& P = T.p[prob];
        const GridDesc& g = P.g;
        const long long s = sg - P.s_off;
        int my_need = 0;
        const VertexRec* v[4];
        // (an index between two problems, or a simplex of another level of an AMR projection)
        const bool mine = s < P.ns && (!levels || (int)levels[s] == prob);
        bool ok = mine;
        for (int k = 0; k < 4 && ok; ++k) {
            const int id = __ldg(P.simplices + s * 4 + k);
            if (id < 0 || id >= P.nv) ok = false;
            v[k] = V + P.v_off + (ok ? id : 0);
        }
        if (!mine) {
        } else if (!ok) {
            atomicOr(&ctr->flags, CDP_FLAG_INDEX);
        } else {
            Tet S;
            const unsigned rc = canon_tet(g, v, S);
            if (rc == 1) {
                n_zero = 1;
            } else if (rc) {
                atomicOr(&ctr->flags, rc);
            } else if (S.lo[0] == S.hi[0] && S.lo[1] == S.hi[1] && S.lo[2] == S.hi[2]) {
                const long long idx =
                    flat_cell(g, S.anchor[0] + S.lo[0], S.anchor[1] + S.lo[1], S.anchor[2] + S.lo[2]);
                if (idx >= 0) atomicAdd(P.out + idx, tet_mass_cells(S));
                n_single = 1;
            } else {
                const long long cells =
                    (long long)(S.hi[0] - S.lo[0] + 1) * (S.hi[1] - S.lo[1] + 1) * (S.hi[2] - S.lo[2] + 1);
                if (cells > max_cells) {
                    list_append(big_list, big_cap, &ctr->big_count, (int)sg);
                } else {
                    tet_setup(S, S.lo, stage[threadIdx.x]);
                    stage[threadIdx.x].prob = prob;
                    const int route = acc_route(stage[threadIdx.x], acc, second, ctr);
                    if (route == 1) {
                        list_append(defer_list, defer_cap, &ctr->defer_count, (int)sg);
                    } else if (route == 2) {
                        list_append(clip_list, clip_cap, &ctr->clip_count, (int)sg);
                    } else {
                        my_need = (int)cells;
                        n_box = 1;
                        float rmax, gn;
                        acc_terms(stage[threadIdx.x], rmax, gn);
                        ebm = fmax(ebm, acc.eps_k_rho * (double)rmax + acc.eps_k_grad * (double)gn);
                    }
                }
            }
        }
        need[i] = my_need;
    }
    __syncthreads();
    {
        constexpr int W = sizeof(TetGeo<R>) / 8;
        const int n = (int)(nb - first < (long long)blockDim.x ? nb - first : (long long)blockDim.x);
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(stage);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(geo + first);
        for (int w = threadIdx.x; w < n * W; w += blockDim.x) dst[w] = src[w];
    }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ebm = fmax(ebm, __shfl_xor_sync(FULL, ebm, o));
    if ((threadIdx.x & 31) == 0 && ebm > 0.0) atomicMax(&ctr->ebmax_bits, (unsigned long long)__double_as_longlong(ebm));
    if (count) {
        n_zero = __reduce_add_sync(FULL, n_zero);
        n_single = __reduce_add_sync(FULL, n_single);
        n_box = __reduce_add_sync(FULL, n_box);
        if ((threadIdx.x & 31) == 0) {
            if (n_zero) atomicAdd(&ctr->n_zero, (unsigned long long)n_zero);
            if (n_single) atomicAdd(&ctr->n_class0, (unsigned long long)n_single);
            if (n_box) atomicAdd(&ctr->n_small, (unsigned long long)n_box);
        }
    }
}

// Between the two passes: the largest |cell mass| of every problem's grid (after the first pass)
// into ctr->mmax_bits[p], and (block 0) the first pass's count of large tetrahedra kept in
// big_first while the list of large tetrahedra is emptied for the second pass.  The cells of all
// the grids are taken in the group's cell numbering.
__global__ void __launch_bounds__(256) k_pass_boundary(const __grid_constant__ ProbTable T, Counters* __restrict__ ctr) {
    // problem by problem: the grid's threads stride over its cells (four independent loads in flight
    // per step), then one maximum per block goes to the problem's word (a thread-level atomic on
    // the few words of a group would serialise)
    __shared__ double wmax[8];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
    for (int p = 0; p < T.n; ++p) {
        const double* const out = T.p[p].out;
        const long long n = (p + 1 < T.n ? T.p[p + 1].c_off : T.ncells) - T.p[p].c_off;
        double m = 0.0;
        long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 1
        for (; c + 3 * stride < n; c += 4 * stride) {
            const double a = out[c], b = out[c + stride], d = out[c + 2 * stride], e = out[c + 3 * stride];
            m = fmax(fmax(m, fmax(fabs(a), fabs(b))), fmax(fabs(d), fabs(e)));
        }
#pragma unroll 1
        for (; c < n; c += stride) m = fmax(m, fabs(out[c]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(FULL, m, o));
        if (lane == 0) wmax[warp] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double bm = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) bm = fmax(bm, wmax[w]);
            if (bm > 0.0) atomicMax(&ctr->mmax_bits[p], (unsigned long long)__double_as_longlong(bm));
        }
        __syncthreads();  // wmax is free
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->big_first = ctr->big_count;
        ctr->big_count = 0u;
        ctr->big_next = 0u;
    }
}

// Whether the tetrahedron B (in the frame of its tile 0) certainly misses tile t of its tiling: the
// tile's box lies more than 1/16 cell outside the plane of one of its facets (then every piece of
// the tile's cells is zero; the margin covers the rounding of the unit normals and coordinates, far
// below it for extents up to CDP_MAX_EXTENT cells).
template <typename R>
__device__ __forceinline__ bool tile_misses(const TetGeo<R>& B, const BigState& b, int t) {
    const int i0 = t % b.nt[0], r = t / b.nt[0], i1 = r % b.nt[1], i2 = r / b.nt[1];
    const int te = b.te;
    const int lo[3] = {i0 * te, i1 * te, i2 * te};
    const int hi[3] = {min(lo[0] + te, b.ext[0]), min(lo[1] + te, b.ext[1]), min(lo[2] + te, b.ext[2])};
    bool miss = false;
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        const int va = f == 0 ? 1 : 0;
        float m = 0.f;  // largest signed distance over the box from the plane of facet f (inward)
        for (int a = 0; a < 3; ++a) {
            const float n = (float)B.n[f][a];
            m += n * ((float)(n > 0.f ? hi[a] : lo[a]) - (float)B.x[va][a]);
        }
        miss = miss || m < -0.0625f;
    }
    return miss;
}

// Warp 0 of a tile round: the first tile at or after bs.tile that the tetrahedron may meet (32
// candidates tested at a time), and its unit: the record of the tetrahedron in the tile's frame (the
// values tet_setup gives for that tile: the frame moves the exact coordinates, cells, box and
// anchor, and the fields rounded from them, one coordinate per lane; the normals, gradient,
// densities and mass do not depend on it), its box, and the item counts of unit_prepare (one
// (edge, axis) pair per lane).  Returns whether a tile was found; lane 0 gets n_cross,
// n_lines and pre_box, and moves bs.tile past the tile.
template <class SH>
__device__ __noinline__ bool tile_setup_warp(SH* sh, int& n_cross, int& n_lines, int& pre_box) {
    using R = typename SH::Real;
    const int lane = threadIdx.x & 31;
    BigState& b = sh->bs;
    const TetGeo<R>& B = sh->big0;
    const int ntiles = b.ntiles;
    int t = b.tile;
#pragma unroll 1
    for (; t < ntiles; t += 32) {
        const int c = t + lane;
        const unsigned live = __ballot_sync(FULL, c < ntiles && !tile_misses(B, b, c));
        if (live) {
            t += __ffs(live) - 1;
            break;
        }
    }
    __syncwarp();  // every lane has read bs
    if (t >= ntiles) {
        if (lane == 0) {
            b.tile = ntiles;
            sh->boff[0] = -1;  // an empty round
        }
        return false;
    }
    const int i0 = t % b.nt[0], r = t / b.nt[0], i1 = r % b.nt[1], i2 = r / b.nt[1];
    const int dT[3] = {i0 * b.te, i1 * b.te, i2 * b.te};
    TetGeo<R>& G = sh->geo[0];
    {
        constexpr int W = sizeof(TetGeo<R>) / 8;
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&B);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&G);
        for (int w = lane; w < W; w += 32) dst[w] = src[w];
    }
    __syncwarp();
    if (lane < 12) {
        const int k = lane / 3, a = lane - 3 * k;
        const int d = pick3(dT[0], dT[1], dT[2], a);
        G.Lt[k][a] = B.Lt[k][a] - ((i64)d << CDP_Q);
        G.x[k][a] = i64_to_real<R>(G.Lt[k][a], CDP_Q);
        G.xl[k][a] = low_part<R>(G.Lt[k][a], G.x[k][a]);
        G.cell[k][a] = B.cell[k][a] - d;
    } else if (lane < 15) {
        const int a = lane - 12;
        const int d = pick3(dT[0], dT[1], dT[2], a);
        G.lo[a] = B.lo[a] - d;
        G.hi[a] = B.hi[a] - d;
        G.anchor[a] = B.anchor[a] + d;
        sh->td[0][a] = min(b.te, pick3(b.ext[0], b.ext[1], b.ext[2], a) - d);
    }
    __syncwarp();
    if (lane == 0) {
        tet_frame_bounds(G);
        sh->boff[0] = 0;
        b.tile = t + 1;
        b.live += 1;
    }
    // crossings of the (edge, axis) pairs with the tile's planes, as running counts
    int run = 0;
    if (lane < 18) {
        const int e = lane / 3, k = lane - 3 * e;
        int a, bb, pp, qq;
        tet_edge(e, a, bb, pp, qq);
        const int ca = G.cell[a][k], cb = G.cell[bb][k];
        const int lo = (ca < cb ? ca : cb) + 1, hi = ca < cb ? cb : ca;
        const int tdk = sh->td[0][k];
        const int c0 = lo > 0 ? lo : 0, c1 = hi < tdk ? hi : tdk;
        run = c1 >= c0 ? c1 - c0 + 1 : 0;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, run, o);
        if (lane >= o) run += u;
    }
    if (lane < 18) sh->xcum[0][lane] = (unsigned short)run;
    n_cross = __shfl_sync(FULL, run, 17);
    int r0[3], n[3];
    unit_line_ranges(G, sh->td[0], r0, n);
    if (lane < 3) {
        sh->lr[0][lane] = pick3(r0[0], r0[1], r0[2], lane);
        sh->lr[0][3 + lane] = pick3(n[0], n[1], n[2], lane);
    }
    n_lines = n[1] * n[2] + n[0] * n[2] + n[0] * n[1];
    pre_box = sh->td[0][0] * sh->td[0][1] * sh->td[0][2];
    return true;
}

// Thread 0 of a block in tiling mode, once the tiles of the current pass are done: switch the FP32
// path from the summing pass to the flush pass (with the tetrahedron's closure scale), or close the
// tetrahedron (FP32: the FP64 remainder to the cell of vertex 0) and take the next one of the list
// (bs.ntiles < 0 when the list is exhausted).
//   The accuracy control (AccCtl) on the taken tetrahedron: first pass, a steep one is deferred;
//   second pass, one whose cancellation bound exceeds the accepted error goes to the clip list.
//   Either way it gets no tile (ntiles = 0) and the next one is taken at the next round.
template <class SH>
__device__ __forceinline__ void big_advance(SH* sh, const ProbTable& T, const VertexRec* V,
                                            const int* big_list, long long big_cap, Counters* ctr,
                                            const BigPass& bp) {
    using R = typename SH::Real;
    constexpr bool fp32 = sizeof(R) == 4;
    BigState& b = sh->bs;
    if (fp32 && b.ntiles > 0) {
        const TetGeo<R>& G = sh->big0;
        const GridDesc& g = T.p[G.prob].g;
        double* const out = T.p[G.prob].out;
        if (b.pass == 0) {
            b.scale = b.s[2] > 0.f ? ((G.mexact_hi - b.s[0]) + (G.mexact_lo - b.s[1])) / b.s[2] : 0.f;
            b.pass = 1;
            b.tile = 0;
            b.live = 0;
            b.s[0] = b.s[1] = b.s[2] = 0.f;
            return;
        }
        // what the rounded pieces of the flush pass still miss of the closed-form mass, in FP64
        const double left =
            (G.mexact - ((double)b.s[0] + (double)b.s[1])) - (double)b.scale * (double)b.s[2];
        const long long idx =
            flat_cell(g, G.anchor[0] + G.cell[0][0], G.anchor[1] + G.cell[0][1], G.anchor[2] + G.cell[0][2]);
        if (idx >= 0) atomicAdd(out + idx, left);
    }
    // the next tetrahedron of the list (complete: every batch was set up before this launch)
    const long long listed = (long long)*(volatile unsigned*)&ctr->big_count;
    const long long nbig = listed < big_cap ? listed : big_cap;
    const long long bi = nbig > 0 ? (long long)atomicAdd(&ctr->big_next, 1u) : 0;
    if (bi >= nbig) {
        b.ntiles = -1;
        return;
    }
    const long long sg = big_list[bi];  // in the group's numbering
    const int prob = find_simplex(T, sg);
    const ProbEntry& P = T.p[prob];
    const long long s = sg - P.s_off;
    const VertexRec* v[4];
    bool ok = true;
    for (int k = 0; k < 4; ++k) {
        const int id = __ldg(P.simplices + s * 4 + k);
        ok = ok && id >= 0 && id < P.nv;
        v[k] = V + P.v_off + (ok ? id : 0);
    }
    // (the set-up kernel listed it after the same checks: no tile when they fail)
    Tet S;
    bool good = ok && canon_tet<1>(P.g, v, S) == 0;
    if (good) {
        tet_setup<R, 1>(S, S.lo, sh->big0);
        sh->big0.prob = prob;
        const int route = acc_route(sh->big0, bp.acc, bp.second != 0, ctr);
        if (route == 1) {
            list_append(bp.defer_list, bp.defer_cap, &ctr->defer_count, (int)sg);
            good = false;
        } else if (route == 2) {
            list_append(bp.clip_list, bp.clip_cap, &ctr->clip_count, (int)sg);
            good = false;
        } else {
            float rmax, gn;
            acc_terms(sh->big0, rmax, gn);
            const double eb = bp.acc.eps_k_rho * (double)rmax + bp.acc.eps_k_grad * (double)gn;
            atomicMax(&ctr->ebmax_bits, (unsigned long long)__double_as_longlong(eb));
        }
    }
    int n = 1;
    b.te = bp.te;
    for (int a = 0; a < 3; ++a) {
        b.ext[a] = good ? S.hi[a] - S.lo[a] + 1 : 0;
        b.nt[a] = (b.ext[a] + b.te - 1) / b.te;
        n *= b.nt[a];
    }
    b.ntiles = n;
    b.pass = fp32 ? 0 : 1;
    b.tile = 0;
    b.live = 0;
    b.scale = 0.f;
    b.s[0] = b.s[1] = b.s[2] = 0.f;
    for (int t = 1; t < SH::kNT; ++t) sh->boff[t] = -1;
}

// The chunks: block b takes chunks b, b + gridDim.x, ... of the batch's geometry records (thread
// t < TB_NT speaks for tetrahedron t of the chunk) and projects them in rounds whose boxes fit
// the block's slots together.
//   SECOND: the batch holds the records of deferred tetrahedra (entries [list_off, list_off + nb) of
//   the deferred list, nb capped by the list's count on the device), each closed on its own.
template <typename R, bool STATS, bool SECOND>
__global__ void __launch_bounds__(TB_THREADS, sizeof(R) == 4 ? 3 : 1)
    k_project_tet(const __grid_constant__ ProbTable T, long long nb, const TetGeo<R>* __restrict__ geo,
                  const int* __restrict__ need_in, UnitCounts* __restrict__ stats, const Counters* __restrict__ ctr,
                  long long list_off, long long list_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int BOX = BoxCap<R>::value;
    TetShared<R>* sh = reinterpret_cast<TetShared<R>*>(smem_raw);
    const int tid = threadIdx.x;
    if (SECOND) {
        const long long listed = (long long)*(volatile const unsigned*)&ctr->defer_count;
        const long long avail = (listed < list_cap ? listed : list_cap) - list_off;
        nb = avail < 0 ? 0 : (avail < nb ? avail : nb);
    }
    for (int e = tid; e < BOX; e += TB_THREADS) sh->box[e] = R(0);
    UnitCounts cnt = {0, 0, 0, 0, 0};   // corner counts (registers)
    UnitCounts xcnt = {0, 0, 0, 0, 0};  // exact-predicate count, updated through a pointer
    UnitCounts* pc = STATS ? &xcnt : nullptr;
    const long long nchunks = (nb + TB_NT - 1) / TB_NT;
#pragma unroll 1
    for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        // ---- the chunk's geometry records (written by k_tet_setup) into shared memory
        const long long first = chunk * TB_NT;
        const long long last = first + TB_NT < nb ? first + TB_NT : nb;
        __syncthreads();  // the previous chunk is done with the records
        {
            constexpr int W = sizeof(TetGeo<R>) / 8;
            static_assert(sizeof(TetGeo<R>) % 8 == 0, "geometry records are copied in 8-byte words");
            const unsigned long long* src = reinterpret_cast<const unsigned long long*>(geo + first);
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(sh->geo);
            const int words = (int)(last - first) * W;
            for (int w = tid; w < words; w += TB_THREADS) dst[w] = __ldg(src + w);
        }
        const int need = (tid < TB_NT && first + tid < nb) ? __ldg(need_in + first + tid) : 0;
        {
            // the block's next chunk of records toward L2 while this one is projected
            const long long nfirst = (chunk + gridDim.x) * TB_NT;
            if (nfirst < nb) {
                const long long nlast = nfirst + TB_NT < nb ? nfirst + TB_NT : nb;
                const long long bytes = (nlast - nfirst) * (long long)sizeof(TetGeo<R>);
                const char* base = reinterpret_cast<const char*>(geo + nfirst);
                if ((long long)tid * 128 < bytes) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + tid * 128));
            }
        }
        __syncthreads();
        int n_cross = 0, n_lines = 0;
        if (need > 0) {
            for (int a = 0; a < 3; ++a) sh->td[tid][a] = sh->geo[tid].hi[a] + 1;
            unit_prepare(sh, tid, n_cross, n_lines);
        }
        bool pending = need > 0;
        // ---- rounds: tetrahedra in chunk order while their boxes fit the block's slots together
#pragma unroll 1
        while (__syncthreads_or(pending)) {
            const int pre_box = block_scan(pending ? need : 0, sh->wsum);
            const bool in = pending && pre_box <= BOX;
            pending = pending && !in;
            if (tid < TB_NT) sh->boff[tid] = in ? pre_box - need : -1;
            round_phases<STATS, false>(sh, in, n_cross, n_lines, cnt, pc);
            round_flush(sh, T, in, pre_box, SECOND ? FLUSH_CLOSE_UNITS : FLUSH_CLOSE_ROUND, 0.f, false, nullptr,
                           nullptr);
        }
    }
    if (STATS) {
        if (cnt.a) atomicAdd(&stats->a, cnt.a);
        if (cnt.b) atomicAdd(&stats->b, cnt.b);
        if (cnt.c) atomicAdd(&stats->c, cnt.c);
        if (cnt.d) atomicAdd(&stats->d, cnt.d);
        if (xcnt.exact) atomicAdd(&stats->exact, xcnt.exact);
    }
}

// The large tetrahedra of the list, taken one at a time by the blocks, each in tiles of TB_TE^3
// cells: one unit per tile (thread 0 speaks for it), the block's rounds one tile each.  FP32 path in
// two passes over a tetrahedron's tiles (the pieces' sums, then the flush with its closure scale).
template <typename R, bool STATS>
__global__ void __launch_bounds__(TB_THREADS, sizeof(R) == 4 ? 3 : 1)
    k_project_big(const __grid_constant__ ProbTable T, const VertexRec* __restrict__ V,
                  const int* __restrict__ big_list, long long big_cap, float* __restrict__ tile_store, int store_tiles,
                  Counters* __restrict__ ctr, UnitCounts* __restrict__ stats, BigPass bp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool fp32 = sizeof(R) == 4;
    using SH = TetSharedBig<R>;
    constexpr int BOX = SH::kBox;
    static_assert(TB_TILE_CELLS <= BOX, "a tile must fit the block's slots");
    SH* sh = reinterpret_cast<SH*>(smem_raw);
    const int tid = threadIdx.x;
    for (int e = tid; e < BOX; e += TB_THREADS) sh->box[e] = R(0);
    if (tid == 0) {
        sh->bs.ntiles = 0;
        sh->bs.tile = 0;
    }
    __syncthreads();  // the state is set before any thread reads it
    UnitCounts cnt = {0, 0, 0, 0, 0};       // corner counts of the counted pass (registers)
    UnitCounts cnt_none = {0, 0, 0, 0, 0};  // (FP32 second pass: not counted)
    UnitCounts xcnt = {0, 0, 0, 0, 0};      // exact-predicate count, updated through a pointer
    UnitCounts* pc = STATS ? &xcnt : nullptr;
    int n_cross = 0, n_lines = 0;
#pragma unroll 1
    for (;;) {
        const bool advance = sh->bs.tile >= sh->bs.ntiles;
        __syncthreads();  // every thread has read the state; the previous round is done
        if (advance) {
            if (tid == 0) big_advance(sh, T, V, big_list, big_cap, ctr, bp);
            __syncthreads();
            if (sh->bs.ntiles < 0) break;
            continue;
        }
        // ---- a tile round: warp 0 finds the next tile the tetrahedron may meet and sets up its unit
        // (thread 0), clipped to the tile; no unit when none is left (an empty round)
        const int mode = sh->bs.pass == 0 ? FLUSH_SUM_ONLY : FLUSH_SCALED;
        bool in = false;
        int pre_box = 0;
        for (int i = tid; i < SH::kRuns; i += TB_THREADS) sh->runs[i] = make_short2(1, 0);
        // the corners are counted in the first pass (FP32: the second may reuse the stored pieces)
        const int pass = sh->bs.pass;
        const bool counted = fp32 ? pass == 0 : true;
        if (tid < 32) {
            const bool found = tile_setup_warp(sh, n_cross, n_lines, pre_box);
            in = found && tid == 0;
            if (STATS && in && counted) atomicAdd(&ctr->n_big_tiles, 1ull);
            // the round's item counts (one unit: every prefix entry is the unit's count)
            static_assert(SH::kScan == 32, "one warp writes the tile round's item counts");
            sh->pre3[0][tid] = found ? 4 : 0;
            sh->pre3[1][tid] = found ? n_cross : 0;
            sh->pre3[2][tid] = found ? n_lines : 0;
        }
        __syncthreads();  // the tile's unit (or its absence) is set up
        // FP32: the first store_tiles tiles of a pass keep their pieces in the block's slots of
        // tile_store between the two passes
        const int j = sh->bs.live - 1;
        const bool stored = fp32 && sh->boff[0] >= 0 && j < store_tiles;
        float* const slot = stored ? tile_store + ((size_t)blockIdx.x * store_tiles + j) * TB_TILE_CELLS : nullptr;
        if (pass == 1 && stored) {
            // the pieces of the first pass, as they were
            const int size = sh->td[0][0] * sh->td[0][1] * sh->td[0][2];
            for (int e = tid; e < size; e += TB_THREADS) sh->box[e] = slot[e];
        } else {
            round_phases<STATS, true>(sh, in, n_cross, n_lines, counted ? cnt : cnt_none, counted ? pc : nullptr);
            // the cells of the tile, column by column, from the run table of the line phase
            const int ncol = sh->boff[0] >= 0 ? sh->td[0][1] * sh->td[0][2] : 0;
            unsigned na = 0;
            for (int c = tid; c < ncol; c += TB_THREADS) na += item_column(sh, c);
            if (STATS && counted) cnt.a += na;
            __syncthreads();
        }
        round_flush(sh, T, in, pre_box, mode, sh->bs.scale, true, sh->bs.s, pass == 0 ? slot : nullptr);
    }
    if (STATS) {
        if (cnt.a) atomicAdd(&stats->a, cnt.a);
        if (cnt.b) atomicAdd(&stats->b, cnt.b);
        if (cnt.c) atomicAdd(&stats->c, cnt.c);
        if (cnt.d) atomicAdd(&stats->d, cnt.d);
        if (xcnt.exact) atomicAdd(&stats->exact, xcnt.exact);
    }
}

// three FP32 blocks per SM, for both kernels: 228 KB of shared memory per SM, 1 KB of it reserved
// per block
static_assert(3 * (sizeof(TetShared<float>) + 1024) <= 228 * 1024, "three FP32 chunk blocks per SM");
static_assert(3 * (sizeof(TetSharedBig<float>) + 1024) <= 228 * 1024, "three FP32 tile blocks per SM");

template <typename R>
static size_t tet_shared_bytes() {
    return sizeof(TetShared<R>);
}
template <typename R>
static size_t big_shared_bytes() {
    return sizeof(TetSharedBig<R>);
}

template <typename R, bool STATS>
static cudaError_t configure_one() {
    cudaError_t e = cudaFuncSetAttribute(k_project_tet<R, STATS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tet_shared_bytes<R>());
    if (e) return e;
    e = cudaFuncSetAttribute(k_project_tet<R, STATS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tet_shared_bytes<R>());
    if (e) return e;
    return cudaFuncSetAttribute(k_project_big<R, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)big_shared_bytes<R>());
}

cudaError_t configure_tet() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_tet_setup<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(128 * sizeof(TetGeo<float>)))) ||
        (e = cudaFuncSetAttribute(k_tet_setup<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(128 * sizeof(TetGeo<double>)))))
        return e;
    if ((e = configure_one<float, false>()) || (e = configure_one<float, true>()) ||
        (e = configure_one<double, false>()))
        return e;
    return configure_one<double, true>();
}

int resident_blocks_tet(int fp32) {
    int n = 0;
    cudaError_t e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_project_tet<float, false, false>,
                                                                         TB_THREADS, tet_shared_bytes<float>())
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_project_tet<double, false, false>,
                                                                         TB_THREADS, tet_shared_bytes<double>());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

size_t tet_geo_bytes(int fp32) { return fp32 ? sizeof(TetGeo<float>) : sizeof(TetGeo<double>); }

size_t tet_tile_cells() { return TB_TILE_CELLS; }

int tet_tile_edge() { return TB_TE; }

int tet_max_cells() { return TB_MAX_CELLS; }

int tet_box_slots(int fp32) { return fp32 ? BoxCap<float>::value : BoxCap<double>::value; }

template <typename R>
static cudaError_t launch_tet_r(const LaunchArgs& L, cudaStream_t st, cudaEvent_t after_setup, cudaEvent_t mid) {
    const long long batch = L.geo_cap > 0 ? L.geo_cap : 1;
    const long long cap = (long long)L.num_sms * L.small_blocks_per_sm;
    AccCtl acc = acc_ctl(sizeof(R) == 4);
    if (!L.accuracy) acc.defer_ratio = 3.0e38f;  // nothing is deferred
    TetGeo<R>* G = reinterpret_cast<TetGeo<R>*>(L.geo);
    const size_t stage = 128 * sizeof(TetGeo<R>);
    // the size-class threshold (at most the block's box slots) and the tile edge (at most TB_TE)
    const int max_cells = L.max_cells > 0 && L.max_cells <= BoxCap<R>::value ? L.max_cells : TB_MAX_CELLS;
    const int te = L.tile_edge >= 4 && L.tile_edge <= TB_TE ? L.tile_edge : TB_TE;
    // the main kernel over a batch of nb records (second pass: nb capped on the device)
    auto chunks = [&](long long nb, int second, long long off) {
        long long blocks = (nb + TB_NT - 1) / TB_NT;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        const unsigned b = (unsigned)blocks;
        const size_t sm = tet_shared_bytes<R>();
        if (second) {
            if (L.stats)
                k_project_tet<R, true, true><<<b, TB_THREADS, sm, st>>>(L.T, nb, G, L.need, L.stats, L.ctr, off,
                                                                       L.defer_cap);
            else
                k_project_tet<R, false, true><<<b, TB_THREADS, sm, st>>>(L.T, nb, G, L.need, nullptr, L.ctr, off,
                                                                        L.defer_cap);
        } else {
            if (L.stats)
                k_project_tet<R, true, false><<<b, TB_THREADS, sm, st>>>(L.T, nb, G, L.need, L.stats, L.ctr, 0, 0);
            else
                k_project_tet<R, false, false><<<b, TB_THREADS, sm, st>>>(L.T, nb, G, L.need, nullptr, L.ctr, 0, 0);
        }
    };
    // the large tetrahedra of the list (their number is read on the device; a block that finds the
    // list exhausted exits at once): one block per resident slot.  FP32: each block keeps the pieces
    // of up to tile_store_per_block tiles between the two passes over a tetrahedron's tiles.
    const long long big_blocks = (long long)L.num_sms * (L.resident_per_sm > 0 ? L.resident_per_sm : 1);
    const int store_tiles = sizeof(R) == 4 && L.tile_store &&
                                    L.tile_store_cap >= (size_t)big_blocks * L.tile_store_per_block * TB_TILE_CELLS
                                ? L.tile_store_per_block
                                : 0;
    auto big = [&](int second) {
        const BigPass bp = {acc, second, te, L.defer_list, L.defer_cap, L.clip_list, L.clip_cap};
        if (L.stats)
            k_project_big<R, true><<<(unsigned)big_blocks, TB_THREADS, big_shared_bytes<R>(), st>>>(
                L.T, L.verts, L.big_list, L.big_cap, L.tile_store, store_tiles, L.ctr, L.stats + 1, bp);
        else
            k_project_big<R, false><<<(unsigned)big_blocks, TB_THREADS, big_shared_bytes<R>(), st>>>(
                L.T, L.verts, L.big_list, L.big_cap, L.tile_store, store_tiles, L.ctr, nullptr, bp);
    };
    // first pass: every tetrahedron, batch by batch; steep ones are deferred
    const long long ns = L.T.ns;  // (the group's numbering, gaps between problems included)
    for (long long s0 = 0; s0 < ns; s0 += batch) {
        const long long nb = ns - s0 < batch ? ns - s0 : batch;
        k_tet_setup<R><<<(unsigned)((nb + 127) / 128), 128, stage, st>>>(
            L.T, s0, nb, L.verts, L.ctr, G, L.need, L.big_list, L.big_cap, L.stats != nullptr, max_cells, L.levels,
            nullptr, acc, L.defer_list, L.defer_cap, L.clip_list, L.clip_cap);
        if (after_setup && s0 == 0) cudaEventRecord(after_setup, st);
        chunks(nb, 0, 0);
    }
    if (mid) cudaEventRecord(mid, st);
    big(0);
    if (L.ev_acc) cudaEventRecord(L.ev_acc, st);
    if (!L.accuracy) return cudaGetLastError();
    cudaError_t e = launch_pass_boundary(L, st);
    if (e != cudaSuccess) return e;
    // second pass: the deferred tetrahedra (at most min(ns, defer_cap)), batch by batch of the
    // geometry buffer, then the deferred large ones, then those sent to clipping
    const long long most = ns < L.defer_cap ? ns : L.defer_cap;
    for (long long s0 = 0; s0 < most; s0 += batch) {
        long long blocks = (batch + 127) / 128;
        if (blocks > (long long)L.num_sms * 16) blocks = (long long)L.num_sms * 16;
        k_tet_setup<R><<<(unsigned)blocks, 128, stage, st>>>(L.T, s0, batch, L.verts, L.ctr, G, L.need, L.big_list,
                                                            L.big_cap, L.stats != nullptr, max_cells, nullptr,
                                                            L.defer_list, acc, L.defer_list, L.defer_cap, L.clip_list,
                                                            L.clip_cap);
        chunks(batch, 1, s0);
    }
    big(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_clip(L, sizeof(R) == 4, st);
}

// the largest |cell mass| after the first pass, and the list of large tetrahedra emptied
cudaError_t launch_pass_boundary(const LaunchArgs& L, cudaStream_t st) {
    long long blocks = (L.T.ncells + 255) / 256;
    if (blocks > (long long)L.num_sms * 8) blocks = (long long)L.num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_pass_boundary<<<(unsigned)blocks, 256, 0, st>>>(L.T, L.ctr);
    return cudaGetLastError();
}

cudaError_t launch_tet(const LaunchArgs& L, int fp32, cudaStream_t st, cudaEvent_t after_setup, cudaEvent_t mid) {
    return fp32 ? launch_tet_r<float>(L, st, after_setup, mid) : launch_tet_r<double>(L, st, after_setup, mid);
}

}  // namespace cdp
