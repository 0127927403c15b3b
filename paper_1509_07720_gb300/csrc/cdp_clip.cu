// Accuracy control (Sect. 3.4): the projection of the simplices whose Franklin sum cannot be trusted
// in the arithmetic at hand.
//
// Each (vertex, edge, facet) contribution of eqs. contrib, E0, E1 is a product of offsets of the
// order of a cell and, for its first-order part, of the density gradient.  Summed over the corners
// of a piece they cancel down to the piece's mass, so the rounding error of a piece is a few units in
// the last place of the LARGEST contribution (eq. accuracy: eps_P = 2^(e_max - S + W)), not of the
// piece.  In a nearly flat simplex with unequal vertex densities (or a steep density contrast) the
// gradient, and with it e_max, is orders of magnitude above the simplex's own density, and the
// pieces lose all their digits.  Sect. 3.4 prescribes comparing e_max with the result and, where
// accuracy is lacking, re-projecting the simplices concerned with higher precision or with a
// different algorithm whose degenerate configurations differ.  This file is that different
// algorithm:
//
//   for every cell of the simplex's bounding box, the polytope P = simplex intersect cell is bounded
//   by the simplex's facets clipped to the cell and by the cell's faces clipped to the simplex
//   (Sutherland-Hodgman clipping of each face polygon by the other body's half-spaces, FP64).  P is
//   convex, hence star-shaped from any of its vertices v0, and the integral of the linear density is
//   the sum over the fan tetrahedra (v0, f0, f_i, f_{i+1}) of every face polygon of |det| / 6 times
//   the mean density at their four corners (exact for a linear function).  Every term is positive,
//   so nothing cancels: the error of a piece is a few ulps of the density times the cell volume,
//   whatever the simplex's shape.  (2D: the triangle clipped by the cell's four half-planes, fanned
//   from one vertex of the polygon.)
//
// The test that sends a simplex here (its bound on e_max against the grid's largest cell) is made by
// the projection kernels; they append the simplex to a list.  Tetrahedra: k_clip_setup3 sets up one
// record per listed tetrahedron, and k_project_clip3 takes each with one warp, classifying the cells
// of its bounding box and clipping the crossed ones 32 at a time.  Triangles: k_project_clip2 takes
// each with one block, its threads going over the cells of the bounding box.
#include <cuda_runtime.h>

#include "cdp_mesh.cuh"
#include "cdp_project.h"

namespace cdp {

namespace {

constexpr int CLIP_THREADS = 128;
constexpr int MAXP = 12;  // a triangle cut by 6 planes has at most 9 vertices, a square cut by 4 at most 8

// Clips the convex polygon p[0..n) by the half-space  c . x + c0 >= 0  into q; returns q's size.
// Points on the plane are kept; crossing points are interpolated on the edge (all three components,
// so a third one that is not a coordinate is interpolated too).
template <typename R>
__device__ int clip_by(const R (*p)[3], int n, R (*q)[3], const R c[3], R c0) {
    int m = 0;
    if (n == 0) return 0;
    R dprev = c[0] * p[n - 1][0] + c[1] * p[n - 1][1] + c[2] * p[n - 1][2] + c0;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const int ip = i == 0 ? n - 1 : i - 1;
        const R d = c[0] * p[i][0] + c[1] * p[i][1] + c[2] * p[i][2] + c0;
        if ((d >= R(0)) != (dprev >= R(0)) && m < MAXP) {
            // the edge (ip, i) crosses the plane strictly inside: t from the inside end
            const R t = dprev / (dprev - d);
            q[m][0] = p[ip][0] + t * (p[i][0] - p[ip][0]);
            q[m][1] = p[ip][1] + t * (p[i][1] - p[ip][1]);
            q[m][2] = p[ip][2] + t * (p[i][2] - p[ip][2]);
            ++m;
        }
        if (d >= R(0) && m < MAXP) {
            q[m][0] = p[i][0];
            q[m][1] = p[i][1];
            q[m][2] = p[i][2];
            ++m;
        }
        dprev = d;
    }
    return m;
}

// A simplex in the frame of one cell, read by every thread of the block.
struct ClipTet {
    double x[4][3];   // vertex coordinates relative to the anchor cell (grid units, exact)
    double n[4][3];   // unit inward normal of the facet opposite each vertex
    double nx[4];     // n_f . x of a vertex of facet f
    double hw[4];     // (|n_0| + |n_1| + |n_2|) / 2: half the spread of n_f . x over a unit cell
    double g[3];      // density gradient (per cell)
    double c[3];      // centroid, and the density there
    double rhoc;
    double mexact;    // |V| mean(rho), FP64 closed form (the FP32 closure)
    int lo[3], hi[3]; // bounding box (cells, relative to the anchor)
    int anchor[3];
    int cell0[3];     // absolute cell of vertex 0
    int prob;         // the problem of the group
    int ok;
};

struct ClipTri {
    double x[3][2];   // vertex coordinates relative to the anchor cell (grid units, exact)
    double rho[3];
    int lo[2], hi[2]; // bounding box (cells, relative to the anchor)
    int anchor[2];
    int ok;
};

// the simplex in the frame of one cell: vertex offsets from the cell's lower corner, facet normals,
// and the density as rc + g . x in that frame (taken in FP64, then rounded to R)
template <typename R>
struct CellFrame {
    R x[4][3];
    R n[4][3];
    R g[3];
    R rc;
};

template <typename R>
__device__ __forceinline__ R rho_at(const CellFrame<R>& F, const R x[3]) {
    return F.rc + F.g[0] * x[0] + F.g[1] * x[1] + F.g[2] * x[2];
}

template <typename R>
__device__ __forceinline__ R abs_r(R v) { return v < R(0) ? -v : v; }

// |det(b - a, c - a, d - a)| / 6
template <typename R>
__device__ __forceinline__ R tet_vol(const R a[3], const R b[3], const R c[3], const R d[3]) {
    const R u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
    const R v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
    const R w0 = d[0] - a[0], w1 = d[1] - a[1], w2 = d[2] - a[2];
    return abs_r(u0 * (v1 * w2 - v2 * w1) - u1 * (v0 * w2 - v2 * w0) + u2 * (v0 * w1 - v1 * w0)) * R(1.0 / 6.0);
}

// The unit cell whose lower corner is o (relative to the anchor) against each facet plane of the
// tetrahedron, in FP64: entirely outside one of them (0: no piece), inside all (1: the whole cell,
// whose integral, the density at its centre, goes to *whole), or crossed (2).  Over the corners of
// the unit cell the signed distance n . x - n . x_f ranges over its value at the centre +- hw.
__device__ __forceinline__ int clip_classify(const ClipTet& T, const double o[3], double* whole) {
    bool inside = true;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const double dc = T.n[f][0] * (o[0] + 0.5) + T.n[f][1] * (o[1] + 0.5) + T.n[f][2] * (o[2] + 0.5) - T.nx[f];
        if (dc + T.hw[f] < 0.0) return 0;
        inside = inside && dc - T.hw[f] >= 0.0;
    }
    if (!inside) return 2;
    *whole = T.rhoc + T.g[0] * ((o[0] + 0.5) - T.c[0]) + T.g[1] * ((o[1] + 0.5) - T.c[1]) +
             T.g[2] * ((o[2] + 0.5) - T.c[2]);
    return 1;
}

// Integral of rho over (tetrahedron intersect the unit cell whose lower corner is o, relative to the
// anchor), for a cell the facets cross (clip_classify 2), in arithmetic R.  The simplex is first
// taken into the cell's frame in FP64 (exact offsets, then rounded once), so that every coordinate
// the clipping sees is within a few cells of 0.
template <typename R>
__device__ R clip_cell_3d(const ClipTet& T, const double o[3]) {
    CellFrame<R> F;
#pragma unroll 1
    for (int k = 0; k < 4; ++k)
        for (int a = 0; a < 3; ++a) {
            F.x[k][a] = (R)(T.x[k][a] - o[a]);
            F.n[k][a] = (R)T.n[k][a];
        }
    for (int a = 0; a < 3; ++a) F.g[a] = (R)T.g[a];
    F.rc = (R)(T.rhoc + T.g[0] * (o[0] - T.c[0]) + T.g[1] * (o[1] - T.c[1]) + T.g[2] * (o[2] - T.c[2]));
    R bufa[MAXP][3], bufb[MAXP][3];
    R v0[3] = {R(0), R(0), R(0)};
    R r0 = R(0);
    bool have_v0 = false;
    R sum = R(0);
    // the faces of the polytope: 4 clipped facets, then 6 clipped cell faces
#pragma unroll 1
    for (int face = 0; face < 10; ++face) {
        int n;
        if (face < 4) {
            // facet `face` (opposite vertex `face`), clipped by the cell's 6 half-spaces
            n = 0;
#pragma unroll 1
            for (int k = 0; k < 4; ++k) {
                if (k == face) continue;
                bufa[n][0] = F.x[k][0];
                bufa[n][1] = F.x[k][1];
                bufa[n][2] = F.x[k][2];
                ++n;
            }
#pragma unroll 1
            for (int pl = 0; pl < 6 && n > 0; ++pl) {
                const int a = pl >> 1;
                const R sg = (pl & 1) ? R(-1) : R(1);  // x_a >= 0, then 1 - x_a >= 0
                const R c[3] = {a == 0 ? sg : R(0), a == 1 ? sg : R(0), a == 2 ? sg : R(0)};
                n = clip_by<R>(bufa, n, bufb, c, (pl & 1) ? R(1) : R(0));
#pragma unroll 1
                for (int i = 0; i < n; ++i) {
                    bufa[i][0] = bufb[i][0];
                    bufa[i][1] = bufb[i][1];
                    bufa[i][2] = bufb[i][2];
                }
            }
        } else {
            // cell face x_a = s clipped by the tetrahedron's 4 half-spaces; a face lying in a facet's
            // plane is that facet's polygon already (counted above) and is skipped
            const int a = (face - 4) >> 1, sd = (face - 4) & 1;
            const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
            const R sq[4][2] = {{R(0), R(0)}, {R(1), R(0)}, {R(1), R(1)}, {R(0), R(1)}};
            n = 4;
#pragma unroll 1
            for (int i = 0; i < 4; ++i) {
                bufa[i][a] = R(sd);
                bufa[i][b] = sq[i][0];
                bufa[i][cc] = sq[i][1];
            }
#pragma unroll 1
            for (int f = 0; f < 4 && n > 0; ++f) {
                const int va = f == 0 ? 1 : 0;
                const R* nf = F.n[f];
                const R c0 = -(nf[0] * F.x[va][0] + nf[1] * F.x[va][1] + nf[2] * F.x[va][2]);
                bool coplanar = true;
#pragma unroll 1
                for (int i = 0; i < n; ++i)
                    coplanar = coplanar && nf[0] * bufa[i][0] + nf[1] * bufa[i][1] + nf[2] * bufa[i][2] + c0 == R(0);
                if (coplanar) {
                    n = 0;
                    break;
                }
                n = clip_by<R>(bufa, n, bufb, nf, c0);
#pragma unroll 1
                for (int i = 0; i < n; ++i) {
                    bufa[i][0] = bufb[i][0];
                    bufa[i][1] = bufb[i][1];
                    bufa[i][2] = bufb[i][2];
                }
            }
        }
        if (n < 3) continue;
        if (!have_v0) {
            // the apex of every fan: a vertex of the polytope (its own faces add nothing)
            v0[0] = bufa[0][0];
            v0[1] = bufa[0][1];
            v0[2] = bufa[0][2];
            r0 = rho_at(F, v0);
            have_v0 = true;
        }
        const R rf = rho_at(F, bufa[0]);
        R rprev = rho_at(F, bufa[1]);
#pragma unroll 1
        for (int i = 1; i + 1 < n; ++i) {
            const R rnext = rho_at(F, bufa[i + 1]);
            sum += tet_vol<R>(v0, bufa[0], bufa[i], bufa[i + 1]) * (R(0.25) * ((r0 + rf) + (rprev + rnext)));
            rprev = rnext;
        }
    }
    return sum;
}

// 2D: the triangle clipped by the cell's four half-planes, fanned from the polygon's first vertex;
// the density is interpolated along the clipped edges (x, y, rho carried together).
template <typename R>
__device__ R clip_cell_2d(const ClipTri& T, const double o[2]) {
    R pa[MAXP][3], pb[MAXP][3];
    for (int k = 0; k < 3; ++k) {
        pa[k][0] = (R)(T.x[k][0] - o[0]);
        pa[k][1] = (R)(T.x[k][1] - o[1]);
        pa[k][2] = (R)T.rho[k];
    }
    int n = 3;
#pragma unroll 1
    for (int pl = 0; pl < 4 && n > 0; ++pl) {
        const int a = pl >> 1;
        const R sg = (pl & 1) ? R(-1) : R(1);
        const R c[3] = {a == 0 ? sg : R(0), a == 1 ? sg : R(0), R(0)};
        n = clip_by<R>(pa, n, pb, c, (pl & 1) ? R(1) : R(0));
        for (int i = 0; i < n; ++i) {
            pa[i][0] = pb[i][0];
            pa[i][1] = pb[i][1];
            pa[i][2] = pb[i][2];
        }
    }
    R sum = R(0);
    for (int i = 1; i + 1 < n; ++i) {
        const R u0 = pa[i][0] - pa[0][0], u1 = pa[i][1] - pa[0][1];
        const R w0 = pa[i + 1][0] - pa[0][0], w1 = pa[i + 1][1] - pa[0][1];
        sum += abs_r(u0 * w1 - u1 * w0) * R(0.5) * ((pa[0][2] + pa[i][2] + pa[i + 1][2]) * R(1.0 / 3.0));
    }
    return sum;
}

}  // namespace

// 2D: the listed triangles (list[0, min(*count, cap))), one per block in turn; every cell of the
// bounding box by the block's threads, in arithmetic R.  R = float (FP32-mixed path): the simplex's pieces
// are summed over the block and its FP64 closed-form mass minus that sum (a few FP32 ulps of the
// pieces) goes to the cell of its vertex 0, so the total mass stays exact to FP64 rounding.  The
// simplices passed the vertex-index and canonicalisation checks when they were listed.
// One thread per listed tetrahedron of entries [e0, e0 + cap) of the clip list (the list's count read
// on the device): canonicalise and set up in FP64, into recs[e - e0].  (The set-up is long FP64
// and 128-bit integer work; one thread each keeps the SMs busy with it.)
__global__ void __launch_bounds__(128) k_clip_setup3(const __grid_constant__ ProbTable T, const VertexRec* __restrict__ V,
                                                      const int* __restrict__ list, const unsigned* count,
                                                      long long list_cap, long long e0, long long cap,
                                                      ClipTet* __restrict__ recs) {
    const long long listed = (long long)*(volatile const unsigned*)count;
    const long long n = (listed < list_cap ? listed : list_cap) - e0;
    const long long m = n < cap ? n : cap;
#pragma unroll 1
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        ClipTet& st = recs[i];
        const long long sg = list[e0 + i];  // in the group's numbering
        const int prob = find_simplex(T, sg);
        const ProbEntry& P = T.p[prob];
        const long long s = sg - P.s_off;
        const VertexRec* v[4];
        bool ok = true;
        for (int k = 0; k < 4; ++k) {
            const int id = P.simplices[s * 4 + k];
            ok = ok && id >= 0 && id < P.nv;
            v[k] = V + P.v_off + (ok ? id : 0);
        }
        Tet S;
        st.ok = ok && canon_tet<2>(P.g, v, S) == 0;
        st.prob = prob;
        if (!st.ok) continue;
        TetGeo<double> G;
        tet_setup<double, 2>(S, S.lo, G);
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a) {
                st.x[k][a] = G.x[k][a] + (double)S.lo[a];
                st.n[k][a] = G.n[k][a];
            }
        for (int f = 0; f < 4; ++f) {
            const int va = f == 0 ? 1 : 0;
            st.nx[f] = st.n[f][0] * st.x[va][0] + st.n[f][1] * st.x[va][1] + st.n[f][2] * st.x[va][2];
            st.hw[f] = 0.5 * (fabs(st.n[f][0]) + fabs(st.n[f][1]) + fabs(st.n[f][2]));
        }
        for (int a = 0; a < 3; ++a) {
            st.g[a] = G.g[a];
            st.c[a] = G.c[a] + (double)S.lo[a];
            st.lo[a] = S.lo[a];
            st.hi[a] = S.hi[a];
            st.anchor[a] = S.anchor[a];
            st.cell0[a] = S.anchor[a] + S.cell[0][a];
        }
        st.rhoc = G.rhoc;
        st.mexact = G.mexact;
    }
}

// One warp per record of k_clip_setup3 (records [0, min(n, cap)), n the clip list's count less e0):
// the cells of the bounding box are classified by the warp's lanes 32 at a time (outside, inside:
// the closed form at once, crossed); the crossed ones are queued in shared memory and clipped 32 at a
// time, one per lane, in arithmetic R.  R = float: the tetrahedron's pieces are summed over the warp
// and its FP64 closed-form mass minus that sum goes to the cell of its vertex 0.
template <typename R>
__global__ void __launch_bounds__(CLIP_THREADS) k_project_clip3(const __grid_constant__ ProbTable T,
                                                                const ClipTet* __restrict__ recs, const unsigned* count,
                                                                long long list_cap, long long e0, long long cap) {
    constexpr bool closure = sizeof(R) == 4;
    __shared__ long long crossed[CLIP_THREADS / 32][64];  // crossed cells awaiting their clipping, per warp
    const long long listed = (long long)*(volatile const unsigned*)count;
    const long long n0 = (listed < list_cap ? listed : list_cap) - e0;
    const long long n = n0 < cap ? n0 : cap;
    const int lane = threadIdx.x & 31;
    long long* const q = crossed[threadIdx.x >> 5];
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
#pragma unroll 1
    for (long long e = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < n; e += warps) {
        const ClipTet& st = recs[e];
        if (!st.ok) continue;
        const GridDesc& g = T.p[st.prob].g;
        double* const out = T.p[st.prob].out;
        const long long ex = st.hi[0] - st.lo[0] + 1, ey = st.hi[1] - st.lo[1] + 1, ez = st.hi[2] - st.lo[2] + 1;
        const long long ncell = ex * ey * ez;
        // cell c of the box: (i, j, k) = (c mod ex, (c / ex) mod ey, c / (ex ey)); its lower corner
        auto corner = [&](long long c, double o[3], long long& idx) {
            const long long r = c / ex;
            const int i = (int)(c - r * ex), j = (int)(r % ey), k = (int)(r / ey);
            o[0] = (double)(st.lo[0] + i);
            o[1] = (double)(st.lo[1] + j);
            o[2] = (double)(st.lo[2] + k);
            idx = flat_cell(g, st.anchor[0] + st.lo[0] + i, st.anchor[1] + st.lo[1] + j, st.anchor[2] + st.lo[2] + k);
        };
        double mine = 0.0;
        int nq = 0;  // queued crossed cells (the same in every lane)
#pragma unroll 1
        for (long long base = 0; base < ncell; base += 32) {
            const long long c = base + lane;
            int cls = 0;
            if (c < ncell) {
                double o[3], whole = 0.0;
                long long idx;
                corner(c, o, idx);
                cls = clip_classify(st, o, &whole);
                if (cls == 1) {
                    const R m = (R)whole;
                    mine += (double)m;
                    if (idx >= 0) atomicAdd(out + idx, (double)m);
                }
            }
            const unsigned cm = __ballot_sync(0xffffffffu, cls == 2);
            if (cls == 2) q[nq + __popc(cm & ((1u << lane) - 1u))] = c;
            nq += __popc(cm);
            __syncwarp();
            // a full batch (or, after the last cells, what is left): one crossed cell per lane
            const bool last = base + 32 >= ncell;
            if (nq >= 32 || (last && nq > 0)) {
                if (lane < nq) {
                    double o[3];
                    long long idx;
                    corner(q[lane], o, idx);
                    const R m = clip_cell_3d<R>(st, o);
                    if (m != R(0)) {
                        mine += (double)m;
                        if (idx >= 0) atomicAdd(out + idx, (double)m);
                    }
                }
                __syncwarp();
                const int left = nq > 32 ? nq - 32 : 0;
                if (lane < left) q[lane] = q[32 + lane];
                nq = left;
                __syncwarp();
                if (last && nq > 0) {  // (at most 31 after a full batch of the last cells)
                    if (lane < nq) {
                        double o[3];
                        long long idx;
                        corner(q[lane], o, idx);
                        const R m = clip_cell_3d<R>(st, o);
                        if (m != R(0)) {
                            mine += (double)m;
                            if (idx >= 0) atomicAdd(out + idx, (double)m);
                        }
                    }
                    nq = 0;
                    __syncwarp();
                }
            }
        }
        if (closure) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
            if (lane == 0) {
                const long long idx = flat_cell(g, st.cell0[0], st.cell0[1], st.cell0[2]);
                if (idx >= 0) atomicAdd(out + idx, st.mexact - mine);
            }
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(CLIP_THREADS) k_project_clip2(const __grid_constant__ ProbTable T,
                                                               const VertexRec* __restrict__ V,
                                                               const int* __restrict__ list, const unsigned* count,
                                                               long long cap) {
    constexpr bool closure = sizeof(R) == 4;
    __shared__ ClipTri s2;
    __shared__ double mexact;
    __shared__ int cell0[3];
    __shared__ int prob;
    __shared__ double wsum[CLIP_THREADS / 32];
    const long long listed = (long long)*(volatile const unsigned*)count;
    const long long n = listed < cap ? listed : cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
    for (long long e = blockIdx.x; e < n; e += gridDim.x) {
        __syncthreads();  // the previous simplex is done
        if (threadIdx.x == 0) {
            const long long sg = list[e];  // in the group's numbering
            prob = find_simplex(T, sg);
            const ProbEntry& P = T.p[prob];
            const GridDesc& g = P.g;
            const long long s = sg - P.s_off;
            const VertexRec* v[3];
            bool ok = true;
            for (int k = 0; k < 3; ++k) {
                const int id = P.simplices[s * 3 + k];
                ok = ok && id >= 0 && id < P.nv;
                v[k] = V + P.v_off + (ok ? id : 0);
            }
            {
                Tri S;
                s2.ok = ok && canon_tri(g, v, S) == 0;
                if (s2.ok) {
                    for (int k = 0; k < 3; ++k) {
                        for (int a = 0; a < 2; ++a) s2.x[k][a] = i64_to_real<double>(S.L[k][a], CDP_Q);
                        s2.rho[k] = S.rho[k];
                    }
                    for (int a = 0; a < 2; ++a) {
                        s2.lo[a] = S.lo[a];
                        s2.hi[a] = S.hi[a];
                        s2.anchor[a] = S.anchor[a];
                        cell0[a] = S.anchor[a] + S.cell[0][a];
                    }
                    cell0[2] = 0;
                    mexact = tri_mass_cells(S);
                }
            }
        }
        __syncthreads();
        if (!s2.ok) continue;
        const GridDesc& g = T.p[prob].g;
        double* const out = T.p[prob].out;
        const int* lo = s2.lo;
        const int* hi = s2.hi;
        const int* an = s2.anchor;
        const long long ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1;
        const long long ncell = ex * ey;
        double mine = 0.0;  // this thread's pieces (for the closure)
#pragma unroll 1
        for (long long c = threadIdx.x; c < ncell; c += blockDim.x) {
            const long long r = c / ex;
            const int i = (int)(c - r * ex), j = (int)r;
            const double o[2] = {(double)(lo[0] + i), (double)(lo[1] + j)};
            const R m = clip_cell_2d<R>(s2, o);
            if (m == R(0)) continue;
            mine += (double)m;
            const long long idx = flat_cell(g, an[0] + lo[0] + i, an[1] + lo[1] + j, 0);
            if (idx >= 0) atomicAdd(out + idx, (double)m);
        }
        if (closure) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
            if (lane == 0) wsum[warp] = mine;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < CLIP_THREADS / 32; ++w) tot += wsum[w];
                const long long idx = flat_cell(g, cell0[0], cell0[1], cell0[2]);
                if (idx >= 0) atomicAdd(out + idx, mexact - tot);
            }
        }
    }
}

cudaError_t launch_clip(const LaunchArgs& L, int fp32, cudaStream_t st) {
    if (!L.clip_list || !L.ctr) return cudaSuccess;
    const unsigned* cnt = &L.ctr->clip_count;
    if (L.T.dim == 3) {
        // records in the geometry buffer (free once the second pass is done), batch by batch; the
        // clip list holds at most min(ns, clip_cap) entries, its count read on the device
        const long long cap = (long long)(L.geo_bytes / sizeof(ClipTet));
        if (cap < 1) return cudaErrorInvalidValue;
        ClipTet* recs = reinterpret_cast<ClipTet*>(L.geo);
        const long long most = L.T.ns < L.clip_cap ? L.T.ns : L.clip_cap;
        for (long long e0 = 0; e0 < most; e0 += cap) {
            long long sb = (cap + 127) / 128;
            if (sb > (long long)L.num_sms * 16) sb = (long long)L.num_sms * 16;
            k_clip_setup3<<<(unsigned)sb, 128, 0, st>>>(L.T, L.verts, L.clip_list, cnt, L.clip_cap, e0, cap, recs);
            const unsigned blocks = (unsigned)(L.num_sms * 8);
            if (fp32)
                k_project_clip3<float><<<blocks, CLIP_THREADS, 0, st>>>(L.T, recs, cnt, L.clip_cap, e0, cap);
            else
                k_project_clip3<double><<<blocks, CLIP_THREADS, 0, st>>>(L.T, recs, cnt, L.clip_cap, e0, cap);
        }
    } else {
        const unsigned blocks = (unsigned)(L.num_sms * 4);
        if (fp32)
            k_project_clip2<float><<<blocks, CLIP_THREADS, 0, st>>>(L.T, L.verts, L.clip_list, cnt, L.clip_cap);
        else
            k_project_clip2<double><<<blocks, CLIP_THREADS, 0, st>>>(L.T, L.verts, L.clip_list, cnt, L.clip_cap);
    }
    return cudaGetLastError();
}

}  // namespace cdp
