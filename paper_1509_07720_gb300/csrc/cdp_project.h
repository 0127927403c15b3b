// Internal interface between the C-ABI layer (cdp_api.cu) and the projection kernels.
#pragma once

#include <cuda_runtime.h>

#include "cdp_mesh.cuh"

namespace cdp {

constexpr int CDP_WBLOCK = 128;   // threads per block of the projection kernel (4 warps)
constexpr int CDP_CHUNK = 32;     // simplices per warp chunk, at most (one per lane during set-up)
constexpr int CDP_LOG_WTBL = 9;   // per-warp piece table: 2^9 entries
constexpr int CDP_WTBL = 1 << CDP_LOG_WTBL;
constexpr int CDP_QCAP = 512;     // per-warp queue of (corner, cell) records (power of two)

// Problems projected together (cdp_project_batched, cdp_step_batched; a single projection is a
// group of one): up to CDP_GROUP problems of one dimension per launch.  The kernels take the table
// by value (a __grid_constant__ parameter, read in place) and map a global vertex, simplex or cell
// index to its problem by a binary search over the offsets.
constexpr int CDP_GROUP = 64;

struct ProbEntry {
    GridDesc g;
    const int* simplices;  // caller's (dim + 1) indices per simplex, local to the problem
    double* out;           // the problem's grid
    const double* pos[3];  // caller's coordinates
    const double* rho;
    long long nv, ns;
    long long v_off;       // first vertex record of the problem (the group's records are concatenated)
    long long s_off;       // first simplex of the problem in the group's simplex numbering
    long long c_off;       // first cell of the problem in the group's cell numbering
};

struct ProbTable {
    int n;                 // problems (1 .. CDP_GROUP)
    int dim;
    long long nv, ns, ncells;  // totals over the group
    ProbEntry p[CDP_GROUP];
};

// the problem holding global index i of the numbering whose first indices are off(p) (n >= 1)
template <class Off>
__host__ __device__ __forceinline__ int table_find(const ProbTable& T, long long i, Off off) {
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off(T.p[mid]) <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}
__host__ __device__ __forceinline__ int find_vertex(const ProbTable& T, long long i) {
    return table_find(T, i, [](const ProbEntry& e) { return e.v_off; });
}
__host__ __device__ __forceinline__ int find_simplex(const ProbTable& T, long long i) {
    return table_find(T, i, [](const ProbEntry& e) { return e.s_off; });
}
__host__ __device__ __forceinline__ int find_cell(const ProbTable& T, long long i) {
    return table_find(T, i, [](const ProbEntry& e) { return e.c_off; });
}

// Per-call device counters (zeroed at the start of every projection).
struct Counters {
    unsigned flags;       // CDP_FLAG_* bits
    unsigned big_count;   // tetrahedra listed as large (bounding box above the main kernel's box)
    unsigned big_next;    // next entry of that list to be tiled by the main kernel's blocks
    unsigned defer_count; // simplices deferred by the first pass (steep density gradient)
    unsigned long long n_class0, n_small, n_zero, n_big_tiles;
    unsigned clip_count;  // simplices re-projected by clipping (accuracy control)
    unsigned big_first;   // large tetrahedra listed by the first pass (big_count is reused after it)
    unsigned long long mmax_bits[CDP_GROUP];  // per problem: largest |cell mass| after the first pass
                                              // (FP64 bits, >= 0)
    unsigned long long ebmax_bits;  // largest error bound of a simplex projected by Franklin's sum
};

// Accuracy control (Sect. 3.4, eqs. accuracy, accuracy2).  The rounding error of the pieces of a
// simplex projected by Franklin's sum is bounded, per piece, by
//     eb = eps_R (k_rho rho_max + k_grad |grad rho|)
// (rho premultiplied by the cell volume, the gradient per cell): the first term is the fixed-point
// rounding of the vertex positions and the rounding of contributions of the size of the density,
// the second the cancellation of contributions carrying the gradient.  The constants were measured
// (the number W of wrong trailing bits found statistically, as Sect. 3.4 does) on simplices of
// every shape -- generic, nearly flat, needle-like, with facets nearly parallel to grid planes, and
// density contrasts up to e^6 -- each alone in its block of cells, against the oracle: largest
// ratios 26 (FP32, with the mass closure of the chunk rounds) and 6400 (FP64) for the first term,
// 2.1 (FP32) and 4 (FP64) for the second; the constants below take those with a margin of 1.5 to 2.
//   A simplex whose gradient exceeds defer_ratio times its density is deferred by the first pass
// (its pieces are not flushed); once the first pass has given the largest cell mass M, a deferred
// simplex is projected by Franklin's sum when eps_R k_grad |grad rho| <= tau M, and by clipping
// (cdp_clip.cu, no cancellation) otherwise.  tau is half the stated accuracy (1e-5 of the largest
// cell for FP32-mixed, 1e-11 for FP64).
struct AccCtl {
    float defer_ratio;  // |grad rho| / rho_max above which the first pass defers a simplex
    double eps_k_rho;   // eps_R k_rho
    double eps_k_grad;  // eps_R k_grad
    double tau;         // accepted cancellation error, relative to the largest cell
};

__host__ __device__ inline AccCtl acc_ctl(int fp32) {
    AccCtl a;
    if (fp32) {
        a.defer_ratio = 30.f;
        a.eps_k_rho = 48.0 * 5.9604644775390625e-08;   // 48 eps_32
        a.eps_k_grad = 4.0 * 5.9604644775390625e-08;   // 4 eps_32
        a.tau = 5e-6;
    } else {
        a.defer_ratio = 30.f;
        a.eps_k_rho = 9800.0 * 1.1102230246251565e-16;  // 9800 eps_64
        a.eps_k_grad = 8.0 * 1.1102230246251565e-16;    // 8 eps_64
        a.tau = 5e-12;
    }
    return a;
}

struct LaunchArgs {
    ProbTable T;        // the problems (their grids, inputs and offsets)
    VertexRec* verts;   // vertex records of the whole group
    Counters* ctr;
    UnitCounts* stats;  // may be null (else two blocks: chunks of the main kernel, tiled large tetrahedra)
    int num_sms;
    int small_blocks_per_sm;  // blocks per SM of the main kernel's grid (a multiple of resident_per_sm)
    int resident_per_sm;      // resident blocks per SM of the main kernel
    int* big_list;      // tetrahedra whose bounding box exceeds the shared box (capacity big_cap),
                        // projected tile by tile by the main kernel
    long long big_cap;
    float* tile_store;        // FP32 pieces of tiles kept between the two passes over a large tetrahedron
    size_t tile_store_cap;    // (floats; null / 0: every tile is computed twice)
    int tile_store_per_block; // tiles kept per block of the large-tetrahedron kernel
    void* geo;          // geometry records of one batch of tetrahedra (capacity geo_cap records;
                        // geo_bytes bytes, also the clip records of the accuracy control in 3D)
    size_t geo_bytes;
    int* need;          // their box sizes (geo_cap entries)
    long long geo_cap;
    int* defer_list;    // simplices deferred by the first pass (capacity defer_cap)
    long long defer_cap;
    int* clip_list;     // simplices projected by clipping (capacity clip_cap)
    long long clip_cap;
    int accuracy;       // 1: accuracy control (AccCtl); 0: every simplex by Franklin's sum
    int max_cells;      // 3D size-class threshold: largest bounding box (cells) of the main kernel
                        // (0: the default; at most the block's box slots, tet_box_slots)
    int tile_edge;      // tile edge (cells) of the large tetrahedra (0: the default; 4 .. tet_tile_edge())
    const unsigned char* levels;  // AMR projection (cdp_amr.cu): the level of every simplex of the
                        // mesh; the table's entry p is level p and sets up only the simplices of
                        // that level (null: every simplex in every entry)
    cudaEvent_t ev_acc; // optional: recorded where the accuracy control starts (timing)
};

// precision argument of the C ABI: arithmetic (CDP_FP64 / CDP_FP32_MIXED) and the accuracy-control
// flag; false for an invalid value
inline bool parse_precision(int precision, int* fp32, int* accuracy) {
    const int base = precision & 0xff;
    if ((precision & ~0x1ff) != 0 || (base != 0 && base != 1)) return false;
    *fp32 = base;
    *accuracy = (precision & 0x100) ? 0 : 1;
    return true;
}

// AMR projection (cdp_amr.cu): the level (0 .. max_level) of every simplex of the mesh of the
// table's entry 0, from its vertex records (launch_prep)
cudaError_t launch_amr_levels(const LaunchArgs& L, int max_level, unsigned char* levels, cudaStream_t st);

cudaError_t configure_all();
// resident blocks per SM of the projection kernel of dimension `dim` (occupancy calculator)
int resident_blocks(int dim, int fp32);
// the tetrahedron kernel (cdp_tetproj.cu)
cudaError_t configure_tet();
int resident_blocks_tet(int fp32);
// bytes of one geometry record of the tetrahedron kernel
size_t tet_geo_bytes(int fp32);
// cells of one tile of a large tetrahedron (of the largest edge), and that edge
size_t tet_tile_cells();
int tet_tile_edge();
// the default size-class threshold (cells of a bounding box) of the main kernel
int tet_max_cells();
// box slots of a block of the main kernel (the largest size-class threshold)
int tet_box_slots(int fp32);
// tiles of a large tetrahedron whose FP32 pieces a block keeps between the two passes
constexpr int CDP_TILE_STORE_PER_BLOCK = 32;
// set-up and main kernel over batches of geo_cap tetrahedra, then the large-tetrahedron kernel;
// `after_setup` and `mid` (optional) are recorded after the first batch's set-up kernel and before
// the large-tetrahedron kernel
cudaError_t launch_tet(const LaunchArgs& L, int fp32, cudaStream_t st, cudaEvent_t after_setup, cudaEvent_t mid);
cudaError_t launch_prep(const LaunchArgs& L, cudaStream_t st);
// `after_setup` and `mid` (optional) are recorded after the (first) set-up kernel and after the
// main kernel (3D: before the large-tetrahedron kernel)
cudaError_t launch_project(const LaunchArgs& L, int fp32, cudaStream_t st, cudaEvent_t after_setup,
                           cudaEvent_t mid);
// between the two passes: the largest |cell mass| of the grid into ctr->mmax_bits, and the first
// pass's count of large tetrahedra kept while the list is emptied for the second pass
cudaError_t launch_pass_boundary(const LaunchArgs& L, cudaStream_t st);
// the simplices of clip_list (cdp_clip.cu)
cudaError_t launch_clip(const LaunchArgs& L, int fp32, cudaStream_t st);

}  // namespace cdp
