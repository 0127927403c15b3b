// Internal interface between the C-ABI layer (cdp_api.cu) and the projection kernels.
#pragma once

#include <cuda_runtime.h>

#include "cdp_mesh.cuh"

namespace cdp {

constexpr int CDP_WBLOCK = 128;   // threads per block of the projection kernel (4 warps)
constexpr int CDP_CHUNK = 16;     // simplices per warp chunk (one per lane during set-up)
constexpr int CDP_LOG_WTBL = 10;  // per-warp piece table: 2^10 entries
constexpr int CDP_WTBL = 1 << CDP_LOG_WTBL;
constexpr int CDP_QCAP = 512;     // per-warp queue of (corner, cell) records (power of two)

// Per-call device counters (zeroed at the start of every projection).
struct Counters {
    unsigned flags;       // CDP_FLAG_* bits
    unsigned big_count;   // tetrahedra listed as large (bounding box above the main kernel's box)
    unsigned big_next;    // next entry of that list to be tiled by the main kernel's blocks
    unsigned pad;
    unsigned long long n_class0, n_small, n_zero, n_big_tiles;
};

struct LaunchArgs {
    GridDesc g;
    long long nv, ns;
    const int* simplices;
    VertexRec* verts;
    double* out;
    double cellvol;
    int* queue;
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
    void* geo;          // geometry records of one batch of tetrahedra (capacity geo_cap records)
    int* need;          // their box sizes (geo_cap entries)
    long long geo_cap;
};

cudaError_t configure_all();
// resident blocks per SM of the projection kernel of dimension `dim` (occupancy calculator)
int resident_blocks(int dim, int fp32);
// the tetrahedron kernel (cdp_tetproj.cu)
cudaError_t configure_tet();
int resident_blocks_tet(int fp32);
// bytes of one geometry record of the tetrahedron kernel
size_t tet_geo_bytes(int fp32);
// cells of one tile of a large tetrahedron
size_t tet_tile_cells();
// tiles of a large tetrahedron whose FP32 pieces a block keeps between the two passes
constexpr int CDP_TILE_STORE_PER_BLOCK = 64;
// set-up and main kernel over batches of geo_cap tetrahedra, then the large-tetrahedron kernel;
// `after_setup` and `mid` (optional) are recorded after the first batch's set-up kernel and before
// the large-tetrahedron kernel
cudaError_t launch_tet(const LaunchArgs& L, int fp32, cudaStream_t st, cudaEvent_t after_setup, cudaEvent_t mid);
cudaError_t launch_prep(const LaunchArgs& L, const double* px, const double* py, const double* pz,
                        const double* rho, cudaStream_t st);
// `after_setup` and `mid` (optional) are recorded after the (first) set-up kernel and after the
// main kernel (3D: before the large-tetrahedron kernel)
cudaError_t launch_project(const LaunchArgs& L, int fp32, cudaStream_t st, cudaEvent_t after_setup,
                           cudaEvent_t mid);

}  // namespace cdp
