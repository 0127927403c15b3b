// Internal interface between the C-ABI layer (cdp_api.cu) and the projection kernels.
#pragma once

#include <cuda_runtime.h>

#include "cdp_mesh.cuh"

namespace cdp {

constexpr int CDP_BLOCK = 128;        // threads per block of the projection kernels
constexpr int CDP_SMALL_CELLS = 64;   // bounding boxes up to this many cells: one thread, one unit
constexpr int CDP_TILE = 4;           // tile edge (cells) for large tetrahedra: 4^3 = 64 slots
constexpr int CDP_TILE2 = 8;          // tile edge for large triangles: 8^2 = 64 slots

// Per-call device counters (zeroed at the start of every projection).
struct Counters {
    unsigned flags;       // CDP_FLAG_* bits
    unsigned big_count;   // simplices queued for the tiled kernel
    unsigned big_next;    // work cursor of the tiled kernel
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
    UnitCounts* stats;  // may be null
    int num_sms;
    int small_blocks_per_sm;
    int big_blocks_per_sm;
};

cudaError_t configure_all();
cudaError_t launch_prep(const LaunchArgs& L, const double* px, const double* py, const double* pz,
                        const double* rho, cudaStream_t st);
// `mid` (optional) is recorded between the one-thread kernel and the tiled kernel
cudaError_t launch_project(const LaunchArgs& L, int fp32, cudaStream_t st, cudaEvent_t mid);

}  // namespace cdp
