// Internal interface between the C-ABI layer (cdp_api.cu) and the projection kernels.
#pragma once

#include <cuda_runtime.h>

#include "cdp_mesh.cuh"

namespace cdp {

constexpr int CDP_BLOCK = 128;             // threads per block of the projection kernels
constexpr int CDP_ONE_THREAD_CELLS = 512;  // bounding boxes up to this many cells: one thread
constexpr int CDP_TILE = 8;                // tile edge (cells) of the larger simplices

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
