// Definition of the context object shared by the C-ABI translation units (internal).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <vector>

#include "cdp_project.h"

namespace cdp {

// cached cuFFT plans and spectrum buffer of one grid shape
struct FftPlan {
    int dim;
    int n[3];
    cufftHandle r2c, c2r;
    cufftDoubleComplex* spec;
    size_t spec_elems;
    // single-precision transforms of the FP32-mixed time step (made on first use)
    int have32;
    cufftHandle r2c32, c2r32;
    cufftComplex* spec32;
    float* real32;  // the source, then the potential, in FP32
};

}  // namespace cdp

struct cdp_ctx;
struct cdp_problem_tag;

namespace cdp {
constexpr int CDP_TEV = 6;
void solver_release(cdp_ctx* c);
void step_release(cdp_ctx* c);
}  // namespace cdp

struct cdp_ctx {
    int device;
    int num_sms;
    int blocks_small[2];  // resident blocks per SM of the 3D kernel (fp64, fp32)
    int blocks_big[2];    // of the 2D kernel
    int grid_mult[2][2];  // [dim == 3][fp32]: the main kernel's persistent grid, in multiples of its
                          // resident blocks (8 unless cdp_autotune chose another)
    int max_cells[2];     // [fp32]: 3D size-class threshold (0: the default, tet_max_cells())
    int tile_edge[2];     // [fp32]: tile edge of the large tetrahedra (0: the default, tet_tile_edge() cells)
    cdp::VertexRec* verts;
    size_t verts_cap;
    int* queue;           // list of the large tetrahedra (tiled by the main kernel)
    size_t queue_cap;
    unsigned char* geo;   // geometry records of one batch of tetrahedra (bytes)
    size_t geo_cap;
    int* need;            // their box sizes
    size_t need_cap;
    int* defer;           // simplices deferred by the first pass (accuracy control)
    size_t defer_cap;
    int* clip;            // simplices projected by clipping
    size_t clip_cap;
    double* amr;          // coarse levels' grids of an AMR projection (cdp_project_amr)
    size_t amr_cap;
    unsigned char* levels;  // level of every simplex of an AMR projection
    size_t levels_cap;
    float* tiles;         // FP32 pieces of large-tetrahedron tiles kept between the two passes
    size_t tiles_cap;     // (floats)
    cdp::Counters* ctr;       // device
    cdp::UnitCounts* stats;   // device
    cdp::Counters* h_ctr;     // pinned host mirrors
    cdp::UnitCounts* h_stats;
    // per-kernel timing: CDP_TEV events per timed call (before the vertex records, after them,
    // after the set-up kernel, after the main kernel, after the large-tetrahedron kernel, after the
    // accuracy control), folded into totals[CDP_TEV - 1] when read
    int timing;
    std::vector<cudaEvent_t>* pending;
    std::vector<cudaEvent_t>* pool;
    double totals[cdp::CDP_TEV - 1];
    int calls;
    // solver scratch
    std::vector<cdp::FftPlan>* plans;
    double* vsum;  // per-vertex accumulators of the vertex density (mass, volume)
    size_t vsum_cap;
    float* preal;  // FP32 sources / potentials of a batched step's Poisson solves, one per mesh
    size_t preal_cap;
    cufftComplex* pspec;  // and their half spectra
    size_t pspec_cap;
    // captured time steps (see cdp_step_batched) and the device copy of their dt.  `epoch` advances
    // whenever a scratch buffer is reallocated or the launch shapes are retuned; a graph recorded
    // at an older epoch holds stale addresses and is recaptured instead of replayed
    unsigned long long epoch;
    struct StepGraph* graphs;
    double* d_dt;
    cudaStream_t capture_stream;  // private stream the step graphs are recorded on
};
