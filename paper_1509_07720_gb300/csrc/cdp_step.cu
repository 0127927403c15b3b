// One time step of many independent meshes (Sect. 4, steps (ii)-(iv)), optionally captured once
// into a CUDA graph and replayed:  drift dt/2 -> vertex densities -> exact projection -> FFT
// Poisson -> force at the vertices -> kick dt -> drift dt/2.
#include <cuda_runtime.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/coldproj.h"
#include "cdp_ctx.h"

namespace cdp {
int reserve_scratch(cdp_ctx* c, const cdp_problem* probs, int n);
int project_batch(cdp_ctx* c, const cdp_problem* probs, int n, int precision, cudaStream_t st);
int poisson_enqueue(cdp_ctx* c, int dim, const int32_t grid[3], const double box_len[3], double four_pi_G,
                    const double* mass, double* phi, cudaStream_t st, bool fp32);
int step_drift_density_enqueue(cdp_ctx* c, const cdp_step_problem* probs, int n, const double* dtp, cudaStream_t st);
int step_force_kick_drift_enqueue(cdp_ctx* c, const cdp_step_problem* probs, int n, const double* dtp,
                                  cudaStream_t st);
long long step_group_vertices(const cdp_step_problem* probs, int n);
int reserve_vsum(cdp_ctx* c, size_t need);
int reserve_poisson32(cdp_ctx* c, const cdp_step_problem* probs, int n);
int step_poisson32_enqueue(cdp_ctx* c, const cdp_step_problem* probs, int n, double four_pi_G, cudaStream_t st);
}  // namespace cdp

// a captured step: the exact arguments it was recorded with, and its executable graph
struct StepGraph {
    std::vector<cdp_step_problem> key;
    int precision;
    double four_pi_G;
    unsigned long long epoch;  // the context's epoch when it was recorded
    cudaGraphExec_t exec;
    StepGraph* next;
};

namespace {

struct Guard {
    int prev;
    bool changed;
    explicit Guard(int dev) : prev(0), changed(false) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~Guard() {
        if (changed) cudaSetDevice(prev);
    }
};

// every kernel of the step, in order; `dtp` is the device scalar holding dt
int enqueue_step(cdp_ctx* c, const cdp_step_problem* probs, int n, int precision, double four_pi_G, const double* dtp,
                 cudaStream_t st) {
    int rc;
    // drift dt/2 and the vertex densities: one launch of each kernel per group of meshes
    if ((rc = cdp::step_drift_density_enqueue(c, probs, n, dtp, st))) return rc;
    // the projections of all the meshes, grouped (one launch of each projection kernel per group of
    // up to 64 meshes of one dimension)
    {
        std::vector<cdp_problem> meshes((size_t)n);
        for (int i = 0; i < n; ++i) meshes[(size_t)i] = probs[i].mesh;
        if ((rc = cdp::project_batch(c, meshes.data(), n, precision, st))) return rc;
    }
    // the potential of every mesh (its own FFT plans): FP64 transforms one mesh after the other, or
    // (FP32-mixed) single-precision transforms with the element-wise steps batched per group
    if ((precision & 0xff) == CDP_FP32_MIXED) {
        if ((rc = cdp::step_poisson32_enqueue(c, probs, n, four_pi_G, st))) return rc;
    } else {
        for (int i = 0; i < n; ++i) {
            const cdp_problem& m = probs[i].mesh;
            if ((rc = cdp::poisson_enqueue(c, m.dim, m.grid, m.box_len, four_pi_G, m.cell_mass, probs[i].phi, st,
                                           false)))
                return rc;
        }
    }
    // force, kick dt and drift dt/2 of every vertex: one launch per group of meshes
    return cdp::step_force_kick_drift_enqueue(c, probs, n, dtp, st);
}

int check_step_problem(const cdp_step_problem& s) {
    const cdp_problem& m = s.mesh;
    if (m.dim != 2 && m.dim != 3) return CDP_ERR_ARG;
    if (m.n_verts < 0 || m.n_simplices < 0 || m.n_verts > 0x7fffffffLL || m.n_simplices > 0x7fffffffLL)
        return CDP_ERR_ARG;
    if (!m.cell_mass || !s.phi || (m.n_simplices > 0 && (!m.simplices || !s.simplex_mass))) return CDP_ERR_ARG;
    if (!m.periodic) return CDP_ERR_ARG;  // the FFT Poisson solve is periodic
    long long cells = 1;
    for (int a = 0; a < m.dim; ++a) {
        if (m.grid[a] < 1 || m.grid[a] > (1 << 20) || !(m.box_len[a] > 0.0)) return CDP_ERR_ARG;
        if (m.n_verts > 0 && (!m.pos[a] || !s.vel[a] || !s.acc[a])) return CDP_ERR_ARG;
        cells *= m.grid[a];
        if (cells > (1LL << 32)) return CDP_ERR_ARG;
    }
    if (m.n_verts > 0 && !m.rho) return CDP_ERR_ARG;
    return CDP_OK;
}

// destroy the graphs recorded at an older epoch of the context (an executable graph still running
// is freed when it completes)
void drop_stale_graphs(cdp_ctx* c) {
    StepGraph** link = &c->graphs;
    while (*link) {
        StepGraph* g = *link;
        if (g->epoch == c->epoch) {
            link = &g->next;
            continue;
        }
        *link = g->next;
        cudaGraphExecDestroy(g->exec);
        delete g;
    }
}

}  // namespace

namespace cdp {
void step_release(cdp_ctx* c) {
    StepGraph* g = c->graphs;
    while (g) {
        StepGraph* nx = g->next;
        cudaGraphExecDestroy(g->exec);
        delete g;
        g = nx;
    }
    c->graphs = nullptr;
    if (c->d_dt) cudaFree(c->d_dt);
    c->d_dt = nullptr;
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->capture_stream = nullptr;
}
}  // namespace cdp

extern "C" int cdp_step_batched(cdp_ctx* c, const cdp_step_problem* probs, int n, int precision, double dt,
                                double four_pi_G, int use_graph, void* stream) {
    if (!c || n < 0 || (n > 0 && !probs)) return CDP_ERR_ARG;
    {
        int f = 0, a = 0;
        if (!cdp::parse_precision(precision, &f, &a)) return CDP_ERR_ARG;
    }
    if (!(dt == dt) || !(four_pi_G == four_pi_G)) return CDP_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        int rc = check_step_problem(probs[i]);
        if (rc) return rc;
    }
    Guard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->d_dt && cudaMalloc(&c->d_dt, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_OOM;
    }
    // dt travels through device memory so that a replayed graph picks up the current value
    if (cudaMemcpyAsync(c->d_dt, &dt, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) return CDP_ERR_CUDA;
    if (!use_graph) return enqueue_step(c, probs, n, precision, four_pi_G, c->d_dt, st);

    // graphs recorded before a scratch buffer moved (or the launch shapes were retuned) hold stale
    // addresses: drop them, then replay a current one recorded with these arguments
    drop_stale_graphs(c);
    for (StepGraph* g = c->graphs; g; g = g->next) {
        if ((int)g->key.size() == n && g->precision == precision && g->four_pi_G == four_pi_G &&
            memcmp(g->key.data(), probs, (size_t)n * sizeof(cdp_step_problem)) == 0) {
            return cudaGraphLaunch(g->exec, st) == cudaSuccess ? CDP_OK : CDP_ERR_CUDA;
        }
    }
    // first call with these arguments: size every scratch buffer and create every FFT plan before
    // the capture (nothing may allocate inside it)
    std::vector<cdp_problem> meshes((size_t)n);
    for (int i = 0; i < n; ++i) meshes[(size_t)i] = probs[i].mesh;
    int rc = cdp::reserve_scratch(c, meshes.data(), n);
    if (rc) return rc;
    {
        const long long most = cdp::step_group_vertices(probs, n);
        if ((rc = cdp::reserve_vsum(c, 2 * (size_t)(most > 0 ? most : 1)))) return rc;
        if ((precision & 0xff) == CDP_FP32_MIXED && (rc = cdp::reserve_poisson32(c, probs, n))) return rc;
    }
    for (int i = 0; i < n; ++i) {
        // creates the FFT plan (and its spectrum buffers) of every grid shape, with a harmless
        // solve on the problem's own arrays
        const cdp_problem& m = probs[i].mesh;
        if ((rc = cdp::poisson_enqueue(c, m.dim, m.grid, m.box_len, four_pi_G, m.cell_mass, probs[i].phi, st,
                                       (precision & 0xff) == CDP_FP32_MIXED)))
            return rc;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return CDP_ERR_CUDA;
    // the sequence is recorded on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is then launched on the caller's stream
    if (!c->capture_stream && cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    cudaStream_t cs = c->capture_stream;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    int timing = c->timing;
    c->timing = 0;  // no event bookkeeping inside the captured sequence
    const unsigned long long epoch = c->epoch;
    rc = enqueue_step(c, probs, n, precision, four_pi_G, c->d_dt, cs);
    c->timing = timing;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc ? rc : CDP_ERR_CUDA;
    }
    if (c->epoch != epoch) {
        // a buffer moved while the sequence was recorded (the reservation above missed it): the
        // recording is not replayable, the step runs eagerly on the sized scratch instead
        cudaGraphDestroy(graph);
        return enqueue_step(c, probs, n, precision, four_pi_G, c->d_dt, st);
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    StepGraph* g = new (std::nothrow) StepGraph;
    if (!g) {
        cudaGraphExecDestroy(exec);
        return CDP_ERR_OOM;
    }
    g->key.assign(probs, probs + n);
    g->precision = precision;
    g->four_pi_G = four_pi_G;
    g->epoch = epoch;
    g->exec = exec;
    g->next = c->graphs;
    c->graphs = g;
    return cudaGraphLaunch(exec, st) == cudaSuccess ? CDP_OK : CDP_ERR_CUDA;
}
