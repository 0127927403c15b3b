// Kernels of the projection (Sect. 3; Algorithm 2 organised per simplex instead of per vertex).
//
//  k_prep_vertices   one thread per vertex: world coordinates -> 32-byte fixed-point records.
//  k_project_warp    warp-cooperative projection of chunks of triangles (2D; see below).  Tetrahedra
//                    are projected by the kernels of cdp_tetproj.cu.
#include <cuda_runtime.h>

#include "cdp_mesh.cuh"
#include "cdp_project.h"

namespace cdp {

// One thread per vertex of the group: world coordinates -> 32-byte fixed-point record (its problem's
// grid), at the vertex's place in the group's numbering.
__global__ void k_prep_vertices(const __grid_constant__ ProbTable T, VertexRec* __restrict__ out,
                                unsigned* __restrict__ flags) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.nv) return;
    const ProbEntry& P = T.p[find_vertex(T, i)];
    const long long v = i - P.v_off;
    double p[3] = {P.pos[0][v], P.pos[1][v], P.g.dim == 3 ? P.pos[2][v] : 0.0};
    VertexRec r;
    unsigned f = vertex_to_fixed(P.g, p, P.rho[v], r);
    out[i] = r;
    if (f) atomicOr(flags, f);
}

// ------------------------------------------------------------------------------------------
// Warp-cooperative projection.
//
// A warp takes CDP_CHUNK consecutive simplices.  Each lane canonicalises one of them and writes its
// geometry to shared memory; a simplex inside one cell deposits |V| mean(rho) at once (Algorithm 2,
// step 1).  The work of the chunk is then split into three phases of independent items -- the
// vertices (corners B), the (edge, axis, plane) crossings (corners C) and the grid lines (corners D,
// and along x the grid nodes between the two pierced facets, corners A) -- and each phase's items
// of all simplices are numbered consecutively and dealt to the 32 lanes in turn, so that every
// lane runs the same code on work of similar size (SIMT efficiency and load balance do not depend
// on how unequal the simplices are).  Every (corner, cell) contribution is added into a per-warp
// open-addressing table in shared memory keyed by (simplex of the chunk, cell); the table is
// flushed with one FP64 atomic per (simplex, cell) piece.
//
// FP32-mixed path only: the mass closure (not in the paper).  The FP64 closed-form mass of each
// simplex minus the FP64 sum of its flushed FP32 pieces is added to its largest piece, so the
// total mass is exact to FP64 rounding.
// ------------------------------------------------------------------------------------------

constexpr unsigned EMPTY_KEY = 0xffffffffu;
constexpr int KEY_BITS = 26;                 // cell key bits; the owner slot sits above them
constexpr int MAX_PROBES = 64;

template <int DIM, typename R>
struct GeoOf;
template <typename R>
struct GeoOf<2, R> {
    typedef TriGeo<R> T;
};

template <int DIM, typename R>
struct WarpShared {
    typename GeoOf<DIM, R>::T geo[CDP_CHUNK];
    unsigned keys[CDP_WTBL];
    R vals[CDP_WTBL];
    double csum[CDP_CHUNK];              // FP64 sum of a simplex's pieces (mass closure)
    float asum[CDP_CHUNK];               // sum of |piece| over its table entries
    double resid[CDP_CHUNK];             // closure residual, spread over the table entries
    unsigned long long cmax[CDP_CHUNK];  // largest piece sent straight to the grid (packed |v|, cell)
    unsigned long long queue[CDP_QCAP];  // (corner, cell) records awaiting evaluation
    unsigned qtail;
};

// appends records of simplex `owner` to the warp's queue
struct QueuePush {
    unsigned long long* q;
    unsigned* tail;
    unsigned long long owner_bits;
    __device__ __forceinline__ void operator()(unsigned long long r) {
        unsigned pos = atomicAdd(tail, 1u);
        q[pos & (CDP_QCAP - 1)] = r | owner_bits;
    }
};

// Adds into the per-warp table on behalf of simplex `owner` of the chunk; cells that do not fit
// (table crowded, or a bounding box beyond 2^26 cells) go straight to the grid.
template <int DIM, typename R>
struct WarpAcc {
    WarpShared<DIM, R>* sh;
    int owner;
    int ex, ey;
    bool direct_only;
    const GridDesc* g;  // the owner's problem's grid
    double* out;
    bool closure;

    __device__ __forceinline__ void direct(int x, int y, int z, R v) {
        const int* an = sh->geo[owner].anchor;
        long long idx = flat_cell(*g, an[0] + x, an[1] + y, an[2] + z);
        if (idx < 0) return;
        atomicAdd(out + idx, (double)v);
        if (closure) {
            atomicAdd(&sh->csum[owner], (double)v);
            unsigned long long packed = ((unsigned long long)__float_as_uint(fabsf((float)v)) << 32) |
                                        (unsigned long long)(unsigned)idx;
            atomicMax(&sh->cmax[owner], packed);
        }
    }

    __device__ __forceinline__ void operator()(int x, int y, int z, R v) {
        if (direct_only) {
            direct(x, y, z, v);
            return;
        }
        unsigned key = ((unsigned)owner << KEY_BITS) | (unsigned)(x + ex * (y + ey * z));
        unsigned h = (key * 2654435761u) >> (32 - CDP_LOG_WTBL);
        volatile unsigned* keys = sh->keys;
        for (int p = 0; p < MAX_PROBES; ++p) {
            unsigned k = keys[h];
            if (k == key) {
                atomicAdd(&sh->vals[h], v);
                return;
            }
            if (k == EMPTY_KEY) {
                unsigned old = atomicCAS(&sh->keys[h], EMPTY_KEY, key);
                if (old == EMPTY_KEY || old == key) {
                    atomicAdd(&sh->vals[h], v);
                    return;
                }
            }
            h = (h + 1) & (CDP_WTBL - 1);
        }
        direct(x, y, z, v);
    }
};

__device__ __forceinline__ void add_counts(UnitCounts* dst, const UnitCounts& c) {
    if (c.a) atomicAdd(&dst->a, c.a);
    if (c.b) atomicAdd(&dst->b, c.b);
    if (c.c) atomicAdd(&dst->c, c.c);
    if (c.d) atomicAdd(&dst->d, c.d);
    if (c.exact) atomicAdd(&dst->exact, c.exact);
}

__device__ __forceinline__ bool fetch_vertices(const int* __restrict__ simp, long long s, int nvs, long long nv,
                                               const VertexRec* __restrict__ V, const VertexRec* v[4]) {
    for (int k = 0; k < nvs; ++k) {
        int id = __ldg(simp + s * nvs + k);
        if (id < 0 || id >= nv) return false;
        v[k] = V + id;
    }
    return true;
}

// owner lane of flat item u: the first lane whose inclusive prefix exceeds u
__device__ __forceinline__ int owner_of(int pre, int u) {
    int own = 0;
    for (int step = 16; step > 0; step >>= 1) {
        int p = __shfl_sync(0xffffffffu, pre, own + step - 1);
        if (p <= u) own += step;
    }
    return own > 31 ? 31 : own;
}

// per-triangle item counts of the three phases
template <typename R>
__device__ __forceinline__ void tri_counts(const TriGeo<R>& G, int n[3]) {
    const int td[2] = {G.hi[0] + 1, G.hi[1] + 1};
    n[0] = 3;
    n[1] = 0;
    for (int o = 0; o < 3; ++o)
        for (int k = 0; k < 2; ++k) {
            int c0;
            n[1] += tri_crossings(G, o, k, td, c0);
        }
    int dy0;
    n[2] = tri_rows(G, td, dy0);
}

template <int DIM, typename R>
__device__ __forceinline__ WarpAcc<DIM, R> make_acc(WarpShared<DIM, R>* sh, int own, const ProbTable& T,
                                                    bool closure) {
    const typename GeoOf<DIM, R>::T& G = sh->geo[own];
    WarpAcc<DIM, R> acc;
    acc.sh = sh;
    acc.owner = own;
    acc.ex = G.hi[0] + 1;
    acc.ey = G.hi[1] + 1;
    long long cells = (long long)acc.ex * acc.ey;
    acc.direct_only = cells >= (1ll << KEY_BITS);
    acc.g = &T.p[G.prob].g;
    acc.out = T.p[G.prob].out;
    acc.closure = closure;
    return acc;
}

// phase items with the queue: 0 vertex (evaluated), 1 crossing (queued), 2 row (evaluated)
template <typename R, class Acc, class Push>
__device__ __forceinline__ void tri_phase_item(const TriGeo<R>& G, int ph, int t, Acc& acc, Push& push,
                                               UnitCounts* cnt) {
    const int td[2] = {G.hi[0] + 1, G.hi[1] + 1};
    if (ph == 0) {
        tri_item_vertex(G, t, td, acc, cnt);
    } else if (ph == 1) {
        for (int o = 0; o < 3; ++o)
            for (int k = 0; k < 2; ++k) {
                int c0, n = tri_crossings(G, o, k, td, c0);
                if (t < n) {
                    tri_locate_crossing(G, o, k, c0 + t, td, push, cnt);
                    return;
                }
                t -= n;
            }
    } else {
        int dy0;
        tri_rows(G, td, dy0);
        tri_item_row(G, dy0 + t, td, acc, cnt);
    }
}

// evaluate one queued corner record of phase ph and add its cells to its simplex's pieces
template <int DIM, typename R>
__device__ __forceinline__ void eval_record(WarpShared<DIM, R>* sh, unsigned long long r, int ph, const ProbTable& T,
                                            bool closure, UnitCounts* cnt) {
    const int own = (int)((r >> 40) & 31);
    const typename GeoOf<DIM, R>::T& G = sh->geo[own];
    WarpAcc<DIM, R> acc = make_acc<DIM, R>(sh, own, T, closure);
    (void)ph;
    int v0, v1, v2;
    R val = tri_eval_crossing(G, r, v0, v1, v2);
    if (cnt) cnt->c++;
    acc(v0, v1, v2, val);
}

// The lists of the accuracy control and the pass of the 2D kernel (second pass: the simplices of
// the deferred list, their number read on the device).
struct WarpPass {
    AccCtl acc;
    int second;
    const unsigned char* levels;  // AMR projection: the level of every simplex (entry p = level p)
    int* defer_list;
    long long defer_cap;
    int* clip_list;
    long long clip_cap;
    int chunk;  // triangles per warp chunk, 8 .. CDP_CHUNK (fewer when the problem is small)
};

template <int DIM, typename R>
__global__ void __launch_bounds__(CDP_WBLOCK, 3) k_project_warp(const __grid_constant__ ProbTable T,
                                                            const VertexRec* __restrict__ V,
                                                            Counters* __restrict__ ctr,
                                                            UnitCounts* __restrict__ stats, WarpPass wp) {
    static_assert(DIM == 2, "tetrahedra are projected by the kernels of cdp_tetproj.cu");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool fp32 = sizeof(R) == 4;
    const int lane = threadIdx.x & 31;
    WarpShared<DIM, R>* sh = reinterpret_cast<WarpShared<DIM, R>*>(smem_raw) + (threadIdx.x >> 5);
    for (int e = lane; e < CDP_WTBL; e += 32) {
        sh->keys[e] = EMPTY_KEY;
        sh->vals[e] = R(0);
    }
    if (lane == 0) sh->qtail = 0u;
    __syncwarp();
    UnitCounts cnt = {0, 0, 0, 0, 0};
    UnitCounts* pc = stats ? &cnt : nullptr;
    unsigned long long n0 = 0, nact = 0, nzero = 0;
    double ebm = 0.0;  // the largest error bound of the simplices this lane set up for Franklin's sum
    long long ns = T.ns;
    if (wp.second) {
        const long long listed = (long long)*(volatile const unsigned*)&ctr->defer_count;
        ns = listed < wp.defer_cap ? listed : wp.defer_cap;
    }
    const int cs = wp.chunk;
    const long long nchunks = (ns + cs - 1) / cs;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long chunk = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); chunk < nchunks;
         chunk += warps) {
        // ---- setup: one simplex per lane
        const long long item = chunk * cs + lane;
        bool active = false;
        int n[3] = {0, 0, 0};
        if (lane < cs && item < ns) {
            const long long sg = wp.second ? (long long)wp.defer_list[item] : item;  // in the group's numbering
            const int prob = find_simplex(T, sg);
            const ProbEntry& P = T.p[prob];
            const GridDesc& g = P.g;
            const long long s = sg - P.s_off;
            const VertexRec* v[4];
            if (s >= P.ns || (wp.levels && (int)wp.levels[s] != prob)) {
                // (an index between two problems, or a simplex of another level of an AMR projection)
            } else if (!fetch_vertices(P.simplices, s, DIM + 1, P.nv, V + P.v_off, v)) {
                atomicOr(&ctr->flags, CDP_FLAG_INDEX);
            } else {
                Tri S;
                unsigned rc = canon_tri(g, v, S);
                if (rc == 1) {
                    ++nzero;
                } else if (rc) {
                    atomicOr(&ctr->flags, rc);
                } else if (S.lo[0] == S.hi[0] && S.lo[1] == S.hi[1]) {
                    long long idx = flat_cell(g, S.anchor[0] + S.lo[0], S.anchor[1] + S.lo[1], 0);
                    if (idx >= 0) atomicAdd(P.out + idx, tri_mass_cells(S));
                    ++n0;
                } else {
                    TriGeo<R>& G = sh->geo[lane];
                    tri_setup(S, S.lo, G);
                    G.prob = prob;
                    // accuracy control (AccCtl): first pass, a steep simplex is deferred; second
                    // pass, one whose cancellation bound exceeds the accepted error is clipped
                    const float rmax = fmaxf(fabsf((float)G.rho[0]), fmaxf(fabsf((float)G.rho[1]), fabsf((float)G.rho[2])));
                    const float gn = sqrtf((float)G.g[0] * (float)G.g[0] + (float)G.g[1] * (float)G.g[1]);
                    if (!wp.second && gn > wp.acc.defer_ratio * rmax) {
                        const unsigned at = atomicAdd(&ctr->defer_count, 1u);
                        if ((long long)at < wp.defer_cap) wp.defer_list[at] = (int)sg;
                    } else if (wp.second &&
                               wp.acc.eps_k_grad * (double)gn >
                                   wp.acc.tau * __longlong_as_double((long long)*(volatile const unsigned long long*)&ctr->mmax_bits[prob])) {
                        const unsigned at = atomicAdd(&ctr->clip_count, 1u);
                        if ((long long)at < wp.clip_cap) wp.clip_list[at] = (int)sg;
                    } else {
                        ebm = fmax(ebm, wp.acc.eps_k_rho * (double)rmax + wp.acc.eps_k_grad * (double)gn);
                        tri_counts(G, n);
                        active = true;
                    }
                }
            }
        }
        if (lane < CDP_CHUNK) {
            sh->csum[lane] = 0.0;
            sh->asum[lane] = 0.f;
            sh->resid[lane] = 0.0;
            sh->cmax[lane] = 0ull;
        }
        nact += active ? 1 : 0;
        __syncwarp();
        if (__ballot_sync(0xffffffffu, active) == 0u) continue;
        // ---- sub-rounds.  The triangles of the chunk share the warp's piece table; when their
        // bounding boxes add up to more cells than the table has entries, the chunk is taken in 2,
        // 4, ... sub-rounds of consecutive lanes so that the pieces of each fit (a crowded table
        // sends pieces straight to the grid, and the FP32 closure then has fewer pieces to spread
        // its residual over).
        int box = 0;
        if (active) {
            const typename GeoOf<DIM, R>::T& G = sh->geo[lane];
            const long long b = (long long)(G.hi[0] + 1) * (G.hi[1] + 1);
            box = b < (1 << 20) ? (int)b : (1 << 20);
        }
        const int boxes = __reduce_add_sync(0xffffffffu, box);
        int nsub = 1;
        while (nsub < 32 && boxes > nsub * CDP_WTBL) nsub <<= 1;
        const int width = 32 / nsub;
        for (int sub = 0; sub < nsub; ++sub) {
            const bool act = active && lane / width == sub;
            if (__ballot_sync(0xffffffffu, act) == 0u) continue;
            // ---- the three phases, items dealt over the lanes.  Phase 0 evaluates its corners (B) at
            // once; phases 1 and 2 locate their corners (C, and D with the A nodes evaluated at once)
            // and queue them, and the queue is drained in full batches of 32 identical evaluations.
            unsigned head = sh->qtail;
            for (int ph = 0; ph < 3; ++ph) {
                int mine = act ? n[ph] : 0;
                int pre = mine;
                for (int o = 1; o < 32; o <<= 1) {
                    int t = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += t;
                }
                const int tot = __shfl_sync(0xffffffffu, pre, 31);
                for (int u0 = 0; u0 < tot; u0 += 32) {
                    const int u = u0 + lane;
                    const int own = owner_of(pre, u);
                    const int before = __shfl_sync(0xffffffffu, pre - mine, own);
                    if (u < tot) {
                        const typename GeoOf<DIM, R>::T& G = sh->geo[own];
                        WarpAcc<DIM, R> acc = make_acc<DIM, R>(sh, own, T, fp32);
                        QueuePush push{sh->queue, &sh->qtail, (unsigned long long)own << 40};
                        const int t = u - before;
                        tri_phase_item(G, ph, t, acc, push, pc);
                    }
                    __syncwarp();
                    // evaluate every full batch of queued records
                    const unsigned tail = *(volatile unsigned*)&sh->qtail;
                    while (tail - head >= 32u) {
                        eval_record<DIM, R>(sh, sh->queue[(head + lane) & (CDP_QCAP - 1)], ph, T, fp32, pc);
                        head += 32u;
                    }
                    __syncwarp();
                }
                // the last partial batch of the phase
                const unsigned tail = *(volatile unsigned*)&sh->qtail;
                if ((unsigned)lane < tail - head)
                    eval_record<DIM, R>(sh, sh->queue[(head + lane) & (CDP_QCAP - 1)], ph, T, fp32, pc);
                head = tail;
                __syncwarp();
            }
            __syncwarp();
            // ---- flush the table: one FP64 atomic per (simplex, cell) piece.  FP32 path: first the
            // FP64 sum of every simplex's pieces, then its closure residual (FP64 closed-form mass
            // minus that sum) is spread over its pieces in proportion to their size while they are
            // flushed (a simplex whose pieces all went straight to the grid gives it to its largest).
            if (fp32) {
                for (int e = lane; e < CDP_WTBL; e += 32) {
                    unsigned k = sh->keys[e];
                    if (k == EMPTY_KEY) continue;
                    R v = sh->vals[e];
                    int own = (int)(k >> KEY_BITS);
                    atomicAdd(&sh->csum[own], (double)v);
                    atomicAdd(&sh->asum[own], fabsf((float)v));
                }
                __syncwarp();
                if (act) {
                    double r = sh->geo[lane].mexact - sh->csum[lane];
                    if (sh->asum[lane] > 0.f) {
                        sh->resid[lane] = r / (double)sh->asum[lane];
                    } else {
                        sh->resid[lane] = 0.0;
                        if (sh->cmax[lane] != 0ull)
                            atomicAdd(T.p[sh->geo[lane].prob].out + (long long)(unsigned)(sh->cmax[lane] & 0xffffffffull), r);
                    }
                }
                __syncwarp();
            }
            for (int e = lane; e < CDP_WTBL; e += 32) {
                unsigned k = sh->keys[e];
                if (k == EMPTY_KEY) continue;
                R v = sh->vals[e];
                sh->keys[e] = EMPTY_KEY;
                sh->vals[e] = R(0);
                int own = (int)(k >> KEY_BITS);
                unsigned lk = k & ((1u << KEY_BITS) - 1u);
                const typename GeoOf<DIM, R>::T& G = sh->geo[own];
                const ProbEntry& P = T.p[G.prob];
                int ex = G.hi[0] + 1, ey = G.hi[1] + 1;
                int x = (int)(lk % (unsigned)ex), r = (int)(lk / (unsigned)ex);
                int y = r % ey, z = r / ey;
                long long idx = flat_cell(P.g, G.anchor[0] + x, G.anchor[1] + y, G.anchor[2] + z);
                if (idx < 0) continue;
                double dv = (double)v;
                if (fp32) dv += sh->resid[own] * (double)fabsf((float)v);
                if (dv != 0.0) atomicAdd(P.out + idx, dv);
            }
            __syncwarp();
        }
    }
    if (ebm > 0.0) atomicMax(&ctr->ebmax_bits, (unsigned long long)__double_as_longlong(ebm));
    if (stats) {
        add_counts(stats, cnt);
        if (n0) atomicAdd(&ctr->n_class0, n0);
        if (nact) atomicAdd(&ctr->n_small, nact);
        if (nzero) atomicAdd(&ctr->n_zero, nzero);
    }
}

// ------------------------------------------------------------------------------------------
// host-side launch sequence (all on `stream`, no synchronisation)
// ------------------------------------------------------------------------------------------

template <int DIM, typename R>
static size_t shared_bytes() {
    return sizeof(WarpShared<DIM, R>) * (CDP_WBLOCK / 32);
}

cudaError_t configure_all() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_project_warp<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shared_bytes<2, float>())))
        return e;
    if ((e = cudaFuncSetAttribute(k_project_warp<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shared_bytes<2, double>())))
        return e;
    return configure_tet();
}

int resident_blocks(int dim, int fp32) {
    if (dim == 3) return resident_blocks_tet(fp32);
    int n = 0;
    cudaError_t e;
    {
        e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_project_warp<2, float>, CDP_WBLOCK,
                                                                 shared_bytes<2, float>())
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_project_warp<2, double>, CDP_WBLOCK,
                                                                 shared_bytes<2, double>());
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

// First pass over every triangle (steep ones deferred), the largest cell mass, second pass over the
// deferred ones (the grid of the first pass's size: the count is read on the device), clipping.
// A problem too small to give every resident warp a chunk of CDP_CHUNK triangles takes chunks of
// 16 or 8 (more warps at work on a latency-bound launch); large ones take full chunks.
template <int DIM, typename R>
static cudaError_t launch_dim(const LaunchArgs& L, cudaStream_t st, cudaEvent_t mid) {
    long long cap = (long long)L.num_sms * L.small_blocks_per_sm;
    const long long warps = cap * (CDP_WBLOCK / 32);
    int cs = CDP_CHUNK;
    while (cs > 8 && L.T.ns < warps * cs) cs >>= 1;
    long long chunks = (L.T.ns + cs - 1) / cs;
    long long blocks = (chunks + CDP_WBLOCK / 32 - 1) / (CDP_WBLOCK / 32);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    WarpPass wp = {acc_ctl(sizeof(R) == 4), 0, L.levels, L.defer_list, L.defer_cap, L.clip_list, L.clip_cap, cs};
    if (!L.accuracy) wp.acc.defer_ratio = 3.0e38f;  // nothing is deferred
    k_project_warp<DIM, R><<<(unsigned)blocks, CDP_WBLOCK, shared_bytes<DIM, R>(), st>>>(L.T, L.verts, L.ctr, L.stats,
                                                                                       wp);
    if (mid) cudaEventRecord(mid, st);
    if (L.ev_acc) cudaEventRecord(L.ev_acc, st);
    if (!L.accuracy) return cudaGetLastError();
    cudaError_t e = launch_pass_boundary(L, st);
    if (e != cudaSuccess) return e;
    wp.second = 1;
    wp.levels = nullptr;  // (the deferred list holds the right entries only)
    k_project_warp<DIM, R><<<(unsigned)blocks, CDP_WBLOCK, shared_bytes<DIM, R>(), st>>>(L.T, L.verts, L.ctr, L.stats,
                                                                                       wp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_clip(L, sizeof(R) == 4, st);
}

cudaError_t launch_prep(const LaunchArgs& L, cudaStream_t st) {
    if (L.T.nv > 0) {
        unsigned blocks = (unsigned)((L.T.nv + 255) / 256);
        k_prep_vertices<<<blocks, 256, 0, st>>>(L.T, L.verts, &L.ctr->flags);
    }
    return cudaGetLastError();
}

cudaError_t launch_project(const LaunchArgs& L, int fp32, cudaStream_t st, cudaEvent_t after_setup,
                           cudaEvent_t mid) {
    if (L.T.ns == 0) {
        if (after_setup) cudaEventRecord(after_setup, st);
        if (mid) cudaEventRecord(mid, st);
        if (L.ev_acc) cudaEventRecord(L.ev_acc, st);
        return cudaSuccess;
    }
    if (L.T.dim == 3) {
        return launch_tet(L, fp32, st, after_setup, mid);
    }
    if (after_setup) cudaEventRecord(after_setup, st);
    return fp32 ? launch_dim<2, float>(L, st, mid) : launch_dim<2, double>(L, st, mid);
}

}  // namespace cdp
