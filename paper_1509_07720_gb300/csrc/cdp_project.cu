// Kernels of the projection (Sect. 3; Algorithm 2 organised per simplex instead of per vertex).
//
//  k_prep_vertices   one thread per vertex: world coordinates -> 32-byte fixed-point records.
//  k_project_small   one thread per simplex: canonicalise; a simplex inside one cell deposits
//                    |V| mean(rho) there (Algorithm 2, step 1); a simplex whose bounding box has
//                    at most CDP_SMALL_CELLS cells is projected by the same thread into a private
//                    slice of shared memory (one slot per bounding-box cell) that is then flushed
//                    with one FP64 atomic per touched cell; larger simplices are queued.
//  k_project_big     persistent warps pull queued simplices; lane t projects tiles t, t+32, ... of
//                    the simplex's bounding box (CDP_TILE^D cells each) the same way.
#include <cuda_runtime.h>

#include "cdp_mesh.cuh"
#include "cdp_project.h"

namespace cdp {

__global__ void k_prep_vertices(GridDesc g, long long nv, const double* __restrict__ px,
                                const double* __restrict__ py, const double* __restrict__ pz,
                                const double* __restrict__ rho, VertexRec* __restrict__ out,
                                unsigned* __restrict__ flags) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double p[3] = {px[i], py[i], g.dim == 3 ? pz[i] : 0.0};
    VertexRec r;
    unsigned f = vertex_to_fixed(g, p, rho[i], r);
    out[i] = r;
    if (f) atomicOr(flags, f);
}

// per-thread accumulator in shared memory: slot (x, y, z) of the current tile
template <typename R>
struct SmemAcc {
    R* base;
    int stride, tdx, tdy;
    __device__ __forceinline__ void operator()(int x, int y, int z, R v) const {
        base[(x + tdx * (y + tdy * z)) * stride] += v;
    }
};

__device__ __forceinline__ void add_counts(UnitCounts* dst, const UnitCounts& c) {
    if (c.a) atomicAdd(&dst->a, c.a);
    if (c.b) atomicAdd(&dst->b, c.b);
    if (c.c) atomicAdd(&dst->c, c.c);
    if (c.d) atomicAdd(&dst->d, c.d);
    if (c.exact) atomicAdd(&dst->exact, c.exact);
}

// Project the part of tetrahedron S that lies in tile T (td cells) and flush it.
template <typename R>
__device__ void tet_tile(const GridDesc& g, const Tet& S, const int T[3], const int td[3], R* slot, int stride,
                         double* __restrict__ out, double cellvol, UnitCounts* cnt) {
    int ncell = td[0] * td[1] * td[2];
    for (int i = 0; i < ncell; ++i) slot[i * stride] = R(0);
    TetGeo<R> G;
    tet_setup(S, T, G);
    SmemAcc<R> acc{slot, stride, td[0], td[1]};
    tet_unit(G, td, acc, cnt);
    for (int z = 0; z < td[2]; ++z)
        for (int y = 0; y < td[1]; ++y)
            for (int x = 0; x < td[0]; ++x) {
                R v = slot[(x + td[0] * (y + td[1] * z)) * stride];
                if (v != R(0)) {
                    long long idx = flat_cell(g, S.anchor[0] + T[0] + x, S.anchor[1] + T[1] + y, S.anchor[2] + T[2] + z);
                    if (idx >= 0) atomicAdd(out + idx, (double)v * cellvol);
                }
            }
}

template <typename R>
__device__ void tri_tile(const GridDesc& g, const Tri& S, const int T[2], const int td[2], R* slot, int stride,
                         double* __restrict__ out, double cellvol, UnitCounts* cnt) {
    int ncell = td[0] * td[1];
    for (int i = 0; i < ncell; ++i) slot[i * stride] = R(0);
    TriGeo<R> G;
    tri_setup(S, T, G);
    SmemAcc<R> acc{slot, stride, td[0], td[1]};
    tri_unit(G, td, acc, cnt);
    for (int y = 0; y < td[1]; ++y)
        for (int x = 0; x < td[0]; ++x) {
            R v = slot[(x + td[0] * y) * stride];
            if (v != R(0)) {
                long long idx = flat_cell(g, S.anchor[0] + T[0] + x, S.anchor[1] + T[1] + y, 0);
                if (idx >= 0) atomicAdd(out + idx, (double)v * cellvol);
            }
        }
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

template <typename R>
__global__ void __launch_bounds__(CDP_BLOCK) k_project_small3(GridDesc g, long long ns, long long nv,
                                                              const int* __restrict__ simp,
                                                              const VertexRec* __restrict__ V,
                                                              double* __restrict__ out, double cellvol,
                                                              int* __restrict__ queue, Counters* __restrict__ ctr,
                                                              UnitCounts* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* slot = reinterpret_cast<R*>(smem_raw) + threadIdx.x;
    UnitCounts cnt = {0, 0, 0, 0, 0};
    UnitCounts* pc = stats ? &cnt : nullptr;
    unsigned long long n0 = 0, nsmall = 0, nzero = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
         s += (long long)gridDim.x * blockDim.x) {
        const VertexRec* v[4];
        if (!fetch_vertices(simp, s, 4, nv, V, v)) {
            atomicOr(&ctr->flags, CDP_FLAG_INDEX);
            continue;
        }
        Tet S;
        unsigned rc = canon_tet(g, v, S);
        if (rc == 1) {
            ++nzero;
            continue;
        }
        if (rc) {
            atomicOr(&ctr->flags, rc);
            continue;
        }
        int td[3] = {S.hi[0] - S.lo[0] + 1, S.hi[1] - S.lo[1] + 1, S.hi[2] - S.lo[2] + 1};
        int nc = td[0] * td[1] * td[2];
        if (nc == 1) {
            long long idx = flat_cell(g, S.anchor[0] + S.lo[0], S.anchor[1] + S.lo[1], S.anchor[2] + S.lo[2]);
            if (idx >= 0) atomicAdd(out + idx, tet_mass_cells(S) * cellvol);
            ++n0;
            continue;
        }
        if (nc <= CDP_SMALL_CELLS) {
            tet_tile<R>(g, S, S.lo, td, slot, CDP_BLOCK, out, cellvol, pc);
            ++nsmall;
            continue;
        }
        unsigned pos = atomicAdd(&ctr->big_count, 1u);
        queue[pos] = (int)s;
    }
    if (stats) {
        add_counts(stats, cnt);
        if (n0) atomicAdd(&ctr->n_class0, n0);
        if (nsmall) atomicAdd(&ctr->n_small, nsmall);
        if (nzero) atomicAdd(&ctr->n_zero, nzero);
    }
}

template <typename R>
__global__ void __launch_bounds__(CDP_BLOCK) k_project_big3(GridDesc g, long long nv, const int* __restrict__ simp,
                                                            const VertexRec* __restrict__ V,
                                                            double* __restrict__ out, double cellvol,
                                                            const int* __restrict__ queue,
                                                            Counters* __restrict__ ctr,
                                                            UnitCounts* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* slot = reinterpret_cast<R*>(smem_raw) + threadIdx.x;
    UnitCounts cnt = {0, 0, 0, 0, 0};
    UnitCounts* pc = stats ? &cnt : nullptr;
    unsigned long long ntiles = 0;
    const int lane = threadIdx.x & 31;
    const unsigned total = ctr->big_count;
    while (true) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&ctr->big_next, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        long long s = queue[w];
        const VertexRec* v[4];
        fetch_vertices(simp, s, 4, nv, V, v);
        Tet S;
        canon_tet(g, v, S);  // succeeded in k_project_small3
        int nt[3];
        for (int a = 0; a < 3; ++a) nt[a] = (S.hi[a] - S.lo[a]) / CDP_TILE + 1;
        int tiles = nt[0] * nt[1] * nt[2];
        for (int t = lane; t < tiles; t += 32) {
            int T[3], td[3];
            int tx = t % nt[0], ty = (t / nt[0]) % nt[1], tz = t / (nt[0] * nt[1]);
            T[0] = S.lo[0] + tx * CDP_TILE;
            T[1] = S.lo[1] + ty * CDP_TILE;
            T[2] = S.lo[2] + tz * CDP_TILE;
            for (int a = 0; a < 3; ++a) {
                td[a] = S.hi[a] - T[a] + 1;
                if (td[a] > CDP_TILE) td[a] = CDP_TILE;
            }
            tet_tile<R>(g, S, T, td, slot, CDP_BLOCK, out, cellvol, pc);
            ++ntiles;
        }
    }
    if (stats) {
        add_counts(stats + 1, cnt);
        if (ntiles) atomicAdd(&ctr->n_big_tiles, ntiles);
    }
}

template <typename R>
__global__ void __launch_bounds__(CDP_BLOCK) k_project_small2(GridDesc g, long long ns, long long nv,
                                                              const int* __restrict__ simp,
                                                              const VertexRec* __restrict__ V,
                                                              double* __restrict__ out, double cellvol,
                                                              int* __restrict__ queue, Counters* __restrict__ ctr,
                                                              UnitCounts* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* slot = reinterpret_cast<R*>(smem_raw) + threadIdx.x;
    UnitCounts cnt = {0, 0, 0, 0, 0};
    UnitCounts* pc = stats ? &cnt : nullptr;
    unsigned long long n0 = 0, nsmall = 0, nzero = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
         s += (long long)gridDim.x * blockDim.x) {
        const VertexRec* v[4];
        if (!fetch_vertices(simp, s, 3, nv, V, v)) {
            atomicOr(&ctr->flags, CDP_FLAG_INDEX);
            continue;
        }
        Tri S;
        unsigned rc = canon_tri(g, v, S);
        if (rc == 1) {
            ++nzero;
            continue;
        }
        if (rc) {
            atomicOr(&ctr->flags, rc);
            continue;
        }
        int td[2] = {S.hi[0] - S.lo[0] + 1, S.hi[1] - S.lo[1] + 1};
        int nc = td[0] * td[1];
        if (nc == 1) {
            long long idx = flat_cell(g, S.anchor[0] + S.lo[0], S.anchor[1] + S.lo[1], 0);
            if (idx >= 0) atomicAdd(out + idx, tri_mass_cells(S) * cellvol);
            ++n0;
            continue;
        }
        if (nc <= CDP_SMALL_CELLS) {
            tri_tile<R>(g, S, S.lo, td, slot, CDP_BLOCK, out, cellvol, pc);
            ++nsmall;
            continue;
        }
        unsigned pos = atomicAdd(&ctr->big_count, 1u);
        queue[pos] = (int)s;
    }
    if (stats) {
        add_counts(stats, cnt);
        if (n0) atomicAdd(&ctr->n_class0, n0);
        if (nsmall) atomicAdd(&ctr->n_small, nsmall);
        if (nzero) atomicAdd(&ctr->n_zero, nzero);
    }
}

template <typename R>
__global__ void __launch_bounds__(CDP_BLOCK) k_project_big2(GridDesc g, long long nv, const int* __restrict__ simp,
                                                            const VertexRec* __restrict__ V,
                                                            double* __restrict__ out, double cellvol,
                                                            const int* __restrict__ queue,
                                                            Counters* __restrict__ ctr,
                                                            UnitCounts* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* slot = reinterpret_cast<R*>(smem_raw) + threadIdx.x;
    UnitCounts cnt = {0, 0, 0, 0, 0};
    UnitCounts* pc = stats ? &cnt : nullptr;
    unsigned long long ntiles = 0;
    const int lane = threadIdx.x & 31;
    const unsigned total = ctr->big_count;
    while (true) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&ctr->big_next, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        long long s = queue[w];
        const VertexRec* v[4];
        fetch_vertices(simp, s, 3, nv, V, v);
        Tri S;
        canon_tri(g, v, S);
        int nt[2];
        for (int a = 0; a < 2; ++a) nt[a] = (S.hi[a] - S.lo[a]) / CDP_TILE2 + 1;
        int tiles = nt[0] * nt[1];
        for (int t = lane; t < tiles; t += 32) {
            int T[2], td[2];
            T[0] = S.lo[0] + (t % nt[0]) * CDP_TILE2;
            T[1] = S.lo[1] + (t / nt[0]) * CDP_TILE2;
            for (int a = 0; a < 2; ++a) {
                td[a] = S.hi[a] - T[a] + 1;
                if (td[a] > CDP_TILE2) td[a] = CDP_TILE2;
            }
            tri_tile<R>(g, S, T, td, slot, CDP_BLOCK, out, cellvol, pc);
            ++ntiles;
        }
    }
    if (stats) {
        add_counts(stats + 1, cnt);
        if (ntiles) atomicAdd(&ctr->n_big_tiles, ntiles);
    }
}

// ------------------------------------------------------------------------------------------
// host-side launch sequence (all on `stream`, no synchronisation)
// ------------------------------------------------------------------------------------------

template <typename R>
static cudaError_t configure_kernels() {
    size_t sm = (size_t)CDP_SMALL_CELLS * CDP_BLOCK * sizeof(R);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_project_small3<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    if ((e = cudaFuncSetAttribute(k_project_big3<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    if ((e = cudaFuncSetAttribute(k_project_small2<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    if ((e = cudaFuncSetAttribute(k_project_big2<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    return cudaSuccess;
}

cudaError_t configure_all() {
    cudaError_t e = configure_kernels<float>();
    if (e) return e;
    return configure_kernels<double>();
}

template <typename R>
static cudaError_t launch_typed(const LaunchArgs& L, cudaStream_t st, cudaEvent_t mid) {
    size_t sm = (size_t)CDP_SMALL_CELLS * CDP_BLOCK * sizeof(R);
    long long blocks = (L.ns + CDP_BLOCK - 1) / CDP_BLOCK;
    long long cap = (long long)L.num_sms * L.small_blocks_per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    int big_blocks = L.num_sms * L.big_blocks_per_sm;
    if (L.g.dim == 3) {
        k_project_small3<R><<<(unsigned)blocks, CDP_BLOCK, sm, st>>>(L.g, L.ns, L.nv, L.simplices, L.verts, L.out,
                                                                     L.cellvol, L.queue, L.ctr, L.stats);
        if (mid) cudaEventRecord(mid, st);
        k_project_big3<R><<<big_blocks, CDP_BLOCK, sm, st>>>(L.g, L.nv, L.simplices, L.verts, L.out, L.cellvol,
                                                             L.queue, L.ctr, L.stats);
    } else {
        k_project_small2<R><<<(unsigned)blocks, CDP_BLOCK, sm, st>>>(L.g, L.ns, L.nv, L.simplices, L.verts, L.out,
                                                                     L.cellvol, L.queue, L.ctr, L.stats);
        if (mid) cudaEventRecord(mid, st);
        k_project_big2<R><<<big_blocks, CDP_BLOCK, sm, st>>>(L.g, L.nv, L.simplices, L.verts, L.out, L.cellvol,
                                                             L.queue, L.ctr, L.stats);
    }
    return cudaGetLastError();
}

cudaError_t launch_prep(const LaunchArgs& L, const double* px, const double* py, const double* pz,
                        const double* rho, cudaStream_t st) {
    if (L.nv > 0) {
        unsigned blocks = (unsigned)((L.nv + 255) / 256);
        k_prep_vertices<<<blocks, 256, 0, st>>>(L.g, L.nv, px, py, pz, rho, L.verts, &L.ctr->flags);
    }
    return cudaGetLastError();
}

cudaError_t launch_project(const LaunchArgs& L, int fp32, cudaStream_t st, cudaEvent_t mid) {
    if (L.ns == 0) {
        if (mid) cudaEventRecord(mid, st);
        return cudaSuccess;
    }
    return fp32 ? launch_typed<float>(L, st, mid) : launch_typed<double>(L, st, mid);
}

}  // namespace cdp
