// Kernels of the projection (Sect. 3; Algorithm 2 organised per simplex instead of per vertex).
//
//  k_prep_vertices   one thread per vertex: world coordinates -> 32-byte fixed-point records.
//  k_project{3,2}    one thread per simplex: canonicalise; a simplex inside one cell deposits
//                    |V| mean(rho) there (Algorithm 2, step 1); a simplex whose bounding box has at
//                    most CDP_ONE_THREAD_CELLS cells is projected by the same thread; larger ones
//                    are queued.
//  k_tiled{3,2}      persistent warps take 32 queued simplices at a time, split each bounding box
//                    into tiles of CDP_TILE^D cells and give the (simplex, tile) units of the 32
//                    simplices to the 32 lanes in turn, so that every lane is busy.
//
// Every unit accumulates its (simplex, cell) pieces in a private 64-entry open-addressing table
// in shared memory (cell key -> partial mass), then flushes one FP64 atomic per piece.  A table
// that fills up sends further new cells straight to the grid (correct, just slower).
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

// Mass closure of the FP32-mixed path (not in the paper): the FP64 closed-form mass of a simplex
// minus the sum of its FP32 pieces is added to its largest piece, so that the total mass is exact
// to FP64 rounding.  `Closure` gathers the sum (compensated, in FP32) and the largest piece.
struct Closure {
    float s, c;      // Kahan sum of the flushed pieces
    float vmax;      // largest |piece| so far
    long long imax;  // its cell (flat index, -1 none)
    __device__ __forceinline__ void reset() {
        s = c = vmax = 0.f;
        imax = -1;
    }
    __device__ __forceinline__ void add(float v, long long idx) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
        float a = fabsf(v);
        if (a > vmax) {
            vmax = a;
            imax = idx;
        }
    }
    __device__ __forceinline__ double total() const { return (double)s - (double)c; }
};

constexpr int HASH_SLOTS = 64;
constexpr int HASH_FILL = 48;  // at most this many distinct cells per unit are kept in the table

// Per-thread piece table: slot i of thread t lives at keys[i * CDP_BLOCK + t] (conflict-free).
// The occupancy is a 64-bit mask in registers, so nothing has to be cleared between units.
template <typename R>
struct PieceTable {
    int* keys;
    R* vals;
    unsigned long long occ;
    int count;
    // unit frame: key = x + ex * (y + ey * z), cell (x, y, z) relative to the tile origin
    int ex, ey;
    // direct path for cells that do not fit
    const GridDesc* g;
    int base[3];  // absolute cell of the tile origin
    double* out;
    Closure* cl;

    __device__ __forceinline__ void direct(int x, int y, int z, R v) {
        long long idx = flat_cell(*g, base[0] + x, base[1] + y, base[2] + z);
        if (idx >= 0) {
            atomicAdd(out + idx, (double)v);
            if (cl) cl->add((float)v, idx);
        }
    }

    __device__ __forceinline__ void operator()(int x, int y, int z, R v) {
        int key = x + ex * (y + ey * z);
        unsigned h = ((unsigned)key * 2654435761u) >> 26;
        for (int p = 0; p < HASH_SLOTS; ++p) {
            unsigned i = (h + p) & (HASH_SLOTS - 1);
            if (!((occ >> i) & 1ull)) {
                if (count >= HASH_FILL) break;
                occ |= 1ull << i;
                ++count;
                keys[i * CDP_BLOCK] = key;
                vals[i * CDP_BLOCK] = v;
                return;
            }
            if (keys[i * CDP_BLOCK] == key) {
                vals[i * CDP_BLOCK] += v;
                return;
            }
        }
        direct(x, y, z, v);
    }

    __device__ __forceinline__ void flush() {
        unsigned long long m = occ;
        while (m) {
            int i = __ffsll((long long)m) - 1;
            m &= m - 1;
            int key = keys[i * CDP_BLOCK];
            R v = vals[i * CDP_BLOCK];
            if (v == R(0)) continue;
            int x = key % ex, r = key / ex;
            int y = r % ey, z = r / ey;
            long long idx = flat_cell(*g, base[0] + x, base[1] + y, base[2] + z);
            if (idx >= 0) {
                atomicAdd(out + idx, (double)v);
                if (cl) cl->add((float)v, idx);
            }
        }
        occ = 0;
        count = 0;
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

template <typename R>
__device__ __forceinline__ PieceTable<R> make_table(unsigned char* smem, const GridDesc& g, double* out, Closure* cl) {
    PieceTable<R> t;
    t.keys = reinterpret_cast<int*>(smem) + threadIdx.x;
    t.vals = reinterpret_cast<R*>(smem + (size_t)HASH_SLOTS * CDP_BLOCK * sizeof(int)) + threadIdx.x;
    t.occ = 0;
    t.count = 0;
    t.ex = t.ey = 1;
    t.base[0] = t.base[1] = t.base[2] = 0;
    t.g = &g;
    t.out = out;
    t.cl = cl;
    return t;
}

// Project the part of tetrahedron S inside tile T (td cells, relative to the anchor) and flush it.
template <typename R>
__device__ void tet_tile(const Tet& S, const int T[3], const int td[3], PieceTable<R>& tab, UnitCounts* cnt) {
    TetGeo<R> G;
    tet_setup(S, T, G);
    tab.ex = td[0];
    tab.ey = td[1];
    for (int a = 0; a < 3; ++a) tab.base[a] = S.anchor[a] + T[a];
    tet_unit(G, td, tab, cnt);
    tab.flush();
}

template <typename R>
__device__ void tri_tile(const Tri& S, const int T[2], const int td[2], PieceTable<R>& tab, UnitCounts* cnt) {
    TriGeo<R> G;
    tri_setup(S, T, G);
    tab.ex = td[0];
    tab.ey = td[1];
    tab.base[0] = S.anchor[0] + T[0];
    tab.base[1] = S.anchor[1] + T[1];
    tab.base[2] = 0;
    tri_unit(G, td, tab, cnt);
    tab.flush();
}

__device__ __forceinline__ void close_mass(double* __restrict__ out, double exact, const Closure& cl) {
    if (cl.imax >= 0) atomicAdd(out + cl.imax, exact - cl.total());
}

// ------------------------------------------------------------------------------------------
// one thread per simplex
// ------------------------------------------------------------------------------------------
template <int DIM, typename R>
__global__ void __launch_bounds__(CDP_BLOCK) k_project(GridDesc g, long long ns, long long nv,
                                                       const int* __restrict__ simp,
                                                       const VertexRec* __restrict__ V, double* __restrict__ out,
                                                       int* __restrict__ queue, Counters* __restrict__ ctr,
                                                       UnitCounts* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    UnitCounts cnt = {0, 0, 0, 0, 0};
    UnitCounts* pc = stats ? &cnt : nullptr;
    unsigned long long n0 = 0, nsmall = 0, nzero = 0;
    constexpr bool fp32 = sizeof(R) == 4;
    Closure cl;
    cl.reset();
    PieceTable<R> tab = make_table<R>(smem_raw, g, out, fp32 ? &cl : nullptr);
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
         s += (long long)gridDim.x * blockDim.x) {
        const VertexRec* v[4];
        if (!fetch_vertices(simp, s, DIM + 1, nv, V, v)) {
            atomicOr(&ctr->flags, CDP_FLAG_INDEX);
            continue;
        }
        if (DIM == 3) {
            Tet S;
            unsigned rc = canon_tet(g, v, S);
            if (rc) {
                if (rc == 1)
                    ++nzero;
                else
                    atomicOr(&ctr->flags, rc);
                continue;
            }
            int td[3] = {S.hi[0] - S.lo[0] + 1, S.hi[1] - S.lo[1] + 1, S.hi[2] - S.lo[2] + 1};
            int nc = td[0] * td[1] * td[2];
            if (nc == 1) {
                long long idx = flat_cell(g, S.anchor[0] + S.lo[0], S.anchor[1] + S.lo[1], S.anchor[2] + S.lo[2]);
                if (idx >= 0) atomicAdd(out + idx, tet_mass_cells(S));
                ++n0;
                continue;
            }
            if (nc > CDP_ONE_THREAD_CELLS) {
                queue[atomicAdd(&ctr->big_count, 1u)] = (int)s;
                continue;
            }
            cl.reset();
            tet_tile<R>(S, S.lo, td, tab, pc);
            if (fp32) close_mass(out, tet_mass_cells(S), cl);
        } else {
            Tri S;
            unsigned rc = canon_tri(g, v, S);
            if (rc) {
                if (rc == 1)
                    ++nzero;
                else
                    atomicOr(&ctr->flags, rc);
                continue;
            }
            int td[2] = {S.hi[0] - S.lo[0] + 1, S.hi[1] - S.lo[1] + 1};
            int nc = td[0] * td[1];
            if (nc == 1) {
                long long idx = flat_cell(g, S.anchor[0] + S.lo[0], S.anchor[1] + S.lo[1], 0);
                if (idx >= 0) atomicAdd(out + idx, tri_mass_cells(S));
                ++n0;
                continue;
            }
            if (nc > CDP_ONE_THREAD_CELLS) {
                queue[atomicAdd(&ctr->big_count, 1u)] = (int)s;
                continue;
            }
            cl.reset();
            tri_tile<R>(S, S.lo, td, tab, pc);
            if (fp32) close_mass(out, tri_mass_cells(S), cl);
        }
        ++nsmall;
    }
    if (stats) {
        add_counts(stats, cnt);
        if (n0) atomicAdd(&ctr->n_class0, n0);
        if (nsmall) atomicAdd(&ctr->n_small, nsmall);
        if (nzero) atomicAdd(&ctr->n_zero, nzero);
    }
}

// ------------------------------------------------------------------------------------------
// tiled simplices: warps over chunks of 32 queued simplices, lanes over their (simplex, tile) units
// ------------------------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ int tile_count(const int lo[3], const int hi[3], int nt[3]) {
    int n = 1;
    for (int a = 0; a < DIM; ++a) {
        nt[a] = (hi[a] - lo[a]) / CDP_TILE + 1;
        n *= nt[a];
    }
    return n;
}

template <int DIM, typename R>
__global__ void __launch_bounds__(CDP_BLOCK) k_tiled(GridDesc g, long long nv, const int* __restrict__ simp,
                                                     const VertexRec* __restrict__ V, double* __restrict__ out,
                                                     const int* __restrict__ queue, Counters* __restrict__ ctr,
                                                     UnitCounts* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool fp32 = sizeof(R) == 4;
    // per-warp closure state of the 32 simplices of the current chunk
    const size_t tab_bytes = (size_t)HASH_SLOTS * CDP_BLOCK * (sizeof(int) + sizeof(R));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* wsum = reinterpret_cast<double*>(smem_raw + tab_bytes) + warp * 32;
    unsigned long long* wmax =
        reinterpret_cast<unsigned long long*>(smem_raw + tab_bytes + (CDP_BLOCK / 32) * 32 * sizeof(double)) +
        warp * 32;
    UnitCounts cnt = {0, 0, 0, 0, 0};
    UnitCounts* pc = stats ? &cnt : nullptr;
    unsigned long long ntiles = 0;
    Closure cl;
    cl.reset();
    PieceTable<R> tab = make_table<R>(smem_raw, g, out, fp32 ? &cl : nullptr);
    const unsigned total = ctr->big_count;
    while (true) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&ctr->big_next, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        // this lane's simplex of the chunk, its tile count and its exact mass
        unsigned e = base + lane;
        int mytiles = 0;
        double exact = 0.0;
        int sid = 0;
        if (e < total) {
            sid = queue[e];
            const VertexRec* v[4];
            fetch_vertices(simp, sid, DIM + 1, nv, V, v);
            int nt[3];
            if (DIM == 3) {
                Tet S;
                canon_tet(g, v, S);  // succeeded in k_project
                mytiles = tile_count<3>(S.lo, S.hi, nt);
                if (fp32) exact = tet_mass_cells(S);
            } else {
                Tri S;
                canon_tri(g, v, S);
                mytiles = tile_count<2>(S.lo, S.hi, nt);
                if (fp32) exact = tri_mass_cells(S);
            }
        }
        wsum[lane] = 0.0;
        wmax[lane] = 0ull;
        // inclusive scan of the tile counts over the chunk
        int pre = mytiles;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += t;
        }
        const int tot = __shfl_sync(0xffffffffu, pre, 31);
        __syncwarp();
        for (int u0 = 0; u0 < tot; u0 += 32) {
            const int u = u0 + lane;
            // owner lane: the first lane whose inclusive prefix exceeds u
            int own = 0;
            for (int step = 16; step > 0; step >>= 1) {
                int p = __shfl_sync(0xffffffffu, pre, own + step - 1);
                if (p <= u) own += step;
            }
            own = own > 31 ? 31 : own;
            const int before = __shfl_sync(0xffffffffu, pre - mytiles, own);
            const int osid = __shfl_sync(0xffffffffu, sid, own);
            if (u < tot) {
                const int t = u - before;
                const VertexRec* v[4];
                fetch_vertices(simp, osid, DIM + 1, nv, V, v);
                cl.reset();
                if (DIM == 3) {
                    Tet S;
                    canon_tet(g, v, S);
                    int nt[3];
                    tile_count<3>(S.lo, S.hi, nt);
                    int T[3], td[3];
                    T[0] = S.lo[0] + (t % nt[0]) * CDP_TILE;
                    T[1] = S.lo[1] + ((t / nt[0]) % nt[1]) * CDP_TILE;
                    T[2] = S.lo[2] + (t / (nt[0] * nt[1])) * CDP_TILE;
                    for (int a = 0; a < 3; ++a) {
                        td[a] = S.hi[a] - T[a] + 1;
                        if (td[a] > CDP_TILE) td[a] = CDP_TILE;
                    }
                    tet_tile<R>(S, T, td, tab, pc);
                } else {
                    Tri S;
                    canon_tri(g, v, S);
                    int nt[3];
                    tile_count<2>(S.lo, S.hi, nt);
                    int T[2], td[2];
                    T[0] = S.lo[0] + (t % nt[0]) * CDP_TILE;
                    T[1] = S.lo[1] + (t / nt[0]) * CDP_TILE;
                    for (int a = 0; a < 2; ++a) {
                        td[a] = S.hi[a] - T[a] + 1;
                        if (td[a] > CDP_TILE) td[a] = CDP_TILE;
                    }
                    tri_tile<R>(S, T, td, tab, pc);
                }
                ++ntiles;
                if (fp32) {
                    atomicAdd(&wsum[own], cl.total());
                    if (cl.imax >= 0) {
                        unsigned long long packed = ((unsigned long long)__float_as_uint(cl.vmax) << 32) |
                                                    (unsigned long long)(unsigned)cl.imax;
                        atomicMax(&wmax[own], packed);
                    }
                }
            }
        }
        __syncwarp();
        if (fp32 && e < total && wmax[lane] != 0ull) {
            long long idx = (long long)(unsigned)(wmax[lane] & 0xffffffffull);
            atomicAdd(out + idx, exact - wsum[lane]);
        }
        __syncwarp();
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
static size_t shared_bytes(bool tiled) {
    size_t b = (size_t)HASH_SLOTS * CDP_BLOCK * (sizeof(int) + sizeof(R));
    if (tiled) b += (size_t)(CDP_BLOCK / 32) * 32 * (sizeof(double) + sizeof(unsigned long long));
    return b;
}

template <typename R>
static cudaError_t configure_kernels() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_project<3, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shared_bytes<R>(false))))
        return e;
    if ((e = cudaFuncSetAttribute(k_project<2, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shared_bytes<R>(false))))
        return e;
    if ((e = cudaFuncSetAttribute(k_tiled<3, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shared_bytes<R>(true))))
        return e;
    if ((e = cudaFuncSetAttribute(k_tiled<2, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shared_bytes<R>(true))))
        return e;
    return cudaSuccess;
}

cudaError_t configure_all() {
    cudaError_t e = configure_kernels<float>();
    if (e) return e;
    return configure_kernels<double>();
}

template <int DIM, typename R>
static cudaError_t launch_dim(const LaunchArgs& L, cudaStream_t st, cudaEvent_t mid) {
    long long blocks = (L.ns + CDP_BLOCK - 1) / CDP_BLOCK;
    long long cap = (long long)L.num_sms * L.small_blocks_per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_project<DIM, R><<<(unsigned)blocks, CDP_BLOCK, shared_bytes<R>(false), st>>>(
        L.g, L.ns, L.nv, L.simplices, L.verts, L.out, L.queue, L.ctr, L.stats);
    if (mid) cudaEventRecord(mid, st);
    k_tiled<DIM, R><<<L.num_sms * L.big_blocks_per_sm, CDP_BLOCK, shared_bytes<R>(true), st>>>(
        L.g, L.nv, L.simplices, L.verts, L.out, L.queue, L.ctr, L.stats);
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
    if (L.g.dim == 3) return fp32 ? launch_dim<3, float>(L, st, mid) : launch_dim<3, double>(L, st, mid);
    return fp32 ? launch_dim<2, float>(L, st, mid) : launch_dim<2, double>(L, st, mid);
}

}  // namespace cdp
