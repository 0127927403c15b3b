// C-ABI entry points (declared in include/coldproj.h): argument checking, scratch management and
// the launch sequence of the projection.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/coldproj.h"
#include "cdp_project.h"

#include "cdp_ctx.h"

namespace {

struct DeviceGuard {
    int prev;
    bool changed;
    explicit DeviceGuard(int dev) : prev(0), changed(false) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

int flags_to_code(unsigned f) {
    if (f & cdp::CDP_FLAG_INDEX) return CDP_ERR_INDEX;
    if (f & cdp::CDP_FLAG_NAN) return CDP_ERR_NAN;
    if (f & cdp::CDP_FLAG_EXTENT) return CDP_ERR_EXTENT;
    return CDP_OK;
}

// grow a scratch buffer of the context; a reallocation moves the buffer, so it advances the
// context's epoch (the captured time steps recorded with the old address are then not replayed)
template <typename T>
int grow(cdp_ctx* c, T** p, size_t* cap, size_t need) {
    if (need <= *cap) return CDP_OK;
    ++c->epoch;
    size_t n = need + need / 4 + 1024;
    T* q = nullptr;
    if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_OOM;
    }
    if (*p) cudaFree(*p);
    *p = q;
    *cap = n;
    return CDP_OK;
}

int check_problem(const cdp_problem* p) {
    if (!p) return CDP_ERR_ARG;
    if (p->dim != 2 && p->dim != 3) return CDP_ERR_ARG;
    if (p->n_verts < 0 || p->n_simplices < 0 || p->n_verts > (int64_t)0x7fffffff ||
        p->n_simplices > (int64_t)0x7fffffff)
        return CDP_ERR_ARG;
    if (!p->cell_mass) return CDP_ERR_ARG;
    for (int a = 0; a < p->dim; ++a) {
        if (p->grid[a] < 1 || p->grid[a] > (1 << 20)) return CDP_ERR_ARG;
        if (!(p->box_len[a] > 0.0) || !(p->box_len[a] < 1e300)) return CDP_ERR_ARG;
        if (!(p->box_lo[a] == p->box_lo[a])) return CDP_ERR_ARG;
        if (p->n_verts > 0 && !p->pos[a]) return CDP_ERR_ARG;
    }
    if (p->n_simplices > 0 && (!p->simplices || !p->rho || p->n_verts == 0)) return CDP_ERR_ARG;
    if (p->n_verts > 0 && !p->rho) return CDP_ERR_ARG;
    long long cells = 1;
    for (int a = 0; a < p->dim; ++a) {
        cells *= p->grid[a];
        if (cells > ((long long)1 << 32)) return CDP_ERR_ARG;
    }
    return CDP_OK;
}

cudaEvent_t take_event(cdp_ctx* c) {
    if (!c->pool->empty()) {
        cudaEvent_t e = c->pool->back();
        c->pool->pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// fold the recorded event groups into the totals (synchronises on them)
int fold_timing(cdp_ctx* c) {
    std::vector<cudaEvent_t>& p = *c->pending;
    constexpr int T = cdp::CDP_TEV;
    for (size_t i = 0; i + T - 1 < p.size(); i += T) {
        if (cudaEventSynchronize(p[i + T - 1]) != cudaSuccess) {
            cudaGetLastError();
            return CDP_ERR_CUDA;
        }
        for (int k = 0; k < T - 1; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p[i + k], p[i + k + 1]) == cudaSuccess) c->totals[k] += ms;
            cudaGetLastError();
        }
        c->calls += 1;
    }
    for (cudaEvent_t e : p) c->pool->push_back(e);
    p.clear();
    return CDP_OK;
}

// largest batch of tetrahedra whose geometry records are held at once
constexpr size_t kGeoBatch = (size_t)1 << 24;

// geometry records and box sizes for min(ns, kGeoBatch) tetrahedra (both precisions)
int grow_geo(cdp_ctx* c, size_t ns) {
    size_t n = ns < kGeoBatch ? ns : kGeoBatch;
    if (n < 1) n = 1;
    size_t rec = cdp::tet_geo_bytes(0) > cdp::tet_geo_bytes(1) ? cdp::tet_geo_bytes(0) : cdp::tet_geo_bytes(1);
    int rc = grow(c, &c->geo, &c->geo_cap, n * rec);
    if (rc) return rc;
    return grow(c, &c->need, &c->need_cap, n);
}

// the slots in which each block of the FP32 large-tetrahedron kernel keeps its tiles' pieces
// between the two passes (CDP_TILE_STORE_PER_BLOCK tiles per resident block)
int grow_tiles(cdp_ctx* c) {
    const size_t blocks = (size_t)c->num_sms * (size_t)(c->blocks_small[1] > 0 ? c->blocks_small[1] : 1);
    return grow(c, &c->tiles, &c->tiles_cap, blocks * cdp::CDP_TILE_STORE_PER_BLOCK * cdp::tet_tile_cells());
}

}  // namespace

namespace cdp {

// argument check of one problem, for the entry points defined in other translation units
int check_problem_args(const cdp_problem* p) { return check_problem(p); }

// grow the scratch to hold the groups of `n` problems (allocation happens here, never inside a
// captured sequence): every buffer sized for the totals of all the problems, at least what any of
// their groups needs
int reserve_scratch(cdp_ctx* c, const cdp_problem* probs, int n) {
    size_t nv = 1, ns = 1;
    bool any3d = false;
    for (int i = 0; i < n; ++i) {
        nv += (size_t)probs[i].n_verts;
        ns += (size_t)probs[i].n_simplices + 64;  // (with the chunk alignment of each problem)
        any3d = any3d || probs[i].dim == 3;
    }
    int rc = grow(c, &c->verts, &c->verts_cap, nv);
    if (rc) return rc;
    if ((rc = grow(c, &c->queue, &c->queue_cap, ns))) return rc;
    if ((rc = grow(c, &c->defer, &c->defer_cap, ns)) || (rc = grow(c, &c->clip, &c->clip_cap, ns))) return rc;
    if (any3d && (rc = grow_tiles(c))) return rc;
    return grow_geo(c, ns);
}

// scratch of an AMR projection: the coarse levels' grids and the level of every simplex
int reserve_amr(cdp_ctx* c, size_t coarse_cells, size_t n_simplices) {
    int rc = grow(c, &c->amr, &c->amr_cap, coarse_cells > 0 ? coarse_cells : 1);
    return rc ? rc : grow(c, &c->levels, &c->levels_cap, n_simplices > 0 ? n_simplices : 1);
}

// the table of a group of problems of one dimension (at most CDP_GROUP, arguments already checked):
// their grids, pointers and offsets in the group's vertex, simplex and cell numberings.  Each
// problem's simplices start at a multiple of the chunk size (3D), so that no chunk of the main
// kernel mixes two problems.  CDP_ERR_ARG when the group's simplex numbering exceeds 2^31 - 1.
int build_table(const cdp_problem* const* probs, int n, ProbTable& T) {  // (also used by cdp_noalloc.cu)
    memset(&T, 0, sizeof(T));
    T.n = n;
    T.dim = probs[0]->dim;
    const long long align = T.dim == 3 ? 64 : 1;
    long long nv = 0, ns = 0, nc = 0;
    for (int i = 0; i < n; ++i) {
        const cdp_problem* p = probs[i];
        ProbEntry& e = T.p[i];
        GridDesc& g = e.g;
        g.dim = p->dim;
        g.periodic = p->periodic ? 1 : 0;
        double cellvol = 1.0;
        long long cells = 1;
        for (int a = 0; a < 3; ++a) {
            if (a < p->dim) {
                g.n[a] = p->grid[a];
                g.lo[a] = p->box_lo[a];
                g.inv_h[a] = (double)p->grid[a] / p->box_len[a];
                cellvol *= p->box_len[a] / (double)p->grid[a];
                cells *= p->grid[a];
            } else {
                g.n[a] = 1;
                g.lo[a] = 0.0;
                g.inv_h[a] = 1.0;
            }
        }
        g.cell_volume = cellvol;
        e.simplices = p->simplices;
        e.out = p->cell_mass;
        for (int a = 0; a < 3; ++a) e.pos[a] = a < p->dim ? p->pos[a] : nullptr;
        e.rho = p->rho;
        e.nv = p->n_verts;
        e.ns = p->n_simplices;
        e.v_off = nv;
        e.s_off = (ns + align - 1) / align * align;
        e.c_off = nc;
        nv += p->n_verts;
        ns = e.s_off + p->n_simplices;
        nc += cells;
    }
    T.nv = nv;
    T.ns = ns;
    T.ncells = nc;
    return ns <= (long long)0x7fffffff ? CDP_OK : CDP_ERR_ARG;
}

// enqueue the projection of one group on `st` (arguments already checked; a single projection is a
// group of one).  With `amr_levels`, the group is the levels 0 .. max_level of one mesh (an AMR
// projection, cdp_amr.cu): the level of every simplex is written there after the vertex records,
// and every entry sets up the simplices of its own level only.
int project_group(cdp_ctx* c, const ProbTable& T, int precision, int accumulate, cudaStream_t st, bool want_stats,
                  unsigned char* amr_levels = nullptr, int max_level = 0) {
    int rc;
    const size_t nv1 = (size_t)(T.nv > 0 ? T.nv : 1), ns1 = (size_t)(T.ns > 0 ? T.ns : 1);
    if ((rc = grow(c, &c->verts, &c->verts_cap, nv1))) return rc;
    if ((rc = grow(c, &c->defer, &c->defer_cap, ns1)) || (rc = grow(c, &c->clip, &c->clip_cap, ns1))) return rc;
    int fp32 = 0, accuracy = 1;
    if (!parse_precision(precision, &fp32, &accuracy)) return CDP_ERR_ARG;
    if (T.dim == 3 && ((rc = grow(c, &c->queue, &c->queue_cap, ns1)) || (rc = grow_geo(c, ns1)))) return rc;
    if (T.dim == 3 && fp32 && (rc = grow_tiles(c))) return rc;

    LaunchArgs L;
    memset(&L, 0, sizeof(L));
    L.T = T;
    L.accuracy = accuracy;
    L.verts = c->verts;
    L.ctr = c->ctr;
    L.stats = want_stats ? c->stats : nullptr;
    L.num_sms = c->num_sms;
    // a persistent grid: every resident block slot of the device, grid_mult times over
    L.small_blocks_per_sm =
        c->grid_mult[T.dim == 3][fp32] * (T.dim == 3 ? c->blocks_small[fp32] : c->blocks_big[fp32]);
    L.resident_per_sm = T.dim == 3 ? c->blocks_small[fp32] : c->blocks_big[fp32];
    L.max_cells = c->max_cells[fp32];
    L.tile_edge = c->tile_edge[fp32];
    L.big_list = c->queue;
    L.big_cap = (long long)c->queue_cap;
    L.geo = c->geo;
    L.geo_bytes = c->geo_cap;
    L.need = c->need;
    L.tile_store = c->tiles;
    L.tile_store_cap = c->tiles_cap;
    L.tile_store_per_block = cdp::CDP_TILE_STORE_PER_BLOCK;
    L.defer_list = c->defer;
    L.defer_cap = (long long)c->defer_cap;
    L.clip_list = c->clip;
    L.clip_cap = (long long)c->clip_cap;
    {
        size_t rec = cdp::tet_geo_bytes(fp32);
        long long by_bytes = rec ? (long long)(c->geo_cap / rec) : 0;
        L.geo_cap = by_bytes < (long long)c->need_cap ? by_bytes : (long long)c->need_cap;
    }

    // zero the per-call counters (the sticky error word at offset 0 is kept)
    if (cudaMemsetAsync((char*)c->ctr + sizeof(unsigned), 0, sizeof(Counters) - sizeof(unsigned), st) !=
        cudaSuccess)
        return CDP_ERR_CUDA;
    if (want_stats && cudaMemsetAsync(c->stats, 0, 2 * sizeof(UnitCounts), st) != cudaSuccess) return CDP_ERR_CUDA;
    if (!accumulate)
        for (int i = 0; i < T.n; ++i) {
            const long long cells = (i + 1 < T.n ? T.p[i + 1].c_off : T.ncells) - T.p[i].c_off;
            if (cudaMemsetAsync(T.p[i].out, 0, (size_t)cells * sizeof(double), st) != cudaSuccess) return CDP_ERR_CUDA;
        }
    constexpr int TE = CDP_TEV;
    cudaEvent_t ev[TE] = {};
    if (c->timing) {
        if (c->pending->size() >= 4096) fold_timing(c);
        bool ok = true;
        for (int k = 0; k < TE; ++k) ok = (ev[k] = take_event(c)) != nullptr && ok;
        if (!ok) {
            for (int k = 0; k < TE; ++k)
                if (ev[k]) c->pool->push_back(ev[k]);
            return CDP_ERR_CUDA;
        }
        cudaEventRecord(ev[0], st);
    }
    if (launch_prep(L, st) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    if (amr_levels) {
        if (launch_amr_levels(L, max_level, amr_levels, st) != cudaSuccess) {
            cudaGetLastError();
            return CDP_ERR_CUDA;
        }
        L.levels = amr_levels;
    }
    if (ev[1]) cudaEventRecord(ev[1], st);
    L.ev_acc = ev[4];
    if (launch_project(L, fp32, st, ev[2], ev[3]) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    if (ev[TE - 1]) {
        cudaEventRecord(ev[TE - 1], st);
        for (int k = 0; k < TE; ++k) c->pending->push_back(ev[k]);
    }
    return CDP_OK;
}

// enqueue one projection on `st` (arguments already checked)
int project_enqueue(cdp_ctx* c, const cdp_problem* p, int precision, int accumulate, cudaStream_t st, bool want_stats) {
    ProbTable* T = new (std::nothrow) ProbTable;
    if (!T) return CDP_ERR_OOM;
    int rc = build_table(&p, 1, *T);
    if (rc == CDP_OK) rc = project_group(c, *T, precision, accumulate, st, want_stats);
    delete T;
    return rc;
}

// enqueue the projections of n problems (arguments already checked, accumulate = 0), grouped by
// dimension into groups of at most CDP_GROUP problems: a group is one launch of every kernel of the
// projection
int project_batch(cdp_ctx* c, const cdp_problem* probs, int n, int precision, cudaStream_t st) {
    std::vector<const cdp_problem*> list;
    ProbTable* T = new (std::nothrow) ProbTable;
    if (!T) return CDP_ERR_OOM;
    int rc = CDP_OK;
    for (int dim = 2; dim <= 3 && rc == CDP_OK; ++dim) {
        list.clear();
        for (int i = 0; i < n; ++i)
            if (probs[i].dim == dim) list.push_back(probs + i);
        for (size_t g0 = 0; g0 < list.size() && rc == CDP_OK; g0 += CDP_GROUP) {
            const int m = (int)(list.size() - g0 < (size_t)CDP_GROUP ? list.size() - g0 : (size_t)CDP_GROUP);
            rc = build_table(list.data() + g0, m, *T);
            if (rc == CDP_OK) rc = project_group(c, *T, precision, 0, st, false);
        }
    }
    delete T;
    return rc;
}

}  // namespace cdp

namespace {

double __longlong_as_double_host(unsigned long long bits) {
    double d;
    memcpy(&d, &bits, sizeof(d));
    return d;
}

int read_stats(cdp_ctx* c, cudaStream_t st, cdp_stats* stats) {
    if (cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(cdp::Counters), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(c->h_stats, c->stats, 2 * sizeof(cdp::UnitCounts), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    memset(stats, 0, sizeof(*stats));
    stats->n_zero_volume = c->h_ctr->n_zero;
    stats->n_single_cell = c->h_ctr->n_class0;
    stats->n_small = c->h_ctr->n_small;
    stats->n_large = c->h_ctr->big_first;
    stats->n_deferred = c->h_ctr->defer_count;
    stats->n_clipped = c->h_ctr->clip_count;
    {
        const double m = __longlong_as_double_host(c->h_ctr->mmax_bits[0]);
        const double eb = __longlong_as_double_host(c->h_ctr->ebmax_bits);
        stats->accuracy_bound = m > 0.0 ? eb / m : 0.0;
    }
    stats->n_large_tiles = c->h_ctr->n_big_tiles;
    const cdp::UnitCounts& s0 = c->h_stats[0];
    const cdp::UnitCounts& s1 = c->h_stats[1];
    stats->corners_a = s0.a + s1.a;
    stats->corners_b = s0.b + s1.b;
    stats->corners_c = s0.c + s1.c;
    stats->corners_d = s0.d + s1.d;
    stats->exact_fallbacks = s0.exact + s1.exact;
    stats->large_corners[0] = s1.a;  // found on the tiles of the large tetrahedra
    stats->large_corners[1] = s1.b;
    stats->large_corners[2] = s1.c;
    stats->large_corners[3] = s1.d;
    stats->error_flags = c->h_ctr->flags;
    unsigned f = c->h_ctr->flags;
    if (f && cudaMemsetAsync(c->ctr, 0, sizeof(unsigned), st) != cudaSuccess) return CDP_ERR_CUDA;
    return flags_to_code(f);
}

}  // namespace

namespace cdp {
int read_stats_ctx(cdp_ctx* c, cudaStream_t st, cdp_stats* stats) { return read_stats(c, st, stats); }
}  // namespace cdp

extern "C" {

int cdp_timing_enable(cdp_ctx* c, int enable) {
    if (!c) return CDP_ERR_ARG;
    DeviceGuard guard(c->device);
    int rc = fold_timing(c);
    c->timing = enable ? 1 : 0;
    for (int k = 0; k < cdp::CDP_TEV - 1; ++k) c->totals[k] = 0.0;
    c->calls = 0;
    return rc;
}

int cdp_timing_read(cdp_ctx* c, double* out_ms, int n, int* calls) {
    if (!c || (n > 0 && !out_ms)) return CDP_ERR_ARG;
    DeviceGuard guard(c->device);
    int rc = fold_timing(c);
    if (rc) return rc;
    int m = n < cdp::CDP_TEV - 1 ? n : cdp::CDP_TEV - 1;
    for (int k = 0; k < m; ++k) out_ms[k] = c->totals[k];
    if (calls) *calls = c->calls;
    return m;
}

const char* cdp_strerror(int code) {
    switch (code) {
        case CDP_OK: return "ok";
        case CDP_ERR_ARG: return "invalid argument";
        case CDP_ERR_INDEX: return "vertex index out of range";
        case CDP_ERR_NAN: return "non-finite or out-of-range coordinate or density";
        case CDP_ERR_EXTENT: return "simplex spans half a periodic box or more than 2048 cells";
        case CDP_ERR_OOM: return "device scratch allocation failed";
        case CDP_ERR_TIMEOUT: return "bounded device wait gave up";
        case CDP_ERR_CUDA: return "CUDA error";
        default: return "unknown error";
    }
}

int cdp_create(cdp_ctx** out, int device) {
    if (!out) return CDP_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return CDP_ERR_ARG;
    DeviceGuard guard(device);
    cdp_ctx* c = new (std::nothrow) cdp_ctx;
    if (!c) return CDP_ERR_OOM;
    memset(c, 0, sizeof(*c));
    c->device = device;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cdp::configure_all() != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return CDP_ERR_CUDA;
    }
    // resident blocks per SM of the projection kernel (3D; the 2D kernel is lighter)
    c->blocks_small[0] = cdp::resident_blocks(3, 0);
    c->blocks_small[1] = cdp::resident_blocks(3, 1);
    c->blocks_big[0] = cdp::resident_blocks(2, 0);
    c->blocks_big[1] = cdp::resident_blocks(2, 1);
    for (int d3 = 0; d3 < 2; ++d3)
        for (int f = 0; f < 2; ++f) c->grid_mult[d3][f] = 8;
    if (cudaMalloc(&c->ctr, sizeof(cdp::Counters)) != cudaSuccess ||
        cudaMalloc(&c->stats, 2 * sizeof(cdp::UnitCounts)) != cudaSuccess ||
        cudaMallocHost(&c->h_ctr, sizeof(cdp::Counters)) != cudaSuccess ||
        cudaMallocHost(&c->h_stats, 2 * sizeof(cdp::UnitCounts)) != cudaSuccess) {
        cudaGetLastError();
        cdp_destroy(c);
        return CDP_ERR_OOM;
    }
    c->pending = new (std::nothrow) std::vector<cudaEvent_t>();
    c->pool = new (std::nothrow) std::vector<cudaEvent_t>();
    c->plans = new (std::nothrow) std::vector<cdp::FftPlan>();
    if (!c->pending || !c->pool || !c->plans) {
        cdp_destroy(c);
        return CDP_ERR_OOM;
    }
    if (cudaMemset(c->ctr, 0, sizeof(cdp::Counters)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        cdp_destroy(c);
        return CDP_ERR_CUDA;
    }
    *out = c;
    return CDP_OK;
}

void cdp_destroy(cdp_ctx* c) {
    if (!c) return;
    DeviceGuard guard(c->device);
    cudaDeviceSynchronize();
    if (c->verts) cudaFree(c->verts);
    if (c->queue) cudaFree(c->queue);
    if (c->defer) cudaFree(c->defer);
    if (c->clip) cudaFree(c->clip);
    if (c->geo) cudaFree(c->geo);
    if (c->need) cudaFree(c->need);
    if (c->tiles) cudaFree(c->tiles);
    if (c->amr) cudaFree(c->amr);
    if (c->levels) cudaFree(c->levels);
    if (c->ctr) cudaFree(c->ctr);
    if (c->stats) cudaFree(c->stats);
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    if (c->h_stats) cudaFreeHost(c->h_stats);
    if (c->pending) {
        for (cudaEvent_t e : *c->pending) cudaEventDestroy(e);
        delete c->pending;
    }
    if (c->pool) {
        for (cudaEvent_t e : *c->pool) cudaEventDestroy(e);
        delete c->pool;
    }
    cdp::step_release(c);
    cdp::solver_release(c);
    cudaGetLastError();
    delete c;
}

int cdp_check(cdp_ctx* c, void* stream) {
    if (!c) return CDP_ERR_ARG;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(cdp::Counters), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    unsigned f = c->h_ctr->flags;
    if (f && cudaMemsetAsync(c->ctr, 0, sizeof(unsigned), st) != cudaSuccess) return CDP_ERR_CUDA;
    return flags_to_code(f);
}

int cdp_project(cdp_ctx* c, const cdp_problem* p, int precision, int accumulate, void* stream, cdp_stats* stats) {
    if (!c) return CDP_ERR_ARG;
    int rc = check_problem(p);
    if (rc) return rc;
    {
        int f = 0, a = 0;
        if (!cdp::parse_precision(precision, &f, &a)) return CDP_ERR_ARG;
    }
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    rc = cdp::project_enqueue(c, p, precision, accumulate, st, stats != nullptr);
    if (rc || !stats) return rc;
    return read_stats(c, st, stats);
}

int cdp_autotune(cdp_ctx* c, const cdp_problem* p, int precision, const char* cache_path, int* chosen) {
    if (!c) return CDP_ERR_ARG;
    int rc = check_problem(p);
    if (rc) return rc;
    int fp32 = 0, accuracy = 1;
    if (!cdp::parse_precision(precision, &fp32, &accuracy)) return CDP_ERR_ARG;
    DeviceGuard guard(c->device);
    ++c->epoch;  // the launch shapes may change: captured time steps are recorded again
    const int d3 = p->dim == 3 ? 1 : 0;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
    char key[96];
    snprintf(key, sizeof(key), "sm%d%d-%dsm dim%d %s", major, minor, c->num_sms, p->dim, fp32 ? "fp32mixed" : "fp64");
    const int slots = cdp::tet_box_slots(fp32);
    auto report = [&]() {
        if (chosen) {
            chosen[0] = c->grid_mult[d3][fp32];
            chosen[1] = d3 ? (c->max_cells[fp32] ? c->max_cells[fp32] : cdp::tet_max_cells()) : 0;
            chosen[2] = d3 ? (c->tile_edge[fp32] ? c->tile_edge[fp32] : cdp::tet_tile_edge()) : 0;
        }
    };
    // the cache: lines "<key> <multiplier> <threshold> <tile edge>", the last entry of a key wins
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            char line[200];
            int found = 0, fmc = 0, fte = 0;
            while (fgets(line, sizeof(line), f)) {
                const size_t n = strlen(key);
                int m = 0, mc = 0, te = 0;
                if (strncmp(line, key, n) == 0 && line[n] == ' ' && sscanf(line + n, "%d %d %d", &m, &mc, &te) == 3 &&
                    (m == 1 || m == 2 || m == 4 || m == 8) && mc >= 0 && mc <= slots && (te == 0 || (te >= 4 && te <= cdp::tet_tile_edge()))) {
                    found = m;
                    fmc = mc;
                    fte = te;
                }
            }
            fclose(f);
            if (found) {
                c->grid_mult[d3][fp32] = found;
                if (d3) {
                    c->max_cells[fp32] = fmc;
                    c->tile_edge[fp32] = fte;
                }
                report();
                return CDP_OK;
            }
        }
    }
    // time the projection of this problem (into its own cell_mass) with each setting: one warm-up
    // call and three timed calls each, on a stream of its own, after the work already queued on the
    // device (the problem's inputs may still be in flight on another stream).  The knobs are tuned
    // one after the other (coordinate descent): the grid multiplier, then (3D) the size-class
    // threshold, then the tile edge of the large tetrahedra.
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (st) cudaStreamDestroy(st);
        return CDP_ERR_CUDA;
    }
    const int timing = c->timing;
    c->timing = 0;  // the tuning calls stay out of the per-kernel totals
    const int before[3] = {c->grid_mult[d3][fp32], c->max_cells[fp32], c->tile_edge[fp32]};
    auto time_now = [&](float* ms) -> int {
        int r = cdp::project_enqueue(c, p, precision, 0, st, false);
        if (r == CDP_OK && cudaEventRecord(e0, st) != cudaSuccess) r = CDP_ERR_CUDA;
        for (int k = 0; k < 3 && r == CDP_OK; ++k) r = cdp::project_enqueue(c, p, precision, 0, st, false);
        if (r == CDP_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
            r = CDP_ERR_CUDA;
        return r;
    };
    static const int kMults[] = {1, 2, 4, 8};
    const int kCells[] = {960, 1920, 3840, slots};
    const int kEdges[] = {18, cdp::tet_tile_edge()};
    float best_ms = 0.f;
    bool have = false;
    for (int i = 0; i < 4 && rc == CDP_OK; ++i) {
        const int keep = c->grid_mult[d3][fp32];
        c->grid_mult[d3][fp32] = kMults[i];
        float ms = 0.f;
        rc = time_now(&ms);
        if (rc == CDP_OK && (!have || ms < best_ms)) {
            best_ms = ms;
            have = true;
        } else {
            c->grid_mult[d3][fp32] = keep;
        }
    }
    for (int i = 0; d3 && i < 4 && rc == CDP_OK; ++i) {
        const int keep = c->max_cells[fp32];
        c->max_cells[fp32] = kCells[i];
        float ms = 0.f;
        rc = time_now(&ms);
        if (rc == CDP_OK && ms < best_ms)
            best_ms = ms;
        else
            c->max_cells[fp32] = keep;
    }
    for (int i = 0; d3 && i < 2 && rc == CDP_OK; ++i) {
        const int keep = c->tile_edge[fp32];
        c->tile_edge[fp32] = kEdges[i];
        float ms = 0.f;
        rc = time_now(&ms);
        if (rc == CDP_OK && ms < best_ms)
            best_ms = ms;
        else
            c->tile_edge[fp32] = keep;
    }
    c->timing = timing;
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaGetLastError();
    if (rc) {
        c->grid_mult[d3][fp32] = before[0];
        c->max_cells[fp32] = before[1];
        c->tile_edge[fp32] = before[2];
        return rc;
    }
    report();
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            int ch[3] = {0, 0, 0};
            int* keep_chosen = chosen;
            chosen = ch;
            report();
            chosen = keep_chosen;
            fprintf(f, "%s %d %d %d\n", key, ch[0], ch[1], ch[2]);
            fclose(f);
        }
    }
    return CDP_OK;
}
int cdp_project_batched(cdp_ctx* c, const cdp_problem* probs, int n, int precision, void* stream) {
    if (!c || n < 0 || (n > 0 && !probs)) return CDP_ERR_ARG;
    {
        int f = 0, a = 0;
        if (!cdp::parse_precision(precision, &f, &a)) return CDP_ERR_ARG;
    }
    for (int i = 0; i < n; ++i) {
        int rc = check_problem(probs + i);
        if (rc) return rc;
    }
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cdp::reserve_scratch(c, probs, n);
    if (rc) return rc;
    return cdp::project_batch(c, probs, n, precision, st);
}

}  // extern "C"
