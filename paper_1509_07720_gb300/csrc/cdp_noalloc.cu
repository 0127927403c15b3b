// Projection entry point that allocates nothing (declared in include/coldproj.h as
// cdp_project_noalloc).  Its scratch (the per-call counters, the vertex records, the lists of the
// large, deferred and clipped simplices and the geometry records of one batch of 16,384
// tetrahedra) is one statically sized device array of this module instead of context-owned memory;
// the kernels are the ones cdp_project launches.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/coldproj.h"
#include "cdp_project.h"

namespace cdp {
int check_problem_args(const cdp_problem* p);
int build_table(const cdp_problem* const* probs, int n, ProbTable& T);
}

namespace {

constexpr long long kMaxVerts = CDP_NOALLOC_MAX_VERTS;
constexpr long long kMaxSimplices = CDP_NOALLOC_MAX_SIMPLICES;
constexpr size_t kCounterBytes = 1024;  // the counters, padded so that the records stay 256-aligned
constexpr long long kGeoBatch = 16384;  // tetrahedra set up per batch
constexpr size_t kGeoRec = sizeof(cdp::TetGeo<double>) > sizeof(cdp::TetGeo<float>) ? sizeof(cdp::TetGeo<double>)
                                                                                     : sizeof(cdp::TetGeo<float>);
constexpr size_t kListOffset = kCounterBytes + (size_t)kMaxVerts * sizeof(cdp::VertexRec);
constexpr size_t kDeferOffset = kListOffset + (size_t)kMaxSimplices * sizeof(int);
constexpr size_t kClipOffset = kDeferOffset + (size_t)kMaxSimplices * sizeof(int);
constexpr size_t kNeedOffset = kClipOffset + (size_t)kMaxSimplices * sizeof(int);
constexpr size_t kGeoOffset = (kNeedOffset + (size_t)kGeoBatch * sizeof(int) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kGeoOffset + (size_t)kGeoBatch * kGeoRec;
static_assert(sizeof(cdp::Counters) <= kCounterBytes, "counters do not fit their slot");
static_assert(kScratchBytes == CDP_NOALLOC_SCRATCH_BYTES, "the static scratch differs from the size the header states");

// [counters | vertex records | list of large tetrahedra | deferred list | clip list | box sizes |
//  geometry records of one batch]; shared by every call on the device
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

// per-device launch parameters and the scratch address, filled once with the device current
struct DeviceSetup {
    bool ready;
    unsigned char* scratch;
    int num_sms;
    int blocks[2][2];  // [dim == 3][fp32]: resident blocks per SM of the projection kernel
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_lock;

int setup_device(int dev, DeviceSetup** out) {
    if (dev < 0 || dev >= kMaxDevices) return CDP_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_lock);
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return CDP_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cdp::configure_all() != cudaSuccess) {
            cudaGetLastError();
            return CDP_ERR_CUDA;
        }
        s.scratch = (unsigned char*)ptr;
        s.num_sms = sms;
        for (int d3 = 0; d3 < 2; ++d3)
            for (int f = 0; f < 2; ++f) s.blocks[d3][f] = cdp::resident_blocks(d3 ? 3 : 2, f);
        s.ready = true;
    }
    *out = &s;
    return CDP_OK;
}

}  // namespace

extern "C" int cdp_project_noalloc(const cdp_problem* p, int precision, int accumulate, uint32_t* error_flags,
                                   void* stream) {
    int rc = cdp::check_problem_args(p);
    if (rc) return rc;
    {
        int f = 0, a = 0;
        if (!cdp::parse_precision(precision, &f, &a)) return CDP_ERR_ARG;
    }
    if (p->n_verts > kMaxVerts || p->n_simplices > kMaxSimplices) return CDP_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    DeviceSetup* s = nullptr;
    if ((rc = setup_device(dev, &s))) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    cdp::LaunchArgs L;
    memset(&L, 0, sizeof(L));
    if ((rc = cdp::build_table(&p, 1, L.T))) return rc;
    L.ctr = (cdp::Counters*)s->scratch;
    L.verts = (cdp::VertexRec*)(s->scratch + kCounterBytes);
    L.stats = nullptr;
    L.num_sms = s->num_sms;
    int fp32 = 0, accuracy = 1;
    cdp::parse_precision(precision, &fp32, &accuracy);
    L.accuracy = accuracy;
    L.small_blocks_per_sm = 8 * s->blocks[p->dim == 3][fp32];
    L.resident_per_sm = s->blocks[p->dim == 3][fp32];
    L.big_list = (int*)(s->scratch + kListOffset);
    L.big_cap = kMaxSimplices;
    L.defer_list = (int*)(s->scratch + kDeferOffset);
    L.defer_cap = kMaxSimplices;
    L.clip_list = (int*)(s->scratch + kClipOffset);
    L.clip_cap = kMaxSimplices;
    L.need = (int*)(s->scratch + kNeedOffset);
    L.geo = s->scratch + kGeoOffset;
    L.geo_bytes = (size_t)kGeoBatch * kGeoRec;
    L.geo_cap = kGeoBatch;

    // every counter, the error word included, starts at zero on each call
    if (cudaMemsetAsync(s->scratch, 0, sizeof(cdp::Counters), st) != cudaSuccess) return CDP_ERR_CUDA;
    if (!accumulate && cudaMemsetAsync(p->cell_mass, 0, (size_t)L.T.ncells * sizeof(double), st) != cudaSuccess)
        return CDP_ERR_CUDA;
    if (cdp::launch_prep(L, st) != cudaSuccess ||
        cdp::launch_project(L, fp32, st, nullptr, nullptr) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_CUDA;
    }
    if (error_flags &&
        cudaMemcpyAsync(error_flags, &L.ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return CDP_ERR_CUDA;
    return CDP_OK;
}
