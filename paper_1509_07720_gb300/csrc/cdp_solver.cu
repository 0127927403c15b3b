// The steps around the projection in one time step of the solver (Sect. 4, steps (ii)-(iv)):
// vertex densities from simplex masses, FFT Poisson solve, force interpolation at the vertices,
// kick and drift.  C-ABI entry points declared in include/coldproj.h.
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>
#include <string.h>

#include <new>

#include "../../include/coldproj.h"
#include "cdp_ctx.h"

namespace cdp {

namespace {

struct DevGuard {
    int prev;
    bool changed;
    explicit DevGuard(int dev) : prev(0), changed(false) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DevGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

int check_grid(int dim, const int32_t grid[3], const double box_len[3]) {
    if (dim != 2 && dim != 3) return CDP_ERR_ARG;
    if (!grid || !box_len) return CDP_ERR_ARG;
    long long cells = 1;
    for (int a = 0; a < dim; ++a) {
        if (grid[a] < 1 || grid[a] > (1 << 20)) return CDP_ERR_ARG;
        if (!(box_len[a] > 0.0) || !(box_len[a] < 1e300)) return CDP_ERR_ARG;
        cells *= grid[a];
        if (cells > ((long long)1 << 32)) return CDP_ERR_ARG;
    }
    return CDP_OK;
}

// ---------------------------------------------------------------------------------------------
// Poisson: spectrum of the cell masses times -four_pi_G / (k^2 * cell volume * N), zero mode 0
// ---------------------------------------------------------------------------------------------
// entry t of an (n0, n1, n2h) half spectrum (2D: n1 = 1) times its Green factor
// -four_pi_G / (k^2 * cell volume * N) (`scale` / k^2), the zero mode set to 0
template <typename C, typename R>
__device__ __forceinline__ void green_at(C& v, long long t, int dim, int n0, int n1, int n2h, R k0, R k1, R k2,
                                         R scale) {
    int c = (int)(t % n2h);
    long long r = t / n2h;
    int b = (int)(r % n1);
    int a = (int)(r / n1);
    R kk;
    if (dim == 3) {
        int fa = a <= n0 / 2 ? a : a - n0;
        int fb = b <= n1 / 2 ? b : b - n1;
        R ka = k0 * fa, kb = k1 * fb, kc = k2 * c;
        kk = ka * ka + kb * kb + kc * kc;
    } else {  // 2D: (n0, n1h) with n1 = 1 placeholder: a = row, c = half column
        int fa = a <= n0 / 2 ? a : a - n0;
        R ka = k0 * fa, kc = k2 * c;
        kk = ka * ka + kc * kc;
    }
    R gfac = kk > R(0) ? scale / kk : R(0);
    v.x *= gfac;
    v.y *= gfac;
}

template <typename C, typename R>
__global__ void k_green(C* __restrict__ spec, int dim, int n0, int n1, int n2h, int n2, R k0, R k1, R k2, R scale) {
    long long total = (long long)n0 * n1 * n2h;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x)
        green_at<C, R>(spec[t], t, dim, n0, n1, n2h, k0, k1, k2, scale);
}

// the FP64 source and potential to and from the FP32 transforms' buffer
__global__ void k_to_f32(long long n, const double* __restrict__ x, float* __restrict__ y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}
__global__ void k_to_f64(long long n, const float* __restrict__ x, double* __restrict__ y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

// the single-precision transforms and buffers of a plan (made once)
int add_plan32(FftPlan& p) {
    if (p.have32) return CDP_OK;
    int n[3] = {p.n[0], p.n[1], p.dim == 3 ? p.n[2] : 1};
    size_t cells = 1;
    for (int a = 0; a < p.dim; ++a) cells *= (size_t)n[a];
    if (cudaMalloc(&p.spec32, p.spec_elems * sizeof(cufftComplex)) != cudaSuccess ||
        cudaMalloc(&p.real32, cells * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        if (p.spec32) cudaFree(p.spec32);
        p.spec32 = nullptr;
        p.real32 = nullptr;
        return CDP_ERR_OOM;
    }
    if (cufftPlanMany(&p.r2c32, p.dim, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1) != CUFFT_SUCCESS ||
        cufftPlanMany(&p.c2r32, p.dim, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1) != CUFFT_SUCCESS) {
        cudaFree(p.spec32);
        cudaFree(p.real32);
        p.spec32 = nullptr;
        p.real32 = nullptr;
        return CDP_ERR_CUDA;
    }
    p.have32 = 1;
    return CDP_OK;
}

FftPlan* get_plan(cdp_ctx* c, int dim, const int32_t grid[3], int* rc) {
    for (FftPlan& p : *c->plans) {
        bool same = p.dim == dim;
        for (int a = 0; a < dim; ++a) same = same && p.n[a] == grid[a];
        if (same) return &p;
    }
    FftPlan p;
    memset(&p, 0, sizeof(p));
    p.dim = dim;
    for (int a = 0; a < dim; ++a) p.n[a] = grid[a];
    int n[3] = {grid[0], grid[1], dim == 3 ? grid[2] : 1};
    size_t half = (size_t)(n[dim - 1] / 2 + 1);
    p.spec_elems = (dim == 3 ? (size_t)n[0] * n[1] : (size_t)n[0]) * half;
    if (cudaMalloc(&p.spec, p.spec_elems * sizeof(cufftDoubleComplex)) != cudaSuccess) {
        cudaGetLastError();
        *rc = CDP_ERR_OOM;
        return nullptr;
    }
    if (cufftPlanMany(&p.r2c, dim, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_D2Z, 1) != CUFFT_SUCCESS ||
        cufftPlanMany(&p.c2r, dim, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_Z2D, 1) != CUFFT_SUCCESS) {
        cudaFree(p.spec);
        *rc = CDP_ERR_CUDA;
        return nullptr;
    }
    c->plans->push_back(p);
    return &c->plans->back();
}

// ---------------------------------------------------------------------------------------------
// force: TSC interpolation of the 4-point central difference (Sect. 4.4), periodic grid
// ---------------------------------------------------------------------------------------------
struct ForceGrid {
    int dim;
    int n[3];
    double lo[3], h[3], inv_h[3];
};

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// acceleration at one point x: the triangular-shaped-cloud weights of the 3^DIM cells around it
// times each cell's 4-point central differences of phi.  Both are linear in phi, so along each axis
// the three weighted differences are summed first into one 7-point stencil over the cells
// c0 - 3 .. c0 + 3 (half the FP64 operations and loads of evaluating every cell's differences),
// which is then applied to the 3^(DIM-1) rows of cells the other axes' weights select.
template <int DIM>
__device__ __forceinline__ void force_at(const ForceGrid& G, const double* __restrict__ phi, const double x[3],
                                         double acc[3]) {
    int c0[3] = {0, 0, 0};
    double w[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        double u = (x[a] - G.lo[a]) * G.inv_h[a] - 0.5;
        double f = floor(u + 0.5);
        double d = u - f;
        c0[a] = (int)f;
        w[a][0] = 0.5 * (0.5 - d) * (0.5 - d);
        w[a][1] = 0.75 - d * d;
        w[a][2] = 0.5 * (0.5 + d) * (0.5 + d);
    }
    // wrapped indices of the cells c0 - 3 .. c0 + 3 of every axis
    int ix[DIM][7];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int k = 0; k < 7; ++k) ix[a][k] = wrapi(c0[a] + k - 3, G.n[a]);
    const long long n1 = G.n[1], n2 = DIM == 3 ? G.n[2] : 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        // stencil along axis a: cell o (slot o + 2) contributes w_o (8 (phi[+1] - phi[-1]) -
        // (phi[+2] - phi[-2])) / (12 h)
        const double q = G.inv_h[a] / 12.0;
        double st[7];
        st[0] = w[a][0] * q;
        st[1] = (w[a][1] - 8.0 * w[a][0]) * q;
        st[2] = (w[a][2] - 8.0 * w[a][1]) * q;
        st[3] = (8.0 * (w[a][0] - w[a][2])) * q;
        st[4] = (8.0 * w[a][1] - w[a][0]) * q;
        st[5] = (8.0 * w[a][2] - w[a][1]) * q;
        st[6] = -w[a][2] * q;
        // the rows of cells along axis a picked by the other axes (b, and c in 3D) and their weights;
        // one row at a time keeps seven loads in flight per thread and the registers few
        const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
        double sum = 0.0;
#pragma unroll 1
        for (int r = 0; r < (DIM == 3 ? 9 : 3); ++r) {
            const int ob = DIM == 3 ? r / 3 : r, oc = DIM == 3 ? r % 3 : 1;
            const double wb = ob == 0 ? w[b][0] : (ob == 1 ? w[b][1] : w[b][2]);
            const double wc = DIM == 3 ? (oc == 0 ? w[c][0] : (oc == 1 ? w[c][1] : w[c][2])) : 1.0;
            const double wo = wb * wc;
            const long long jb = wrapi(c0[b] + ob - 1, G.n[b]);
            const long long jc = DIM == 3 ? wrapi(c0[c] + oc - 1, G.n[c]) : 0;
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                long long i3[3];
                i3[a] = ix[a][k];
                i3[b] = jb;
                i3[c] = jc;
                s += st[k] * phi[(i3[0] * n1 + i3[1]) * n2 + i3[2]];
            }
            sum += wo * s;
        }
        acc[a] = -sum;
    }
    if (DIM == 2) acc[2] = 0.0;
}

__global__ void __launch_bounds__(128, 4) k_force(ForceGrid G, const double* __restrict__ phi, long long np, const double* __restrict__ px,
                        const double* __restrict__ py, const double* __restrict__ pz, double* __restrict__ ax,
                        double* __restrict__ ay, double* __restrict__ az) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    double acc[3];
    if (G.dim == 3) {
        const double x[3] = {px[i], py[i], pz[i]};
        force_at<3>(G, phi, x, acc);
        az[i] = acc[2];
    } else {
        const double x[3] = {px[i], py[i], 0.0};
        force_at<2>(G, phi, x, acc);
    }
    ax[i] = acc[0];
    ay[i] = acc[1];
}

// ---------------------------------------------------------------------------------------------
// kick and drift; `dtp` (device scalar) overrides dt when given, times `fac`
// ---------------------------------------------------------------------------------------------
// x + v d, wrapped into [lo, lo + len) on a periodic box
__device__ __forceinline__ double drift_coord(double x, double v, double d, double lo, double len, int periodic) {
    double y = x + v * d;
    if (periodic) {
        y = lo + (y - lo) - len * floor((y - lo) / len);
        if (y >= lo + len) y -= len;
    }
    return y;
}

__global__ void k_drift(long long n, double* __restrict__ x, const double* __restrict__ v, double dt,
                        const double* __restrict__ dtp, double fac, double lo, double len, int periodic) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = drift_coord(x[i], v[i], (dtp ? *dtp : dt) * fac, lo, len, periodic);
}

__global__ void k_kick(long long n, double* __restrict__ v, const double* __restrict__ a, double dt,
                       const double* __restrict__ dtp, double fac) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    v[i] += a[i] * ((dtp ? *dtp : dt) * fac);
}

// ---------------------------------------------------------------------------------------------
// vertex density: scatter (M_i, |V_i|) of every simplex to its vertices, then divide
// ---------------------------------------------------------------------------------------------
// simplex s of a mesh: its vertex indices, mass and |V| (minimal-image edge vectors on a periodic
// box); false (and the index flag raised) for an out-of-range vertex index
template <int DIM>
__device__ __forceinline__ bool vd_simplex(long long s, long long nv, const int* __restrict__ simp,
                                           const double* const P[3], const double L[3],
                                           const double* __restrict__ mass, int periodic, int id[4], double& m,
                                           double& vol, unsigned* __restrict__ flags) {
    constexpr int dim = DIM, nvs = DIM + 1;
#pragma unroll
    for (int k = 0; k < nvs; ++k) {
        id[k] = simp[s * nvs + k];
        if (id[k] < 0 || id[k] >= nv) {
            atomicOr(flags, CDP_FLAG_INDEX);
            return false;
        }
    }
    double e[3][3];
#pragma unroll
    for (int k = 1; k < nvs; ++k)
#pragma unroll
        for (int a = 0; a < dim; ++a) {
            double d = P[a][id[k]] - P[a][id[0]];
            if (periodic) d -= L[a] * nearbyint(d / L[a]);
            e[k - 1][a] = d;
        }
    if (dim == 3) {
        vol = fabs(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                   e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])) /
              6.0;
    } else {
        vol = fabs(e[0][0] * e[1][1] - e[0][1] * e[1][0]) * 0.5;
    }
    m = mass[s];
    return true;
}

// simplex s's mass and |V| added to the sums of its vertices
template <int DIM>
__device__ __forceinline__ void vd_scatter_one(long long s, long long nv, const int* __restrict__ simp,
                                               const double* const P[3], const double L[3],
                                               const double* __restrict__ mass, int periodic,
                                               double* __restrict__ msum, double* __restrict__ vsum,
                                               unsigned* __restrict__ flags) {
    int id[4];
    double m, vol;
    if (!vd_simplex<DIM>(s, nv, simp, P, L, mass, periodic, id, m, vol, flags)) return;
#pragma unroll
    for (int k = 0; k <= DIM; ++k) {
        atomicAdd(msum + id[k], m);
        atomicAdd(vsum + id[k], vol);
    }
}

__global__ void k_vd_scatter(int dim, long long ns, long long nv, const int* __restrict__ simp,
                             const double* __restrict__ px, const double* __restrict__ py,
                             const double* __restrict__ pz, const double* __restrict__ mass, double L0, double L1,
                             double L2, int periodic, double* __restrict__ msum, double* __restrict__ vsum,
                             unsigned* __restrict__ flags) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const double* P[3] = {px, py, pz};
    const double L[3] = {L0, L1, L2};
    if (dim == 3)
        vd_scatter_one<3>(s, nv, simp, P, L, mass, periodic, msum, vsum, flags);
    else
        vd_scatter_one<2>(s, nv, simp, P, L, mass, periodic, msum, vsum, flags);
}

__global__ void k_vd_divide(long long nv, const double* __restrict__ msum, const double* __restrict__ vsum,
                            double* __restrict__ rho) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double v = vsum[i];
    rho[i] = v > 0.0 ? msum[i] / v : 0.0;
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// internal: used by cdp_step_batched.  fp32: the transforms in single precision (the FP32-mixed
// time step), the source and the potential still FP64 arrays
int poisson_enqueue(cdp_ctx* c, int dim, const int32_t grid[3], const double box_len[3], double four_pi_G,
                    const double* mass, double* phi, cudaStream_t st, bool fp32) {
    int rc = CDP_OK;
    FftPlan* p = get_plan(c, dim, grid, &rc);
    if (!p) return rc;
    if (fp32 && (rc = add_plan32(*p))) return rc;
    double ntot = 1.0, cellvol = 1.0;
    for (int a = 0; a < dim; ++a) {
        ntot *= grid[a];
        cellvol *= box_len[a] / grid[a];
    }
    const long long cells = (long long)ntot;
    const unsigned cb = blocks_for(cells, 256) > 65535u * 16u ? 65535u * 16u : blocks_for(cells, 256);
    double scale = -four_pi_G / (cellvol * ntot);
    const double twopi = 6.283185307179586476925286766559;
    // the Green function on the half spectrum: (n0, n1, n2 / 2 + 1) in 3D, (n0, n1 / 2 + 1) in 2D
    const int nh = grid[dim - 1] / 2 + 1;
    const long long tot = dim == 3 ? (long long)grid[0] * grid[1] * nh : (long long)grid[0] * nh;
    unsigned b = blocks_for(tot, 256);
    if (b > 65535u * 16u) b = 65535u * 16u;
    const double k0 = twopi / box_len[0], k1 = dim == 3 ? twopi / box_len[1] : 0.0, k2 = twopi / box_len[dim - 1];
    const int n1 = dim == 3 ? grid[1] : 1, n2 = grid[dim - 1];
    if (fp32) {
        if (cufftSetStream(p->r2c32, st) != CUFFT_SUCCESS || cufftSetStream(p->c2r32, st) != CUFFT_SUCCESS)
            return CDP_ERR_CUDA;
        k_to_f32<<<cb, 256, 0, st>>>(cells, mass, p->real32);
        if (cufftExecR2C(p->r2c32, p->real32, p->spec32) != CUFFT_SUCCESS) return CDP_ERR_CUDA;
        k_green<cufftComplex, float><<<b, 256, 0, st>>>(p->spec32, dim, grid[0], n1, nh, n2, (float)k0, (float)k1,
                                                        (float)k2, (float)scale);
        if (cufftExecC2R(p->c2r32, p->spec32, p->real32) != CUFFT_SUCCESS) return CDP_ERR_CUDA;
        k_to_f64<<<cb, 256, 0, st>>>(cells, p->real32, phi);
    } else {
        if (cufftSetStream(p->r2c, st) != CUFFT_SUCCESS || cufftSetStream(p->c2r, st) != CUFFT_SUCCESS)
            return CDP_ERR_CUDA;
        if (cufftExecD2Z(p->r2c, const_cast<double*>(mass), p->spec) != CUFFT_SUCCESS) return CDP_ERR_CUDA;
        k_green<cufftDoubleComplex, double><<<b, 256, 0, st>>>(p->spec, dim, grid[0], n1, nh, n2, k0, k1, k2, scale);
        if (cufftExecZ2D(p->c2r, p->spec, phi) != CUFFT_SUCCESS) return CDP_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? CDP_OK : CDP_ERR_CUDA;
}

int force_enqueue(int dim, const int32_t grid[3], const double box_lo[3], const double box_len[3], const double* phi,
                  long long n, const double* const pos[3], double* const acc[3], cudaStream_t st) {
    if (n == 0) return CDP_OK;
    ForceGrid G;
    memset(&G, 0, sizeof(G));
    G.dim = dim;
    for (int a = 0; a < 3; ++a) {
        G.n[a] = a < dim ? grid[a] : 1;
        G.lo[a] = a < dim ? box_lo[a] : 0.0;
        G.h[a] = a < dim ? box_len[a] / grid[a] : 1.0;
        G.inv_h[a] = 1.0 / G.h[a];
    }
    k_force<<<blocks_for(n, 128), 128, 0, st>>>(G, phi, n, pos[0], pos[1], dim == 3 ? pos[2] : nullptr, acc[0],
                                                 acc[1], dim == 3 ? acc[2] : nullptr);
    return cudaGetLastError() == cudaSuccess ? CDP_OK : CDP_ERR_CUDA;
}

int drift_enqueue(int dim, long long n, double* const pos[3], const double* const vel[3], double dt,
                  const double* dtp, double fac, const double box_lo[3], const double box_len[3], int periodic,
                  cudaStream_t st) {
    if (n == 0) return CDP_OK;
    for (int a = 0; a < dim; ++a)
        k_drift<<<blocks_for(n, 256), 256, 0, st>>>(n, pos[a], vel[a], dt, dtp, fac, box_lo[a], box_len[a],
                                                     periodic);
    return cudaGetLastError() == cudaSuccess ? CDP_OK : CDP_ERR_CUDA;
}

int kick_enqueue(int dim, long long n, double* const vel[3], const double* const acc[3], double dt,
                 const double* dtp, double fac, cudaStream_t st) {
    if (n == 0) return CDP_OK;
    for (int a = 0; a < dim; ++a) k_kick<<<blocks_for(n, 256), 256, 0, st>>>(n, vel[a], acc[a], dt, dtp, fac);
    return cudaGetLastError() == cudaSuccess ? CDP_OK : CDP_ERR_CUDA;
}

// the per-vertex accumulators of the vertex density, `need` doubles (grown outside any capture)
int reserve_vsum(cdp_ctx* c, size_t need) {
    if (need <= c->vsum_cap) return CDP_OK;
    double* q = nullptr;
    if (cudaMalloc(&q, need * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return CDP_ERR_OOM;
    }
    if (c->vsum) cudaFree(c->vsum);
    ++c->epoch;
    c->vsum = q;
    c->vsum_cap = need;
    return CDP_OK;
}

int vertex_density_enqueue(cdp_ctx* c, const cdp_problem* p, const double* mass, double* rho_out, cudaStream_t st) {
    int rc = reserve_vsum(c, 2 * (size_t)(p->n_verts > 0 ? p->n_verts : 1));
    if (rc) return rc;
    if (p->n_verts == 0) return CDP_OK;
    double* msum = c->vsum;
    double* vsum = c->vsum + p->n_verts;
    if (cudaMemsetAsync(c->vsum, 0, 2 * (size_t)p->n_verts * sizeof(double), st) != cudaSuccess) return CDP_ERR_CUDA;
    if (p->n_simplices > 0)
        k_vd_scatter<<<blocks_for(p->n_simplices, 128), 128, 0, st>>>(
            p->dim, p->n_simplices, p->n_verts, p->simplices, p->pos[0], p->pos[1], p->dim == 3 ? p->pos[2] : nullptr,
            mass, p->box_len[0], p->box_len[1], p->dim == 3 ? p->box_len[2] : 1.0, p->periodic, msum, vsum,
            &c->ctr->flags);
    k_vd_divide<<<blocks_for(p->n_verts, 256), 256, 0, st>>>(p->n_verts, msum, vsum, rho_out);
    return cudaGetLastError() == cudaSuccess ? CDP_OK : CDP_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------------
// The per-vertex steps of a batched time step, many meshes per launch: a table of up to
// CDP_STEP_GROUP meshes (of either dimension) passed by value, a global vertex or simplex index
// mapped to its mesh by a binary search over the offsets.  Each element does the arithmetic of
// the single-mesh kernels above, in the same order.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int CDP_STEP_GROUP = 64;

struct StepEntry {
    ForceGrid G;  // the mesh's grid (force interpolation)
    double* pos[3];
    double* vel[3];
    double* acc[3];
    const int* simplices;
    const double* smass;
    double* rho;
    const double* phi;
    double len[3];
    int dim, periodic;
    long long nv, ns;
    long long v_off, s_off;  // first vertex and simplex of the mesh in the group's numberings
};

struct StepTable {
    int n;
    long long nv, ns;  // totals over the group
    StepEntry p[CDP_STEP_GROUP];
};
static_assert(sizeof(StepTable) <= 32000, "a kernel parameter holds at most 32764 bytes");

template <class Off>
__device__ __forceinline__ int step_find(const StepTable& T, long long i, Off off) {
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off(T.p[mid]) <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// drift dt/2 (eq. drift1) of every vertex of the group
__global__ void __launch_bounds__(256) k_step_drift(const __grid_constant__ StepTable T, const double* __restrict__ dtp,
                                                    double fac) {
    const double d = *dtp * fac;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.nv; i += (long long)gridDim.x * blockDim.x) {
        const StepEntry& E = T.p[step_find(T, i, [](const StepEntry& e) { return e.v_off; })];
        const long long j = i - E.v_off;
        for (int a = 0; a < E.dim; ++a)
            E.pos[a][j] = drift_coord(E.pos[a][j], E.vel[a][j], d, E.G.lo[a], E.len[a], E.periodic);
    }
}

// the vertex-density sums of every simplex of the group (msum, vsum: the group's vertex numbering).
// (Grouping the lanes of a warp that name the same vertex and adding each group's sums with one
// atomic pair was slower: 3.58 against 2.89 ms per step on the 64-problem workload.)
__global__ void __launch_bounds__(128) k_step_vd_scatter(const __grid_constant__ StepTable T, double* __restrict__ msum,
                                                         double* __restrict__ vsum, unsigned* __restrict__ flags) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < T.ns; s += (long long)gridDim.x * blockDim.x) {
        const StepEntry& E = T.p[step_find(T, s, [](const StepEntry& e) { return e.s_off; })];
        const double* P[3] = {E.pos[0], E.pos[1], E.pos[2]};
        if (E.dim == 3)
            vd_scatter_one<3>(s - E.s_off, E.nv, E.simplices, P, E.len, E.smass, E.periodic, msum + E.v_off,
                              vsum + E.v_off, flags);
        else
            vd_scatter_one<2>(s - E.s_off, E.nv, E.simplices, P, E.len, E.smass, E.periodic, msum + E.v_off,
                              vsum + E.v_off, flags);
    }
}

__global__ void __launch_bounds__(256) k_step_vd_divide(const __grid_constant__ StepTable T, const double* __restrict__ msum,
                                                        const double* __restrict__ vsum) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.nv; i += (long long)gridDim.x * blockDim.x) {
        const StepEntry& E = T.p[step_find(T, i, [](const StepEntry& e) { return e.v_off; })];
        const double v = vsum[i];
        E.rho[i - E.v_off] = v > 0.0 ? msum[i] / v : 0.0;
    }
}

// force at vertex j of a mesh (written to acc), kick dt (eq. kick) and drift dt/2 (eq. drift2)
template <int DIM>
__device__ __forceinline__ void force_kick_drift_one(const StepEntry& E, long long j, double dk, double dd) {
    double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = E.pos[a][j];
    double acc[3];
    force_at<DIM>(E.G, E.phi, x, acc);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        E.acc[a][j] = acc[a];
        const double v = E.vel[a][j] + acc[a] * dk;
        E.vel[a][j] = v;
        E.pos[a][j] = drift_coord(x[a], v, dd, E.G.lo[a], E.len[a], E.periodic);
    }
}

// force, kick and drift of every vertex of the group, from its mesh's potential
__global__ void __launch_bounds__(128, 4) k_step_force_kick_drift(const __grid_constant__ StepTable T,
                                                               const double* __restrict__ dtp) {
    const double dk = *dtp * 1.0, dd = *dtp * 0.5;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.nv; i += (long long)gridDim.x * blockDim.x) {
        const StepEntry& E = T.p[step_find(T, i, [](const StepEntry& e) { return e.v_off; })];
        if (E.dim == 3)
            force_kick_drift_one<3>(E, i - E.v_off, dk, dd);
        else
            force_kick_drift_one<2>(E, i - E.v_off, dk, dd);
    }
}

unsigned step_blocks(long long n, int bs, int num_sms) {
    long long b = (n + bs - 1) / bs;
    const long long cap = (long long)num_sms * 32;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

// the table of probs[0 .. n) (n <= CDP_STEP_GROUP)
void fill_step_table(const cdp_step_problem* probs, int n, StepTable& T) {
    memset(&T, 0, sizeof(T));
    T.n = n;
    for (int i = 0; i < n; ++i) {
        const cdp_problem& m = probs[i].mesh;
        StepEntry& E = T.p[i];
        E.G.dim = m.dim;
        for (int a = 0; a < 3; ++a) {
            E.G.n[a] = a < m.dim ? m.grid[a] : 1;
            E.G.lo[a] = a < m.dim ? m.box_lo[a] : 0.0;
            E.G.h[a] = a < m.dim ? m.box_len[a] / m.grid[a] : 1.0;
            E.G.inv_h[a] = 1.0 / E.G.h[a];
            E.len[a] = a < m.dim ? m.box_len[a] : 1.0;
            E.pos[a] = a < m.dim ? const_cast<double*>(m.pos[a]) : nullptr;
            E.vel[a] = a < m.dim ? probs[i].vel[a] : nullptr;
            E.acc[a] = a < m.dim ? probs[i].acc[a] : nullptr;
        }
        E.simplices = m.simplices;
        E.smass = probs[i].simplex_mass;
        E.rho = const_cast<double*>(m.rho);
        E.phi = probs[i].phi;
        E.dim = m.dim;
        E.periodic = m.periodic;
        E.nv = m.n_verts;
        E.ns = m.n_simplices;
        E.v_off = T.nv;
        E.s_off = T.ns;
        T.nv += m.n_verts;
        T.ns += m.n_simplices;
    }
}

// The FP32 Poisson solves of a batched step (the FP32-mixed precision), many meshes per launch of
// the element-wise kernels: every mesh has its own FP32 real and spectrum arrays in the context's
// scratch (each starting on a 256-byte boundary), so the conversions of the source and the Green
// factors run once for the whole group, with one R2C and one C2R transform per mesh in between.
struct PoisEntry {
    const double* src;  // the cell masses
    double* phi;        // the potential
    long long cells, r_off;   // real array: its cells and first element in the group's real scratch
    long long selems, s_off;  // half spectrum: its entries and first entry in the spectrum scratch
    int dim, n0, n1, n2h;
    float k0, k1, k2, scale;
};

struct PoisTable {
    int n;
    long long rtot, stot;  // the group's real and spectrum scratch (with the padding)
    PoisEntry p[CDP_STEP_GROUP];
};
static_assert(sizeof(PoisTable) <= 32000, "a kernel parameter holds at most 32764 bytes");

__device__ __forceinline__ int pois_find(const PoisTable& T, long long i, bool spectrum) {
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((spectrum ? T.p[mid].s_off : T.p[mid].r_off) <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_pois_to_f32(const __grid_constant__ PoisTable T, float* __restrict__ real) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.rtot; i += (long long)gridDim.x * blockDim.x) {
        const PoisEntry& E = T.p[pois_find(T, i, false)];
        const long long j = i - E.r_off;
        if (j < E.cells) real[i] = (float)E.src[j];
    }
}

__global__ void __launch_bounds__(256) k_pois_green(const __grid_constant__ PoisTable T, cufftComplex* __restrict__ spec) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.stot; i += (long long)gridDim.x * blockDim.x) {
        const PoisEntry& E = T.p[pois_find(T, i, true)];
        const long long u = i - E.s_off;
        if (u < E.selems) green_at<cufftComplex, float>(spec[i], u, E.dim, E.n0, E.n1, E.n2h, E.k0, E.k1, E.k2, E.scale);
    }
}

__global__ void __launch_bounds__(256) k_pois_to_f64(const __grid_constant__ PoisTable T, const float* __restrict__ real) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.rtot; i += (long long)gridDim.x * blockDim.x) {
        const PoisEntry& E = T.p[pois_find(T, i, false)];
        const long long j = i - E.r_off;
        if (j < E.cells) E.phi[j] = (double)real[i];
    }
}

// the table of probs[0 .. n) (n <= CDP_STEP_GROUP)
void fill_pois_table(const cdp_step_problem* probs, int n, double four_pi_G, PoisTable& T) {
    memset(&T, 0, sizeof(T));
    T.n = n;
    const double twopi = 6.283185307179586476925286766559;
    for (int i = 0; i < n; ++i) {
        const cdp_problem& m = probs[i].mesh;
        const int dim = m.dim;
        PoisEntry& E = T.p[i];
        double ntot = 1.0, cellvol = 1.0;
        for (int a = 0; a < dim; ++a) {
            ntot *= m.grid[a];
            cellvol *= m.box_len[a] / m.grid[a];
        }
        E.src = m.cell_mass;
        E.phi = probs[i].phi;
        E.dim = dim;
        E.n0 = m.grid[0];
        E.n1 = dim == 3 ? m.grid[1] : 1;
        E.n2h = m.grid[dim - 1] / 2 + 1;
        E.cells = (long long)ntot;
        E.selems = (long long)E.n0 * E.n1 * E.n2h;
        E.k0 = (float)(twopi / m.box_len[0]);
        E.k1 = (float)(dim == 3 ? twopi / m.box_len[1] : 0.0);
        E.k2 = (float)(twopi / m.box_len[dim - 1]);
        E.scale = (float)(-four_pi_G / (cellvol * ntot));
        E.r_off = T.rtot;
        E.s_off = T.stot;
        T.rtot += (E.cells + 63) / 64 * 64;       // 256-byte boundaries
        T.stot += (E.selems + 31) / 32 * 32;
    }
}

}  // namespace

// the FP32 real and spectrum scratch of the largest group of a batched step's Poisson solves
int reserve_poisson32(cdp_ctx* c, const cdp_step_problem* probs, int n) {
    PoisTable* T = new (std::nothrow) PoisTable;
    if (!T) return CDP_ERR_OOM;
    long long rmax = 1, smax = 1;
    for (int g0 = 0; g0 < n; g0 += CDP_STEP_GROUP) {
        fill_pois_table(probs + g0, n - g0 < CDP_STEP_GROUP ? n - g0 : CDP_STEP_GROUP, 1.0, *T);
        rmax = T->rtot > rmax ? T->rtot : rmax;
        smax = T->stot > smax ? T->stot : smax;
    }
    delete T;
    for (int k = 0; k < 2; ++k) {
        void** buf = k == 0 ? (void**)&c->preal : (void**)&c->pspec;
        size_t* cap = k == 0 ? &c->preal_cap : &c->pspec_cap;
        const size_t need = (size_t)(k == 0 ? rmax : smax), elem = k == 0 ? sizeof(float) : sizeof(cufftComplex);
        if (need <= *cap) continue;
        void* q = nullptr;
        if (cudaMalloc(&q, need * elem) != cudaSuccess) {
            cudaGetLastError();
            return CDP_ERR_OOM;
        }
        if (*buf) cudaFree(*buf);
        ++c->epoch;
        *buf = q;
        *cap = need;
    }
    return CDP_OK;
}

// the Poisson solves of every mesh in single precision (source and potential FP64 arrays): per
// group one launch of each element-wise kernel, one R2C and one C2R per mesh
int step_poisson32_enqueue(cdp_ctx* c, const cdp_step_problem* probs, int n, double four_pi_G, cudaStream_t st) {
    int rc = reserve_poisson32(c, probs, n);
    if (rc) return rc;
    PoisTable* T = new (std::nothrow) PoisTable;
    if (!T) return CDP_ERR_OOM;
    for (int g0 = 0; g0 < n && rc == CDP_OK; g0 += CDP_STEP_GROUP) {
        const int ng = n - g0 < CDP_STEP_GROUP ? n - g0 : CDP_STEP_GROUP;
        fill_pois_table(probs + g0, ng, four_pi_G, *T);
        if (T->rtot == 0) continue;
        k_pois_to_f32<<<step_blocks(T->rtot, 256, c->num_sms), 256, 0, st>>>(*T, c->preal);
        for (int i = 0; i < ng && rc == CDP_OK; ++i) {
            const cdp_problem& m = probs[g0 + i].mesh;
            FftPlan* p = get_plan(c, m.dim, m.grid, &rc);
            if (!p || (rc = add_plan32(*p))) break;
            if (cufftSetStream(p->r2c32, st) != CUFFT_SUCCESS ||
                cufftExecR2C(p->r2c32, c->preal + T->p[i].r_off, c->pspec + T->p[i].s_off) != CUFFT_SUCCESS)
                rc = CDP_ERR_CUDA;
        }
        if (rc) break;
        k_pois_green<<<step_blocks(T->stot, 256, c->num_sms), 256, 0, st>>>(*T, c->pspec);
        for (int i = 0; i < ng && rc == CDP_OK; ++i) {
            const cdp_problem& m = probs[g0 + i].mesh;
            FftPlan* p = get_plan(c, m.dim, m.grid, &rc);
            if (!p) break;
            if (cufftSetStream(p->c2r32, st) != CUFFT_SUCCESS ||
                cufftExecC2R(p->c2r32, c->pspec + T->p[i].s_off, c->preal + T->p[i].r_off) != CUFFT_SUCCESS)
                rc = CDP_ERR_CUDA;
        }
        if (rc) break;
        k_pois_to_f64<<<step_blocks(T->rtot, 256, c->num_sms), 256, 0, st>>>(*T, c->preal);
        if (cudaGetLastError() != cudaSuccess) rc = CDP_ERR_CUDA;
    }
    delete T;
    return rc;
}

// the largest number of vertices of one group of a batched step (sizes the vertex-density sums)
long long step_group_vertices(const cdp_step_problem* probs, int n) {
    long long most = 0;
    for (int g0 = 0; g0 < n; g0 += CDP_STEP_GROUP) {
        long long nv = 0;
        for (int i = g0; i < n && i < g0 + CDP_STEP_GROUP; ++i) nv += probs[i].mesh.n_verts;
        most = nv > most ? nv : most;
    }
    return most;
}

// drift dt/2, then the vertex densities, of every mesh (one launch of each kernel per group)
int step_drift_density_enqueue(cdp_ctx* c, const cdp_step_problem* probs, int n, const double* dtp, cudaStream_t st) {
    const long long most = step_group_vertices(probs, n);
    int rc = reserve_vsum(c, 2 * (size_t)(most > 0 ? most : 1));
    if (rc) return rc;
    StepTable* T = new (std::nothrow) StepTable;
    if (!T) return CDP_ERR_OOM;
    for (int g0 = 0; g0 < n && rc == CDP_OK; g0 += CDP_STEP_GROUP) {
        fill_step_table(probs + g0, n - g0 < CDP_STEP_GROUP ? n - g0 : CDP_STEP_GROUP, *T);
        if (T->nv == 0) continue;
        k_step_drift<<<step_blocks(T->nv, 256, c->num_sms), 256, 0, st>>>(*T, dtp, 0.5);
        double* msum = c->vsum;
        double* vsum = c->vsum + T->nv;
        if (cudaMemsetAsync(c->vsum, 0, 2 * (size_t)T->nv * sizeof(double), st) != cudaSuccess) rc = CDP_ERR_CUDA;
        if (rc == CDP_OK && T->ns > 0)
            k_step_vd_scatter<<<step_blocks(T->ns, 128, c->num_sms), 128, 0, st>>>(*T, msum, vsum, &c->ctr->flags);
        if (rc == CDP_OK) k_step_vd_divide<<<step_blocks(T->nv, 256, c->num_sms), 256, 0, st>>>(*T, msum, vsum);
        if (rc == CDP_OK && cudaGetLastError() != cudaSuccess) rc = CDP_ERR_CUDA;
    }
    delete T;
    return rc;
}

// force, kick dt and drift dt/2 of every mesh (one launch per group), after the potentials
int step_force_kick_drift_enqueue(cdp_ctx* c, const cdp_step_problem* probs, int n, const double* dtp,
                                  cudaStream_t st) {
    StepTable* T = new (std::nothrow) StepTable;
    if (!T) return CDP_ERR_OOM;
    int rc = CDP_OK;
    for (int g0 = 0; g0 < n && rc == CDP_OK; g0 += CDP_STEP_GROUP) {
        fill_step_table(probs + g0, n - g0 < CDP_STEP_GROUP ? n - g0 : CDP_STEP_GROUP, *T);
        if (T->nv == 0) continue;
        k_step_force_kick_drift<<<step_blocks(T->nv, 128, c->num_sms), 128, 0, st>>>(*T, dtp);
        if (cudaGetLastError() != cudaSuccess) rc = CDP_ERR_CUDA;
    }
    delete T;
    return rc;
}

void solver_release(cdp_ctx* c) {
    if (c->plans) {
        for (FftPlan& p : *c->plans) {
            cufftDestroy(p.r2c);
            cufftDestroy(p.c2r);
            if (p.spec) cudaFree(p.spec);
            if (p.have32) {
                cufftDestroy(p.r2c32);
                cufftDestroy(p.c2r32);
            }
            if (p.spec32) cudaFree(p.spec32);
            if (p.real32) cudaFree(p.real32);
        }
        delete c->plans;
        c->plans = nullptr;
    }
    if (c->vsum) cudaFree(c->vsum);
    c->vsum = nullptr;
    if (c->preal) cudaFree(c->preal);
    c->preal = nullptr;
    if (c->pspec) cudaFree(c->pspec);
    c->pspec = nullptr;
}

}  // namespace cdp

extern "C" {

int cdp_poisson(cdp_ctx* c, int dim, const int32_t grid[3], const double box_len[3], double four_pi_G,
                const double* cell_mass, double* phi, void* stream) {
    if (!c || !cell_mass || !phi) return CDP_ERR_ARG;
    int rc = cdp::check_grid(dim, grid, box_len);
    if (rc) return rc;
    if (!(four_pi_G == four_pi_G)) return CDP_ERR_ARG;
    cdp::DevGuard guard(c->device);
    return cdp::poisson_enqueue(c, dim, grid, box_len, four_pi_G, cell_mass, phi, (cudaStream_t)stream, false);
}

int cdp_force(cdp_ctx* c, int dim, const int32_t grid[3], const double box_lo[3], const double box_len[3],
              const double* phi, int64_t n, const double* const pos[3], double* const acc[3], void* stream) {
    if (!c || !phi || !box_lo || n < 0 || !pos || !acc) return CDP_ERR_ARG;
    int rc = cdp::check_grid(dim, grid, box_len);
    if (rc) return rc;
    for (int a = 0; a < dim; ++a)
        if (n > 0 && (!pos[a] || !acc[a])) return CDP_ERR_ARG;
    cdp::DevGuard guard(c->device);
    return cdp::force_enqueue(dim, grid, box_lo, box_len, phi, n, pos, acc, (cudaStream_t)stream);
}

int cdp_drift(cdp_ctx* c, int dim, int64_t n, double* const pos[3], const double* const vel[3], double dt,
              const double box_lo[3], const double box_len[3], int periodic, void* stream) {
    if (!c || (dim != 2 && dim != 3) || n < 0 || !pos || !vel || !box_lo || !box_len || !(dt == dt))
        return CDP_ERR_ARG;
    for (int a = 0; a < dim; ++a) {
        if (n > 0 && (!pos[a] || !vel[a])) return CDP_ERR_ARG;
        if (periodic && !(box_len[a] > 0.0)) return CDP_ERR_ARG;
    }
    cdp::DevGuard guard(c->device);
    return cdp::drift_enqueue(dim, n, pos, vel, dt, nullptr, 1.0, box_lo, box_len, periodic, (cudaStream_t)stream);
}

int cdp_kick(cdp_ctx* c, int dim, int64_t n, double* const vel[3], const double* const acc[3], double dt,
             void* stream) {
    if (!c || (dim != 2 && dim != 3) || n < 0 || !vel || !acc || !(dt == dt)) return CDP_ERR_ARG;
    for (int a = 0; a < dim; ++a)
        if (n > 0 && (!vel[a] || !acc[a])) return CDP_ERR_ARG;
    cdp::DevGuard guard(c->device);
    return cdp::kick_enqueue(dim, n, vel, acc, dt, nullptr, 1.0, (cudaStream_t)stream);
}

int cdp_vertex_density(cdp_ctx* c, const cdp_problem* p, const double* simplex_mass, double* rho_out,
                       void* stream) {
    if (!c || !p || !rho_out || (p->n_simplices > 0 && !simplex_mass)) return CDP_ERR_ARG;
    if ((p->dim != 2 && p->dim != 3) || p->n_verts < 0 || p->n_simplices < 0) return CDP_ERR_ARG;
    if (p->n_simplices > 0 && !p->simplices) return CDP_ERR_ARG;
    for (int a = 0; a < p->dim; ++a) {
        if (p->n_verts > 0 && !p->pos[a]) return CDP_ERR_ARG;
        if (p->periodic && !(p->box_len[a] > 0.0)) return CDP_ERR_ARG;
    }
    cdp::DevGuard guard(c->device);
    return cdp::vertex_density_enqueue(c, p, simplex_mass, rho_out, (cudaStream_t)stream);
}

}  // extern "C"
