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
template <typename C, typename R>
__global__ void k_green(C* __restrict__ spec, int dim, int n0, int n1, int n2h, int n2, R k0, R k1, R k2, R scale) {
    long long total = (long long)n0 * n1 * n2h;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
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
        spec[t].x *= gfac;
        spec[t].y *= gfac;
    }
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

__global__ void k_force(ForceGrid G, const double* __restrict__ phi, long long np, const double* __restrict__ px,
                        const double* __restrict__ py, const double* __restrict__ pz, double* __restrict__ ax,
                        double* __restrict__ ay, double* __restrict__ az) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double* P[3] = {px, py, pz};
    int c0[3] = {0, 0, 0};
    double w[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
    for (int a = 0; a < G.dim; ++a) {
        double u = (P[a][i] - G.lo[a]) * G.inv_h[a] - 0.5;
        double f = floor(u + 0.5);
        double d = u - f;
        c0[a] = (int)f;
        w[a][0] = 0.5 * (0.5 - d) * (0.5 - d);
        w[a][1] = 0.75 - d * d;
        w[a][2] = 0.5 * (0.5 + d) * (0.5 + d);
    }
    double acc[3] = {0.0, 0.0, 0.0};
    const int n0 = G.n[0], n1 = G.n[1], n2 = G.dim == 3 ? G.n[2] : 1;
    const int zr = G.dim == 3 ? 1 : 0;
    for (int oa = -1; oa <= 1; ++oa)
        for (int ob = -1; ob <= 1; ++ob)
            for (int oc = -zr; oc <= zr; ++oc) {
                double wt = w[0][oa + 1] * w[1][ob + 1] * (G.dim == 3 ? w[2][oc + 1] : 1.0);
                int ia = c0[0] + oa, ib = c0[1] + ob, ic = c0[2] + oc;
                int wa = wrapi(ia, n0), wb = wrapi(ib, n1), wc = G.dim == 3 ? wrapi(ic, n2) : 0;
                // 4-point differences along each axis at cell (ia, ib, ic)
                double g0 = (8.0 * (phi[((long long)wrapi(ia + 1, n0) * n1 + wb) * n2 + wc] -
                                    phi[((long long)wrapi(ia - 1, n0) * n1 + wb) * n2 + wc]) -
                             (phi[((long long)wrapi(ia + 2, n0) * n1 + wb) * n2 + wc] -
                              phi[((long long)wrapi(ia - 2, n0) * n1 + wb) * n2 + wc])) *
                            (G.inv_h[0] / 12.0);
                double g1 = (8.0 * (phi[((long long)wa * n1 + wrapi(ib + 1, n1)) * n2 + wc] -
                                    phi[((long long)wa * n1 + wrapi(ib - 1, n1)) * n2 + wc]) -
                             (phi[((long long)wa * n1 + wrapi(ib + 2, n1)) * n2 + wc] -
                              phi[((long long)wa * n1 + wrapi(ib - 2, n1)) * n2 + wc])) *
                            (G.inv_h[1] / 12.0);
                acc[0] -= wt * g0;
                acc[1] -= wt * g1;
                if (G.dim == 3) {
                    long long rowb = ((long long)wa * n1 + wb) * n2;
                    double g2 = (8.0 * (phi[rowb + wrapi(ic + 1, n2)] - phi[rowb + wrapi(ic - 1, n2)]) -
                                 (phi[rowb + wrapi(ic + 2, n2)] - phi[rowb + wrapi(ic - 2, n2)])) *
                                (G.inv_h[2] / 12.0);
                    acc[2] -= wt * g2;
                }
            }
    ax[i] = acc[0];
    ay[i] = acc[1];
    if (G.dim == 3) az[i] = acc[2];
}

// ---------------------------------------------------------------------------------------------
// kick and drift; `dtp` (device scalar) overrides dt when given, times `fac`
// ---------------------------------------------------------------------------------------------
__global__ void k_drift(long long n, double* __restrict__ x, const double* __restrict__ v, double dt,
                        const double* __restrict__ dtp, double fac, double lo, double len, int periodic) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = (dtp ? *dtp : dt) * fac;
    double y = x[i] + v[i] * d;
    if (periodic) {
        y = lo + (y - lo) - len * floor((y - lo) / len);
        if (y >= lo + len) y -= len;
    }
    x[i] = y;
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
__global__ void k_vd_scatter(int dim, long long ns, long long nv, const int* __restrict__ simp,
                             const double* __restrict__ px, const double* __restrict__ py,
                             const double* __restrict__ pz, const double* __restrict__ mass, double L0, double L1,
                             double L2, int periodic, double* __restrict__ msum, double* __restrict__ vsum,
                             unsigned* __restrict__ flags) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int nvs = dim + 1;
    int id[4];
    for (int k = 0; k < nvs; ++k) {
        id[k] = simp[s * nvs + k];
        if (id[k] < 0 || id[k] >= nv) {
            atomicOr(flags, CDP_FLAG_INDEX);
            return;
        }
    }
    const double* P[3] = {px, py, pz};
    const double L[3] = {L0, L1, L2};
    double e[3][3];
    for (int k = 1; k < nvs; ++k)
        for (int a = 0; a < dim; ++a) {
            double d = P[a][id[k]] - P[a][id[0]];
            if (periodic) d -= L[a] * nearbyint(d / L[a]);
            e[k - 1][a] = d;
        }
    double vol;
    if (dim == 3) {
        vol = fabs(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                   e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])) /
              6.0;
    } else {
        vol = fabs(e[0][0] * e[1][1] - e[0][1] * e[1][0]) * 0.5;
    }
    double m = mass[s];
    for (int k = 0; k < nvs; ++k) {
        atomicAdd(msum + id[k], m);
        atomicAdd(vsum + id[k], vol);
    }
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

int vertex_density_enqueue(cdp_ctx* c, const cdp_problem* p, const double* mass, double* rho_out, cudaStream_t st) {
    size_t need = 2 * (size_t)(p->n_verts > 0 ? p->n_verts : 1);
    if (need > c->vsum_cap) {
        double* q = nullptr;
        if (cudaMalloc(&q, need * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return CDP_ERR_OOM;
        }
        if (c->vsum) cudaFree(c->vsum);
        ++c->epoch;
        c->vsum = q;
        c->vsum_cap = need;
    }
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
