// Projection onto an adaptive hierarchy of grids and donor-cell gather onto the uniform grid (Sect.
// 4.4, calculation of the acceleration): the AMR cells are refined while they are larger than the
// smallest perpendicular height of a simplex that crosses them, the projection onto them is exact
// (Sect. 3), and the uniform grid of the Poisson solve receives their masses by a donor-cell gather.
//
// Here the hierarchy is a stack of uniform grids over the whole box, level l with grid / 2^l cells per
// axis (level 0 = the output grid), and every simplex is projected, exactly, onto the coarsest level
// whose cells are no larger than its own smallest perpendicular height (a per-simplex reading of the
// refinement rule: the paper refines a region down to the smallest simplex crossing it).  The gather
// gives every output cell its own exact mass plus, from each coarser level, 1 / 2^(D l) of the mass of
// the coarse cell that contains it (the coarse cell's mass spread evenly over the cells it covers).
// Total mass is kept exactly; the density inside a coarse cell is only resolved at its level, which
// is the accuracy the AMR trades for speed (a large simplex meets far fewer coarse cells).
#include <cuda_runtime.h>

#include <new>

#include "../../include/coldproj.h"
#include "cdp_ctx.h"
#include "cdp_project.h"

namespace cdp {

int check_problem_args(const cdp_problem* p);
int build_table(const cdp_problem* const* probs, int n, ProbTable& T);
int project_group(cdp_ctx* c, const ProbTable& T, int precision, int accumulate, cudaStream_t st, bool want_stats,
                  unsigned char* amr_levels, int max_level);
int reserve_amr(cdp_ctx* c, size_t coarse_cells, size_t n_simplices);
int read_stats_ctx(cdp_ctx* c, cudaStream_t st, cdp_stats* stats);

namespace {

// Level of every simplex from the vertex records of the output grid (entry 0 of the table): its
// smallest perpendicular height eta = D |V| / (largest facet measure), in output cells (3D: 6|V| over
// the largest |facet normal| = twice the facet area; 2D: 2|A| over the longest edge), and the level
// l = min(max_level, floor(log2 eta)) (0 when eta < 2).  The edge vectors are the fixed-point
// differences to vertex 0 at its minimal image (exact in FP64: below 2^53), the rest is FP64
// arithmetic on squares (relative error ~1e-15: a simplex whose height is that close to a power of
// two may take either level).  Invalid simplices get level 0; the set-up reports them there.
template <int DIM>
__global__ void __launch_bounds__(256) k_amr_levels(const __grid_constant__ ProbTable T, const VertexRec* __restrict__ V,
                                                     int max_level, unsigned char* __restrict__ levels) {
    const ProbEntry& P = T.p[0];
    const GridDesc& g = P.g;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < P.ns; s += (long long)gridDim.x * blockDim.x) {
        int id[DIM + 1];
        bool ok = true;
        for (int k = 0; k <= DIM; ++k) {
            id[k] = __ldg(P.simplices + s * (DIM + 1) + k);
            ok = ok && id[k] >= 0 && id[k] < P.nv;
        }
        // D |V| and the largest facet measure, squared (no square root or division: the level is the
        // number of l in 1 .. max_level with (D |V|)^2 >= 4^l (largest facet measure)^2)
        double h2 = 0.0, a2 = 0.0;
        if (ok) {
            const VertexRec* v0 = V + P.v_off + id[0];
            double e[DIM][3];
            for (int k = 1; k <= DIM; ++k) {
                const VertexRec* vk = V + P.v_off + id[k];
                for (int a = 0; a < DIM; ++a) {
                    i64 d = vk->x[a] - v0->x[a];
                    if (g.periodic) {
                        const i64 NQ = (i64)g.n[a] << CDP_Q, half = (i64)g.n[a] << (CDP_Q - 1);
                        if (d > half) d -= NQ;
                        if (d < -half) d += NQ;
                    }
                    e[k - 1][a] = ldexp((double)d, -CDP_Q);
                }
            }
            if (DIM == 3) {
                // facet normals: n_f = (p_b - p_a) x (p_c - p_a) over the facets (a, b, c), p_0 = 0
                const double z[3] = {0.0, 0.0, 0.0};
                const double* p[4] = {z, e[0], e[1], e[2 % DIM]};
                double vol6 = 0.0;
                for (int f = 0; f < 4; ++f) {
                    const int a = f == 0 ? 1 : 0, b = f <= 1 ? 2 : 1, c = f <= 2 ? 3 : 2;
                    double u[3], w[3];
                    for (int i = 0; i < 3; ++i) {
                        u[i] = p[b][i] - p[a][i];
                        w[i] = p[c][i] - p[a][i];
                    }
                    const double n0 = u[1] * w[2] - u[2] * w[1], n1 = u[2] * w[0] - u[0] * w[2],
                                 n2 = u[0] * w[1] - u[1] * w[0];
                    a2 = fmax(a2, n0 * n0 + n1 * n1 + n2 * n2);
                    if (f == 3) vol6 = n0 * e[2 % DIM][0] + n1 * e[2 % DIM][1] + n2 * e[2 % DIM][2];
                }
                h2 = vol6 * vol6;
            } else {
                const double area2 = e[0][0] * e[1 % DIM][1] - e[0][1] * e[1 % DIM][0];
                const double dx = e[1 % DIM][0] - e[0][0], dy = e[1 % DIM][1] - e[0][1];
                a2 = fmax(fmax(e[0][0] * e[0][0] + e[0][1] * e[0][1],
                               e[1 % DIM][0] * e[1 % DIM][0] + e[1 % DIM][1] * e[1 % DIM][1]),
                          dx * dx + dy * dy);
                h2 = area2 * area2;
            }
        }
        int level = 0;
        while (level < max_level && a2 > 0.0 && h2 >= (double)(1 << (2 * level + 2)) * a2) ++level;
        levels[s] = (unsigned char)level;
    }
}

// Donor-cell gather: every output cell adds, from each level l >= 1, the mass of the level-l cell
// that contains it divided by 2^(D l).
__global__ void __launch_bounds__(256) k_donor_gather(const __grid_constant__ ProbTable T) {
    const ProbEntry& F = T.p[0];
    const int D = F.g.dim;
    const long long n1 = F.g.n[1], n2 = D == 3 ? F.g.n[2] : 1;
    const long long cells = (long long)F.g.n[0] * n1 * n2;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (long long)gridDim.x * blockDim.x) {
        const long long i = c / (n1 * n2), j = (c / n2) % n1, k = c % n2;
        double add = 0.0;
        for (int l = 1; l < T.n; ++l) {
            const ProbEntry& P = T.p[l];
            const long long ci = i >> l, cj = j >> l;
            const long long idx = D == 3 ? (ci * P.g.n[1] + cj) * P.g.n[2] + (k >> l) : ci * P.g.n[1] + cj;
            add += ldexp(P.out[idx], -D * l);
        }
        F.out[c] += add;
    }
}

long long grid_blocks(long long n, int num_sms) {
    long long b = (n + 255) / 256;
    const long long cap = (long long)num_sms * 16;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

}  // namespace

// levels of the mesh of entry 0 (its vertex records already made by launch_prep)
cudaError_t launch_amr_levels(const LaunchArgs& L, int max_level, unsigned char* levels, cudaStream_t st) {
    const ProbEntry& P = L.T.p[0];
    if (P.ns <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)grid_blocks(P.ns, L.num_sms);
    if (L.T.dim == 3)
        k_amr_levels<3><<<blocks, 256, 0, st>>>(L.T, L.verts, max_level, levels);
    else
        k_amr_levels<2><<<blocks, 256, 0, st>>>(L.T, L.verts, max_level, levels);
    return cudaGetLastError();
}

}  // namespace cdp

extern "C" int cdp_project_amr(cdp_ctx* c, const cdp_problem* p, int precision, int max_level, int accumulate,
                               void* stream, cdp_stats* stats) {
    using namespace cdp;
    if (!c) return CDP_ERR_ARG;
    int rc = check_problem_args(p);
    if (rc) return rc;
    {
        int f = 0, a = 0;
        if (!parse_precision(precision, &f, &a)) return CDP_ERR_ARG;
    }
    if (max_level < 0 || max_level > CDP_AMR_MAX_LEVEL) return CDP_ERR_ARG;
    for (int a = 0; a < p->dim; ++a)
        if (p->grid[a] % (1 << max_level) != 0) return CDP_ERR_ARG;
    if (max_level == 0) return cdp_project(c, p, precision, accumulate, stream, stats);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    // the coarse levels' grids, one after the other in the context's scratch; every level is a
    // problem of the same mesh
    long long coarse = 0;
    for (int l = 1; l <= max_level; ++l) {
        long long cl = 1;
        for (int a = 0; a < p->dim; ++a) cl *= p->grid[a] >> l;
        coarse += cl;
    }
    rc = reserve_amr(c, (size_t)coarse, (size_t)(p->n_simplices > 0 ? p->n_simplices : 1));
    ProbTable* T = nullptr;
    if (rc == CDP_OK) {
        T = new (std::nothrow) ProbTable;
        if (!T) rc = CDP_ERR_OOM;
    }
    if (rc == CDP_OK) {
        cdp_problem lv[CDP_AMR_MAX_LEVEL + 1];
        const cdp_problem* lp[CDP_AMR_MAX_LEVEL + 1];
        long long off = 0;
        for (int l = 0; l <= max_level; ++l) {
            lv[l] = *p;
            long long cl = 1;
            for (int a = 0; a < p->dim; ++a) {
                lv[l].grid[a] = p->grid[a] >> l;
                cl *= lv[l].grid[a];
            }
            if (l > 0) {
                lv[l].cell_mass = c->amr + off;
                off += cl;
            }
            lp[l] = &lv[l];
        }
        rc = build_table(lp, max_level + 1, *T);
    }
    // every level's grid starts from zero: without accumulate the group's projection zeroes them all;
    // with it the output grid keeps what it holds and only the coarse ones are zeroed here
    if (rc == CDP_OK && accumulate && cudaMemsetAsync(c->amr, 0, (size_t)coarse * sizeof(double), st) != cudaSuccess)
        rc = CDP_ERR_CUDA;
    if (rc == CDP_OK) rc = project_group(c, *T, precision, accumulate, st, stats != nullptr, c->levels, max_level);
    if (rc == CDP_OK) {
        const long long cells = T->p[1].c_off;  // those of the output grid
        k_donor_gather<<<(unsigned)grid_blocks(cells, c->num_sms), 256, 0, st>>>(*T);
        if (cudaGetLastError() != cudaSuccess) rc = CDP_ERR_CUDA;
    }
    delete T;
    if (rc == CDP_OK && stats) rc = read_stats_ctx(c, st, stats);
    if (prev != c->device) cudaSetDevice(prev);
    return rc;
}
