/*
 * CPU oracle for the exact projection of a piecewise-linear density on a simplicial mesh onto a
 * regular grid.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
 * baseline call it; the library never does.  It shares no code with the CUDA path.
 *
 * What it computes is the plain definition of the projection (Sect. 3, Eq. firstOrder; what
 * Algorithm 2 outputs: for every grid cell, the exact mass of the piecewise-linear interpolant of
 * the vertex densities over the mesh):
 *
 *     m_V = sum_S  integral over (S intersect V) of rho_S(x) dx,
 *
 * where rho_S is the linear (barycentric) interpolant of the vertex densities of simplex S and V
 * is the half-open grid cell [lo + i h, lo + (i+1) h) per axis (index taken mod N on a periodic
 * box).  It does NOT use the Franklin vertex/edge/facet formula, predicates or simulation of
 * simplicity.  For every simplex and every cell of its bounding box it clips the simplex by the
 * 2D (resp. 4) half-spaces of the cell, recursively splitting every clipped piece back into
 * simplices, and integrates rho exactly on each piece as |vol| * mean(rho at its vertices)
 * (exact for a linear function; Appendix C uses the same fact).  Clipping is measure-robust:
 * a point that falls exactly on a plane only moves a piece of zero measure.
 *
 * Periodic boxes: every simplex is unwrapped to the minimal image of its vertex 0; a simplex
 * spanning half a box length or more on a periodic axis is rejected (ORACLE_ERR_EXTENT).
 * Non-periodic boxes: mass that falls outside the grid is dropped.
 *
 * Arithmetic: IEEE double throughout; coordinates are taken relative to each cell's lower corner
 * before clipping so that they stay within a few cells in magnitude.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_INDEX (-2)
#define ORACLE_ERR_EXTENT (-4)

typedef struct {
    double x[4][3];
    double r[4];
} piece3;

typedef struct {
    double x[3][2];
    double r[3];
} piece2;

/* ---------------------------------------------------------------------------------------- */
/* 3D: recursive clipping of a tetrahedron by the 6 half-spaces 0 <= x_a <= 1               */
/* ---------------------------------------------------------------------------------------- */

static double tet_mass(const double x[4][3], const double r[4]) {
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = x[1][k] - x[0][k];
        b[k] = x[2][k] - x[0][k];
        c[k] = x[3][k] - x[0][k];
    }
    double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                 a[2] * (b[0] * c[1] - b[1] * c[0]);
    return fabs(det) / 6.0 * 0.25 * (r[0] + r[1] + r[2] + r[3]);
}

/* signed distance of x to half-space number p: p = 2a -> x_a >= 0, p = 2a+1 -> x_a <= 1 */
static inline double hs(const double* x, int p) {
    int a = p >> 1;
    return (p & 1) ? 1.0 - x[a] : x[a];
}

static void lerp3(const double* xi, double ri, double di, const double* xj, double rj, double dj,
                  double* out, double* rout) {
    double t = di / (di - dj);
    for (int k = 0; k < 3; ++k) out[k] = xi[k] + t * (xj[k] - xi[k]);
    *rout = ri + t * (rj - ri);
}

static double clip3(const double x[4][3], const double r[4], int p);

static double emit3(const double* a, double ra, const double* b, double rb, const double* c, double rc,
                    const double* d, double rd, int p) {
    double x[4][3], r[4];
    memcpy(x[0], a, 3 * sizeof(double));
    memcpy(x[1], b, 3 * sizeof(double));
    memcpy(x[2], c, 3 * sizeof(double));
    memcpy(x[3], d, 3 * sizeof(double));
    r[0] = ra;
    r[1] = rb;
    r[2] = rc;
    r[3] = rd;
    return clip3(x, r, p);
}

/* integral of rho over (tet intersect the half-spaces p..5) */
static double clip3(const double x[4][3], const double r[4], int p) {
    if (p == 6) return tet_mass(x, r);
    double d[4];
    int in[4], out[4], ni = 0, no = 0;
    for (int i = 0; i < 4; ++i) {
        d[i] = hs(x[i], p);
        if (d[i] >= 0.0)
            in[ni++] = i;
        else
            out[no++] = i;
    }
    if (no == 0) return clip3(x, r, p + 1);
    if (ni == 0) return 0.0;
    if (ni == 1) {
        int i = in[0];
        double q[3][3], rq[3];
        for (int m = 0; m < 3; ++m) lerp3(x[i], r[i], d[i], x[out[m]], r[out[m]], d[out[m]], q[m], &rq[m]);
        return emit3(x[i], r[i], q[0], rq[0], q[1], rq[1], q[2], rq[2], p + 1);
    }
    if (ni == 3) {
        /* prism with bottom (i,j,k) and top (a,b,c), a on edge o-i etc. */
        int o = out[0], i = in[0], j = in[1], k = in[2];
        double a[3], b[3], c[3], ra, rb, rc;
        lerp3(x[i], r[i], d[i], x[o], r[o], d[o], a, &ra);
        lerp3(x[j], r[j], d[j], x[o], r[o], d[o], b, &rb);
        lerp3(x[k], r[k], d[k], x[o], r[o], d[o], c, &rc);
        return emit3(x[i], r[i], x[j], r[j], x[k], r[k], a, ra, p + 1) +
               emit3(x[j], r[j], x[k], r[k], a, ra, b, rb, p + 1) +
               emit3(x[k], r[k], a, ra, b, rb, c, rc, p + 1);
    }
    /* ni == 2: wedge with triangles (i, ik, il) and (j, jk, jl) */
    int i = in[0], j = in[1], k = out[0], l = out[1];
    double ik[3], il[3], jk[3], jl[3], rik, ril, rjk, rjl;
    lerp3(x[i], r[i], d[i], x[k], r[k], d[k], ik, &rik);
    lerp3(x[i], r[i], d[i], x[l], r[l], d[l], il, &ril);
    lerp3(x[j], r[j], d[j], x[k], r[k], d[k], jk, &rjk);
    lerp3(x[j], r[j], d[j], x[l], r[l], d[l], jl, &rjl);
    return emit3(x[i], r[i], ik, rik, il, ril, x[j], r[j], p + 1) +
           emit3(ik, rik, il, ril, x[j], r[j], jk, rjk, p + 1) +
           emit3(il, ril, x[j], r[j], jk, rjk, jl, rjl, p + 1);
}

/* ---------------------------------------------------------------------------------------- */
/* 2D: recursive clipping of a triangle by the 4 half-planes 0 <= x_a <= 1                  */
/* ---------------------------------------------------------------------------------------- */

static double tri_mass(const double x[3][2], const double r[3]) {
    double det = (x[1][0] - x[0][0]) * (x[2][1] - x[0][1]) - (x[1][1] - x[0][1]) * (x[2][0] - x[0][0]);
    return fabs(det) * 0.5 * (r[0] + r[1] + r[2]) / 3.0;
}

static void lerp2(const double* xi, double ri, double di, const double* xj, double rj, double dj,
                  double* out, double* rout) {
    double t = di / (di - dj);
    for (int k = 0; k < 2; ++k) out[k] = xi[k] + t * (xj[k] - xi[k]);
    *rout = ri + t * (rj - ri);
}

static double clip2(const double x[3][2], const double r[3], int p);

static double emit2(const double* a, double ra, const double* b, double rb, const double* c, double rc,
                    int p) {
    double x[3][2], r[3];
    x[0][0] = a[0]; x[0][1] = a[1];
    x[1][0] = b[0]; x[1][1] = b[1];
    x[2][0] = c[0]; x[2][1] = c[1];
    r[0] = ra;
    r[1] = rb;
    r[2] = rc;
    return clip2(x, r, p);
}

static double clip2(const double x[3][2], const double r[3], int p) {
    if (p == 4) return tri_mass(x, r);
    double d[3];
    int in[3], out[3], ni = 0, no = 0;
    for (int i = 0; i < 3; ++i) {
        d[i] = hs(x[i], p);
        if (d[i] >= 0.0)
            in[ni++] = i;
        else
            out[no++] = i;
    }
    if (no == 0) return clip2(x, r, p + 1);
    if (ni == 0) return 0.0;
    if (ni == 1) {
        int i = in[0];
        double a[2], b[2], ra, rb;
        lerp2(x[i], r[i], d[i], x[out[0]], r[out[0]], d[out[0]], a, &ra);
        lerp2(x[i], r[i], d[i], x[out[1]], r[out[1]], d[out[1]], b, &rb);
        return emit2(x[i], r[i], a, ra, b, rb, p + 1);
    }
    /* ni == 2: quadrilateral (i, j, jk, ik) */
    int i = in[0], j = in[1], k = out[0];
    double ik[2], jk[2], rik, rjk;
    lerp2(x[i], r[i], d[i], x[k], r[k], d[k], ik, &rik);
    lerp2(x[j], r[j], d[j], x[k], r[k], d[k], jk, &rjk);
    return emit2(x[i], r[i], x[j], r[j], jk, rjk, p + 1) + emit2(x[i], r[i], jk, rjk, ik, rik, p + 1);
}

/* ---------------------------------------------------------------------------------------- */
/* Per-simplex driver                                                                         */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
    int dim;
    long long nv, ns;
    const double* p[3];
    const int* simp;
    const double* rho;
    int n[3];
    double lo[3], len[3], h[3];
    int periodic;
} problem;

/* Vertices of simplex s in grid units, unwrapped to the minimal image of vertex 0. */
static int load_simplex(const problem* P, long long s, double u[4][3], double r[4]) {
    int nvs = P->dim + 1;
    for (int i = 0; i < nvs; ++i) {
        long long v = P->simp[s * nvs + i];
        if (v < 0 || v >= P->nv) return ORACLE_ERR_INDEX;
        for (int a = 0; a < P->dim; ++a) u[i][a] = (P->p[a][v] - P->lo[a]) / P->h[a];
        r[i] = P->rho[v];
    }
    if (P->periodic) {
        for (int i = 1; i < nvs; ++i)
            for (int a = 0; a < P->dim; ++a) {
                double d = u[i][a] - u[0][a];
                double N = (double)P->n[a];
                d -= N * nearbyint(d / N);
                if (fabs(d) >= 0.5 * N) return ORACLE_ERR_EXTENT;
                u[i][a] = u[0][a] + d;
            }
        /* the unwrapped simplex must span less than half the box along every axis: then every
           vertex is also the minimal image of every other one, and the simplex does not depend on
           which vertex is listed first */
        for (int a = 0; a < P->dim; ++a) {
            double mn = u[0][a], mx = u[0][a];
            for (int i = 1; i < nvs; ++i) {
                mn = u[i][a] < mn ? u[i][a] : mn;
                mx = u[i][a] > mx ? u[i][a] : mx;
            }
            if (mx - mn >= 0.5 * (double)P->n[a]) return ORACLE_ERR_EXTENT;
        }
    }
    return ORACLE_OK;
}

static long long cell_index(const problem* P, const long long* c, int* ok) {
    long long idx = 0;
    *ok = 1;
    for (int a = 0; a < P->dim; ++a) {
        long long ca = c[a];
        long long N = P->n[a];
        if (P->periodic) {
            ca %= N;
            if (ca < 0) ca += N;
        } else if (ca < 0 || ca >= N) {
            *ok = 0;
            return -1;
        }
        idx = idx * N + ca;
    }
    return idx;
}

/* mass of simplex s inside cell c (grid units; times cell volume gives world units) */
static double piece_mass(const problem* P, double u[4][3], double r[4], const long long* c) {
    if (P->dim == 3) {
        double x[4][3];
        for (int i = 0; i < 4; ++i)
            for (int a = 0; a < 3; ++a) x[i][a] = u[i][a] - (double)c[a];
        return clip3(x, r, 0);
    } else {
        double x[3][2];
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 2; ++a) x[i][a] = u[i][a] - (double)c[a];
        return clip2(x, r, 0);
    }
}

static int setup(problem* P, int dim, long long nv, long long ns, const double* px, const double* py,
                 const double* pz, const int* simplices, const double* rho, const int* grid,
                 const double* box_lo, const double* box_len, int periodic) {
    if (dim != 2 && dim != 3) return ORACLE_ERR_ARG;
    if (nv < 0 || ns < 0 || !grid || !box_lo || !box_len) return ORACLE_ERR_ARG;
    if (ns > 0 && (!px || !py || (dim == 3 && !pz) || !simplices || !rho)) return ORACLE_ERR_ARG;
    P->dim = dim;
    P->nv = nv;
    P->ns = ns;
    P->p[0] = px;
    P->p[1] = py;
    P->p[2] = pz;
    P->simp = simplices;
    P->rho = rho;
    P->periodic = periodic;
    for (int a = 0; a < dim; ++a) {
        if (grid[a] <= 0 || !(box_len[a] > 0)) return ORACLE_ERR_ARG;
        P->n[a] = grid[a];
        P->lo[a] = box_lo[a];
        P->len[a] = box_len[a];
        P->h[a] = box_len[a] / grid[a];
    }
    return ORACLE_OK;
}

static double cell_volume(const problem* P) {
    double v = 1.0;
    for (int a = 0; a < P->dim; ++a) v *= P->h[a];
    return v;
}

static void atomic_add(double* dst, double v) {
#ifdef _OPENMP
#pragma omp atomic
#endif
    *dst += v;
}

/*
 * Project every simplex; cell_mass[prod(grid)] is ADDED to (the caller zeroes it).  Optional
 * outputs: n_pieces = number of (simplex, cell) pairs with nonzero mass; n_cells_tested = number
 * of (simplex, cell) pairs clipped (bounding-box cells).
 */
int cdo_project(int dim, long long nv, long long ns, const double* px, const double* py, const double* pz,
                const int* simplices, const double* rho, const int* grid, const double* box_lo,
                const double* box_len, int periodic, double* cell_mass, long long* n_pieces,
                long long* n_cells_tested, int nthreads) {
    problem P;
    int rc = setup(&P, dim, nv, ns, px, py, pz, simplices, rho, grid, box_lo, box_len, periodic);
    if (rc) return rc;
    if (!cell_mass) return ORACLE_ERR_ARG;
    double cv = cell_volume(&P);
    int err = ORACLE_OK;
    long long pieces = 0, tested = 0;
#ifdef _OPENMP
    /* the thread count of this call only (the process-wide default stays as it was) */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 256) reduction(+ : pieces, tested)
#endif
    for (long long s = 0; s < ns; ++s) {
        double u[4][3], r[4];
        int e = load_simplex(&P, s, u, r);
        if (e) {
            err = e;
            continue;
        }
        long long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            double mn = u[0][a], mx = u[0][a];
            for (int i = 1; i <= dim; ++i) {
                if (u[i][a] < mn) mn = u[i][a];
                if (u[i][a] > mx) mx = u[i][a];
            }
            lo[a] = (long long)floor(mn);
            hi[a] = (long long)floor(mx);
        }
        long long c[3];
        for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0])
            for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
                for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2]) {
                    int ok;
                    long long idx = cell_index(&P, c, &ok);
                    if (!ok) continue;
                    ++tested;
                    double m = piece_mass(&P, u, r, c);
                    if (m != 0.0) {
                        ++pieces;
                        atomic_add(&cell_mass[idx], m * cv);
                    }
                }
    }
    if (n_pieces) *n_pieces = pieces;
    if (n_cells_tested) *n_cells_tested = tested;
    return err;
}

/*
 * Mass of a few chosen cells only (cells[] = flat C-order indices, out[] = their masses).  Every
 * simplex is visited; only the requested cells of its bounding box are clipped.  Used to check
 * sampled outputs of full-size problems one cell at a time.
 */
int cdo_project_cells(int dim, long long nv, long long ns, const double* px, const double* py,
                      const double* pz, const int* simplices, const double* rho, const int* grid,
                      const double* box_lo, const double* box_len, int periodic, long long ncells,
                      const long long* cells, double* out, int nthreads) {
    problem P;
    int rc = setup(&P, dim, nv, ns, px, py, pz, simplices, rho, grid, box_lo, box_len, periodic);
    if (rc) return rc;
    long long total = 1;
    for (int a = 0; a < dim; ++a) total *= P.n[a];
    /* slot[cell] = position in cells[] + 1 (0 = not requested) */
    int* slot = (int*)calloc((size_t)total, sizeof(int));
    if (!slot) return ORACLE_ERR_ARG;
    for (long long i = 0; i < ncells; ++i) {
        if (cells[i] < 0 || cells[i] >= total) {
            free(slot);
            return ORACLE_ERR_ARG;
        }
        slot[cells[i]] = (int)(i + 1);
        out[i] = 0.0;
    }
    double cv = cell_volume(&P);
    int err = ORACLE_OK;
#ifdef _OPENMP
    /* the thread count of this call only (the process-wide default stays as it was) */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4096)
#endif
    for (long long s = 0; s < ns; ++s) {
        double u[4][3], r[4];
        int e = load_simplex(&P, s, u, r);
        if (e) {
            err = e;
            continue;
        }
        long long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            double mn = u[0][a], mx = u[0][a];
            for (int i = 1; i <= dim; ++i) {
                if (u[i][a] < mn) mn = u[i][a];
                if (u[i][a] > mx) mx = u[i][a];
            }
            lo[a] = (long long)floor(mn);
            hi[a] = (long long)floor(mx);
        }
        long long c[3];
        for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0])
            for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
                for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2]) {
                    int ok;
                    long long idx = cell_index(&P, c, &ok);
                    if (!ok || !slot[idx]) continue;
                    double m = piece_mass(&P, u, r, c);
                    if (m != 0.0) atomic_add(&out[slot[idx] - 1], m * cv);
                }
    }
    free(slot);
    return err;
}

/* Total mass of each simplex, |vol| * mean(rho) (world units). */
int cdo_simplex_mass(int dim, long long nv, long long ns, const double* px, const double* py,
                     const double* pz, const int* simplices, const double* rho, const int* grid,
                     const double* box_lo, const double* box_len, int periodic, double* out) {
    problem P;
    int rc = setup(&P, dim, nv, ns, px, py, pz, simplices, rho, grid, box_lo, box_len, periodic);
    if (rc) return rc;
    double cv = cell_volume(&P);
    for (long long s = 0; s < ns; ++s) {
        double u[4][3], r[4];
        int e = load_simplex(&P, s, u, r);
        if (e) return e;
        if (dim == 3) {
            out[s] = tet_mass(u, r) * cv;
        } else {
            double x[3][2];
            for (int i = 0; i < 3; ++i) {
                x[i][0] = u[i][0];
                x[i][1] = u[i][1];
            }
            out[s] = tri_mass(x, r) * cv;
        }
    }
    return ORACLE_OK;
}

int cdo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
