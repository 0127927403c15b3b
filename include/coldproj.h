/*
 * coldproj — exact projection of a piecewise-linear density carried by a simplicial mesh onto a
 * regular grid, on one NVIDIA GB300 (sm_103a), behind a plain C ABI.
 *
 * The method is the exact projection of Sousbie & Colombi, "ColDICE: a parallel Vlasov-Poisson
 * solver using moving adaptive simplicial tessellation" (arXiv:1509.07720), Sect. 3 and
 * Appendices C-E: the mass of every grid cell is the integral, over the cell, of the linear
 * interpolation of the per-vertex densities inside every simplex, evaluated exactly as a sum of
 * Franklin vertex/edge/facet contributions (Sect. 3.1, eqs. firstOrder, contrib, E0, E1) over the
 * corners of every (simplex intersect cell) polyhedron (Sect. 3.2, corner types A-D), with exact
 * predicates and simulation of simplicity (Sect. 3.3, eq. sos; Appendix E).
 *
 * Conventions shared by every entry point:
 *  - All array arguments are DEVICE pointers (current CUDA device of the context) unless stated
 *    otherwise; the caller owns them and keeps them alive until the work on `stream` is done.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Every call
 *    only enqueues work on it and returns; results are valid once the stream has reached them.
 *  - Return value: CDP_OK (0) or a negative CDP_ERR_* code; no C++ exception crosses the ABI and
 *    nothing aborts. Argument errors are detected on the host before anything is enqueued.
 *    Errors found by the kernels (bad vertex index, non-finite coordinate, a simplex too large)
 *    are recorded in the context and returned by cdp_check (or by cdp_project when it is given a
 *    stats block, which makes it synchronise).
 *  - A context is not thread-safe and its scratch memory is reused by every call: do not run two
 *    calls with one context on two streams at the same time.
 *  - Grids are C order with axis 0 slowest: cell (i, j, k) of an (n0, n1, n2) grid is element
 *    (i * n1 + j) * n2 + k. Cell (i, j, k) covers [lo + i h, lo + (i + 1) h) per axis, h = len / n.
 */
#ifndef COLDPROJ_H
#define COLDPROJ_H

#include <stdint.h>

#if defined(__GNUC__)
#define CDP_API __attribute__((visibility("default")))
#else
#define CDP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CDP_OK = 0,
    CDP_ERR_ARG = -1,     /* invalid argument (null pointer, bad size, bad dimension) */
    CDP_ERR_INDEX = -2,   /* a simplex refers to a vertex index outside [0, n_verts) */
    CDP_ERR_NAN = -3,     /* a vertex coordinate or density is not finite, or absurdly far out */
    CDP_ERR_EXTENT = -4,  /* a simplex spans half a periodic box or more, or > 2048 cells per axis */
    CDP_ERR_OOM = -5,     /* device scratch allocation failed */
    CDP_ERR_TIMEOUT = -6, /* reserved for a bounded device-side wait that gives up; no kernel of this
                             library waits on another, so no call returns it at present */
    CDP_ERR_CUDA = -7     /* a CUDA runtime or library call failed */
};

/* Arithmetic of the projection. Both paths take the same exact combinatorial decisions.
 * CDP_FP64: every contribution in FP64; stated accuracy 1e-11 of the largest cell (typically ~1e-13).
 * CDP_FP32_MIXED: contributions in FP32, classification exact (integer) with an FP32 filter,
 *   accumulation of every (simplex, cell) piece into the FP64 grid; stated accuracy 1e-5 of the
 *   largest cell (typically ~1e-6).
 * Both paths control their accuracy (Sect. 3.4; cdp_stats.n_deferred / n_clipped): simplices whose
 * density gradient would make Franklin's sum cancel beyond the stated accuracy are projected by
 * clipping instead.  Total mass: FP64 exact to ~1e-12 relative; FP32-mixed closes the mass of every
 * simplex against its FP64 closed form, so the total is exact to ~1e-12 as well, EXCEPT for simplices
 * that cross the walls of a non-periodic box: the closure knows the mass of the whole simplex, not
 * of its part inside the box, and the total inside the box is then only as exact as the cells
 * (~1e-5 of the largest cell). */
enum { CDP_FP64 = 0, CDP_FP32_MIXED = 1 };
/* OR'ed into a precision argument: no accuracy control -- every simplex is projected by Franklin's
 * sum in the requested arithmetic (faster, but the stated accuracy is then not guaranteed for
 * simplices whose density gradient is steep compared with their density; for measurements and for
 * comparing the two arithmetics on the same work). */
#define CDP_ACCURACY_OFF 0x100

typedef struct cdp_ctx cdp_ctx;

/* One projection problem (Algorithm 2's inputs and output).
 *   dim          2 (triangles) or 3 (tetrahedra)
 *   n_verts      number of vertices; n_simplices number of simplices (0 allowed)
 *   pos[a]       device, double[n_verts]: coordinate a of every vertex (world units), a < dim
 *   simplices    device, int32[n_simplices * (dim + 1)]: vertex indices, one row per simplex;
 *                any vertex order and orientation (inverted simplices are fine, mass is +|V| rho)
 *   rho          device, double[n_verts]: density at every vertex (linear inside each simplex)
 *   grid[a]      cells per axis (1 <= grid[a] <= 2^20, at most 2^32 cells in total), a < dim
 *   box_lo/len   box origin and side lengths (len > 0)
 *   periodic     1: the box is a torus, every simplex is taken at the minimal image of its
 *                vertex 0 and cells wrap; every simplex must span less than half the box along
                every axis (so that every vertex is the minimal image of every other one and the
                simplex does not depend on its vertex order), else CDP_ERR_EXTENT;
 *                0: mass outside the grid is dropped
 *   cell_mass    device, double[prod(grid)]: OUTPUT, integral of rho over every cell */
typedef struct {
    int dim;
    int64_t n_verts;
    int64_t n_simplices;
    const double* pos[3];
    const int32_t* simplices;
    const double* rho;
    int32_t grid[3];
    double box_lo[3];
    double box_len[3];
    int periodic;
    double* cell_mass;
} cdp_problem;

/* Counters of one projection (filled when a stats block is passed). */
typedef struct {
    uint64_t n_zero_volume;   /* simplices of zero volume (no contribution) */
    uint64_t n_single_cell;   /* simplices inside one cell (closed form, Algorithm 2 step 1) */
    uint64_t n_small;         /* simplices projected by the main kernel (3D: bounding box <= 1920 cells) */
    uint64_t n_large;         /* tetrahedra with a larger bounding box: projected tile by tile (23^3 cells)
                                 by the large-tetrahedron kernel */
    uint64_t n_large_tiles;   /* tiles of those tetrahedra */
    uint64_t corners_a;       /* (corner, cell) incidences of type A: grid node inside a simplex */
    uint64_t corners_b;       /* type B: simplex vertex */
    uint64_t corners_c;       /* type C: simplex edge x cell face */
    uint64_t corners_d;       /* type D: simplex facet x cell edge (3D) */
    uint64_t exact_fallbacks; /* predicate evaluations decided by the exact integer stage */
    uint64_t large_corners[4];/* the part of corners_a..d found on the tiles of the large tetrahedra (A, B, C, D);
                                 a corner on a tile face is evaluated, and counted, in each tile it touches */
    uint32_t error_flags;     /* bit 0 bad index, bit 1 non-finite, bit 2 extent */
    uint32_t reserved;
    /* accuracy control (Sect. 3.4): a simplex whose density gradient is steep compared with its density
       is deferred by the first pass; once the largest cell mass M of the first pass is known it is
       projected by Franklin's sum if the bound on its cancellation error is below half the stated
       accuracy (FP32-mixed 1e-5, FP64 1e-11, of M), and otherwise by clipping it against every cell of its
       bounding box (a second algorithm, free of cancellation) */
    uint64_t n_deferred;      /* simplices deferred by the first pass */
    uint64_t n_clipped;       /* simplices projected by clipping */
    double accuracy_bound;    /* largest error bound of a piece of a simplex projected by Franklin's sum,
                                 divided by the largest |cell mass| (a measured-constant bound, see the
                                 accuracy constants in the sources; the stated accuracy is 1e-5 / 1e-11) */
} cdp_stats;

/* Create a context on CUDA device `device` (scratch is allocated lazily and grown as needed).
 * *out receives the context; returns CDP_ERR_ARG / CDP_ERR_CUDA on failure. */
CDP_API int cdp_create(cdp_ctx** out, int device);

/* Free the context and its scratch (synchronises the device first). NULL is ignored. */
CDP_API void cdp_destroy(cdp_ctx* ctx);

/* Exact projection of one mesh (Sect. 3; Algorithm 2): prob->cell_mass[V] = sum over simplices S
 * of the integral over S intersect V of the linear interpolant of rho.
 *   precision    CDP_FP64 or CDP_FP32_MIXED
 *   accumulate   0: cell_mass is overwritten; 1: the projection is added to it
 *   stats        NULL: asynchronous; otherwise the call synchronises `stream`, fills *stats and
 *                returns any error the kernels found.
 * Scratch: 32 bytes per vertex + 4 bytes per simplex (context-owned). */
CDP_API int cdp_project(cdp_ctx* ctx, const cdp_problem* prob, int precision, int accumulate, void* stream,
                cdp_stats* stats);

/* Several projections in one call, enqueued back to back on `stream` (each as cdp_project with
 * accumulate = 0 and no stats).  The scratch is sized once for the largest problem first. */
CDP_API int cdp_project_batched(cdp_ctx* ctx, const cdp_problem* probs, int n, int precision, void* stream);

/* Projection through a hierarchy of coarser grids and donor-cell gather onto prob's grid (Sect. 4.4,
 * calculation of the acceleration: the AMR grid is refined down to the smallest perpendicular height
 * of the simplices crossing it, the projection onto its cells is exact, and the Poisson grid takes
 * their masses by a donor-cell gather).  Level l (0 .. max_level) is prob's grid with every axis
 * divided by 2^l.  Each simplex is projected exactly onto one level: the coarsest whose cells are no
 * larger than its smallest perpendicular height eta (D |volume| / largest facet measure, in cells of
 * prob's grid), i.e. l = min(max_level, floor(log2 eta)), and l = 0 for eta < 2.  Then every cell of
 * prob's grid receives its own mass plus, for each l >= 1, the mass of the level-l cell containing
 * it divided by 2^(D l).  The total mass is that of cdp_project; the mass inside a level-l cell is
 * spread evenly over the 2^(D l) cells it covers.
 *   max_level    0 .. CDP_AMR_MAX_LEVEL; every prob->grid[a] must be divisible by 2^max_level
 *                (CDP_ERR_ARG otherwise); 0 is exactly cdp_project
 *   precision, accumulate, stream, stats   as cdp_project (the stats count the simplices of all
 *                levels; accuracy_bound is relative to the largest cell mass of prob's grid)
 * Scratch (context-owned): the coarse levels' cells (8 bytes each, under 1/7 of prob's grid in 3D)
 * and one byte per simplex; the vertex records are made once per level. */
#define CDP_AMR_MAX_LEVEL 6
CDP_API int cdp_project_amr(cdp_ctx* ctx, const cdp_problem* prob, int precision, int max_level, int accumulate,
                            void* stream, cdp_stats* stats);

/* Largest n_verts and n_simplices accepted by cdp_project_noalloc, and the size of its static
 * device scratch, held by every process that loads the library on every device it uses: 32 bytes
 * per vertex (8 MiB), three lists of 4 bytes per simplex (large, deferred and clipped simplices,
 * 18 MiB), and the geometry records of one batch of 16,384 tetrahedra (9.5 MiB), 37,291,008 bytes
 * in all with the counters and box sizes. */
#define CDP_NOALLOC_MAX_VERTS 262144
#define CDP_NOALLOC_MAX_SIMPLICES 1572864
#define CDP_NOALLOC_SCRATCH_BYTES 37291008

/* The projection of cdp_project (same kernels, same results to the stated accuracy), for callers
 * that must not allocate or free memory when they call: for instance a caller whose framework has
 * reserved the device memory for its own pool, or one that cannot afford the device-wide
 * synchronisation that cudaFree implies while other streams are busy.  It takes no context: its
 * scratch (counters, vertex records, the lists of large, deferred and clipped simplices, and the
 * geometry records of one batch of tetrahedra) is one fixed device array of this library of
 * CDP_NOALLOC_SCRATCH_BYTES bytes, and it calls no allocating routine.  The paper has no
 * counterpart of this entry point; it exists only for the allocation constraint above.
 *  - Throughput: the geometry records are set up 16,384 tetrahedra at a time (cdp_project: up to
 *    2^24), so a problem of n tetrahedra takes ceil(n / 16384) set-up and main-kernel launch pairs
 *    (96 at the 1,572,864-tetrahedron limit), and FP32 tiles of large tetrahedra are computed twice
 *    (no tile store): expect it to be slower than cdp_project on large problems.
 *  - Runs on the CURRENT CUDA device.  The first call on a device looks up the scratch address
 *    and the launch parameters of that device (no allocation); make that first call before any
 *    stream capture is begun.
 *  - n_verts > CDP_NOALLOC_MAX_VERTS or n_simplices > CDP_NOALLOC_MAX_SIMPLICES returns
 *    CDP_ERR_ARG before anything is enqueued; other
 *    argument checks are those of cdp_project.
 *  - Every call on a device shares the one scratch array: two calls whose work overlaps on the
 *    GPU (two streams, or two host threads) race and both results are undefined.  Serialise them
 *    (one stream, or events between the streams).
 *  - error_flags: optional device pointer to one uint32_t; when the call's work has run it holds
 *    the bits of cdp_stats.error_flags for this call (0 = no error).  NULL: errors are not
 *    reported.
 *  - accumulate and precision as in cdp_project.  Only enqueues; nothing synchronises. */
CDP_API int cdp_project_noalloc(const cdp_problem* prob, int precision, int accumulate, uint32_t* error_flags,
                                void* stream);

/* Vertex densities from simplex masses (Sect. 4.4): rho_out[j] = sum of simplex_mass[i] over the
 * simplices i that have vertex j, divided by the sum of their volumes |V_i| (world units,
 * periodic minimal image when prob->periodic).  Uses dim, n_verts, n_simplices, pos, simplices,
 * box_len and periodic of `prob` (its rho and cell_mass are ignored).  simplex_mass: device
 * double[n_simplices]; rho_out: device double[n_verts] (0 for a vertex with no simplex).
 * Scratch: 16 bytes per vertex. */
CDP_API int cdp_vertex_density(cdp_ctx* ctx, const cdp_problem* prob, const double* simplex_mass, double* rho_out,
                               void* stream);

/* Periodic FFT Poisson solve (Sect. 4.4): laplacian(phi) = four_pi_G (rho - mean(rho)) with
 * rho = cell_mass / cell volume, continuous Green function -1/k^2 (k = 2 pi n / L), zero mode
 * removed.  cell_mass, phi: device double[prod(grid)] (C order, cell-centred); phi may alias
 * cell_mass.  cuFFT plans and the spectrum buffer are cached in the context per grid shape. */
CDP_API int cdp_poisson(cdp_ctx* ctx, int dim, const int32_t grid[3], const double box_len[3], double four_pi_G,
                        const double* cell_mass, double* phi, void* stream);

/* Acceleration at n points (Sect. 4.4): acc = - sum over the 3^dim nearest cell centres of the
 * triangular-shaped-cloud weight times the 4-point central difference
 * (8 (phi[i+1] - phi[i-1]) - (phi[i+2] - phi[i-2])) / (12 h) of phi there (periodic grid).
 * pos[a], acc[a]: device double[n], a < dim. */
CDP_API int cdp_force(cdp_ctx* ctx, int dim, const int32_t grid[3], const double box_lo[3], const double box_len[3],
                      const double* phi, int64_t n, const double* const pos[3], double* const acc[3], void* stream);

/* Drift (eqs. drift1, drift2): pos[a] += vel[a] * dt, wrapped into [box_lo, box_lo + box_len)
 * when periodic.  Kick (eq. kick): vel[a] += acc[a] * dt.  Device double[n] arrays, a < dim. */
CDP_API int cdp_drift(cdp_ctx* ctx, int dim, int64_t n, double* const pos[3], const double* const vel[3], double dt,
                      const double box_lo[3], const double box_len[3], int periodic, void* stream);
CDP_API int cdp_kick(cdp_ctx* ctx, int dim, int64_t n, double* const vel[3], const double* const acc[3], double dt,
                     void* stream);

/* One mesh of a batched time step.  mesh.pos is updated in place by the drifts (the pointers
 * are written through), mesh.rho receives the vertex densities, mesh.cell_mass the projection;
 * the box must be periodic. */
typedef struct {
    cdp_problem mesh;
    double* vel[3];             /* device double[n_verts]: velocities, updated by the kick */
    double* acc[3];             /* device double[n_verts]: accelerations, written */
    const double* simplex_mass; /* device double[n_simplices]: fixed masses of the simplices */
    double* phi;                /* device double[prod(grid)]: potential, written */
} cdp_step_problem;

/* One time step of n independent meshes (Sect. 4, steps (ii)-(iv)): drift dt/2 (eq. drift1),
 * vertex densities from the simplex masses, exact projection, FFT Poisson solve, force at the
 * vertices, kick dt (eq. kick), drift dt/2 (eq. drift2).  use_graph != 0: the first call with a
 * given argument array captures the whole sequence into a CUDA graph owned by the context and
 * every later call with byte-identical arguments (dt may differ) replays it in one launch.  The
 * first call also creates the FFT plans and sizes the scratch outside the capture.  A graph holds
 * the addresses of the context's scratch: once a later call on the context reallocates it (a
 * larger projection or vertex density) or cdp_autotune retunes the launch shapes, the graphs
 * recorded before are dropped and the next call with their arguments records the step again.
 *   precision   CDP_FP64: every step in FP64.  CDP_FP32_MIXED: the projection in FP32-mixed and the
 *               Poisson transforms in single precision (the source and the potential stay FP64
 *               arrays; on the 64-problem batched workload the potential is within 1.4e-5 of its
 *               largest value of the FP64 step's, the cell masses within 3.5e-6); the other steps
 *               in FP64. */
CDP_API int cdp_step_batched(cdp_ctx* ctx, const cdp_step_problem* probs, int n, int precision, double dt,
                             double four_pi_G, int use_graph, void* stream);

/* Synchronise `stream` and return the first error the kernels recorded since the last check
 * (and clear it). */
CDP_API int cdp_check(cdp_ctx* ctx, void* stream);

/* Per-kernel timing (instrumentation, off by default).  With `enable` != 0 every later
 * cdp_project records CUDA events around each of its kernels on its stream and adds the elapsed
 * times to per-kernel totals; enabling (or disabling) also resets the totals and the call count. */
CDP_API int cdp_timing_enable(cdp_ctx* ctx, int enable);

/* Synchronise the recorded events and copy the totals (milliseconds) into out_ms[0..n-1], n <= 5:
 * [0] vertex records, [1] per-simplex set-up (3D: the first batch's; the single-cell closed form
 * is applied there), [2] main projection kernel (3D: with the set-up of any later batch),
 * [3] the large-tetrahedron kernel (3D: tetrahedra with a bounding box above 1920 cells, in
 * tiles), [4] the accuracy control (the largest cell mass, the second pass over the deferred
 * simplices, clipping).  *calls receives the number of timed cdp_project calls.  Returns the
 * number of slots written. */
CDP_API int cdp_timing_read(cdp_ctx* ctx, double* out_ms, int n, int* calls);

/* Launch-shape tuning (no counterpart in the paper: the choice of a GPU launch shape).  Times the
 * projection of `prob` (into its own cell_mass, which is overwritten) while tuning, one after the
 * other, three knobs of the context's later projections with the same dimension and precision:
 *   - the main kernel's persistent grid: 1, 2, 4 or 8 times the device's resident blocks (default 8);
 *   - 3D, the size-class threshold: the largest bounding box (cells) a tetrahedron of the main kernel
 *     may have -- larger ones are tiled by the large-tetrahedron kernel -- among 960, 1920 (the
 *     default), 3840 and the block's box slots (6144 FP32, 10240 FP64);
 *   - 3D, the tile edge of the large tetrahedra: 18 or 23 cells (default 23).
 * Each setting is kept only if it is faster than the best so far.  With a non-null cache_path the
 * choice is first looked up in that text file (lines "<device> dim<D> <precision> <multiplier>
 * <threshold> <edge>"; the last entry of a key wins) and, when tuned, appended to it.
 * Synchronises with the device.  chosen (optional) receives int[3]: the multiplier, the threshold and
 * the edge (the last two 0 in 2D).  Returns CDP_OK, CDP_ERR_ARG, an error of the projection, or
 * CDP_ERR_CUDA. */
CDP_API int cdp_autotune(cdp_ctx* ctx, const cdp_problem* prob, int precision, const char* cache_path,
                         int* chosen);

/* Human-readable name of a return code (static string). */
CDP_API const char* cdp_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* COLDPROJ_H */
