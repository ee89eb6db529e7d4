/*
 * npfem.h -- C ABI of the GB300 npFEM cell-suspension solver.
 *
 * The library advances a batch of closed triangulated membranes (red blood
 * cells, platelets) through implicit-Euler time steps of the nodal projective
 * FEM solver of arXiv 1911.03062 (Supplementary Sec. 2.1):
 *
 *   v_{n+1} = (x_{n+1} - x_n) / h                                   Eq. (vel)
 *   x_{n+1} = argmin g(x),  g(x) = 1/(2h^2) (x - y_n)^T Mt (x - y_n) + sum_i E_i(x)
 *   y_n     = x_n + h Mt^{-1} (M v_n + h F_ext),  Mt = M + h C       Eq. (genericOptimizationNewton)
 *
 * minimised by a fixed number of quasi-Newton iterations
 * x^{k+1} = x^k - H grad g(x^k) (the unnumbered update after that equation),
 * with H an L-BFGS operator whose initial matrix is the inverse of the
 * constant SPD matrix P = Mt/h^2 + sum_i w_i A_i^T A_i of the quadratic
 * (projective) energies, and an Armijo line search.  C is the Rayleigh
 * damping of Eq. (Newton2nd), zero unless the material sets it (then y_n =
 * x_n + h v_n + h^2 M^{-1} F_ext).
 *
 * Conventions for every call below
 *  - Return value: NPFEM_OK (0) or a negative NPFEM_E* code; the message of
 *    the last failure is available from npfem_last_error().
 *  - Host arrays are read or written during the call only; the caller keeps
 *    ownership.  The context owns all device memory it allocates.
 *  - Per-cell arrays use the public layout: cell-major in the order cells were
 *    added, each cell nV_type x 3 doubles (vertex major, xyz innermost).
 *  - Units are the caller's (the workloads are non-dimensional).
 *  - A context is used by one host thread at a time.  All device work of a
 *    context runs on its stream (npfem_options.cuda_stream or a stream the
 *    context creates).
 */
#ifndef NPFEM_H
#define NPFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NPFEM_OK 0
#define NPFEM_EINVAL -1      /* bad argument, size, or mesh (open, non-manifold, degenerate) */
#define NPFEM_ENOMEM -2      /* device or host allocation failed */
#define NPFEM_ENOTSPD -3     /* the system matrix P is not positive definite */
#define NPFEM_ECUDA -4       /* a CUDA call failed (message names it) */
#define NPFEM_ENONFINITE -5  /* NaN/Inf in forces or state; message names the cell */
#define NPFEM_ETIMEOUT -6    /* a bounded device wait expired (kernel returned early) */
#define NPFEM_ESTATE -7      /* call not valid in the current state */

#define NPFEM_MAX_HISTORY 8

typedef struct npfem_ctx npfem_ctx;

/* Arithmetic of the global-step apply z = P^{-1} q.
 *  NPFEM_FP64        : everything in FP64 (SIMT); the comparison form.
 *  NPFEM_MIXED_TF32  : FP32 local step; P^{-1} q on tcgen05 tensor cores in
 *                      TF32 with FP32 accumulation, refined against an FP64
 *                      residual q - P z until |r|/|q| <= refine_tol.
 *  NPFEM_MIXED_BF16  : as above with BF16 operands. */
typedef enum { NPFEM_FP64 = 0, NPFEM_MIXED_TF32 = 1, NPFEM_MIXED_BF16 = 2 } npfem_precision;

typedef struct {
    int precision;          /* npfem_precision */
    int iters;              /* K quasi-Newton iterations per step (default 10) */
    int history;            /* L-BFGS history m, 0..NPFEM_MAX_HISTORY (default 5) */
    double armijo_c1;       /* sufficient-decrease constant (default 1e-4) */
    int max_backtracks;     /* halvings of the step before the last trial is taken (default 8) */
    double refine_tol;      /* mixed forms: target |q - P z| / |q| per cell and component (default 1e-6) */
    int refine_max;         /* mixed forms: maximum refinement sweeps (default 3) */
    int use_graph;          /* capture one step as a CUDA graph and replay it (default 1) */
    int device;             /* CUDA device ordinal (default 0) */
    void *cuda_stream;      /* cudaStream_t to run on, or NULL for a context-owned stream */
    const char *autotune_cache; /* file for tuned GEMM tile choices, or NULL (tune, keep in memory) */
    int residual_fp64;      /* mixed forms: refinement residual with FP64 arithmetic (1) or with exact
                               FP32 fused multiply-adds on a float-pair diagonal (0, default); both
                               evaluate q - diag(P) z without cancellation error */
    int refine_split;       /* BF16 form: refinement corrections with P^{-1} and r each split into
                               a BF16 high part and a BF16 low part, three tensor-core products
                               (r_hi P_hi + r_lo P_hi + r_hi P_lo) accumulated in FP32, so one
                               correction reduces the residual ~100x further than a plain BF16
                               one (1, default); plain BF16 corrections (0) */
    int force_median;       /* 1: before each step, replace every vertex force by the component-wise
                               median over the vertex and its edge neighbours (closed one-ring; even
                               count: mean of the two middle values); paper Sec. 2.2.  Default 0.
                               Meshes with a vertex of more than 31 neighbours are rejected (EINVAL). */
    double u_max;           /* > 0: after each step, vertex velocities with |v| > u_max are scaled to
                               |v| = u_max (direction kept), in the state; paper Sec. 2.2.  Default 0
                               (off). */
    double pbd_kappa;       /* in [0, 1]: after each step (before the velocity cap), position-based-
                               dynamics velocity damping per cell: the rigid part of the velocity
                               field (centre-of-mass velocity + omega x r, omega = I^{-1} L) is kept,
                               the rest scaled by 1 - pbd_kappa; paper Sec. 2.1 (kappa_damping),
                               Mueller et al. 2007.  Default 0 (off). */
    double pik_radius;      /* > 0: particle-in-kernel collisions (paper Sec. 2.2, supplementary PIK
                               section), kernel radius rk.  At the start of each step every vertex
                               whose sphere of radius rk holds vertices of other cells takes the
                               closest one (ties: lower public cell, then vertex index) as its
                               colliding neighbour j: its external force is dropped for the step and
                               g gains collision_k/2 |x_i - p_i|^2, p_i = x_i + (rk - s) n_j,
                               s = (x_i - x_j).n_j, n_j the area-weighted vertex normal of j, all at
                               the start-of-step positions.  P is unchanged (the term's curvature
                               enters through the L-BFGS pairs).  Default 0 (off). */
    double collision_k;     /* stiffness of the collision energy; > 0 when pik_radius > 0 */
    double curvature_tol;   /* an iteration's pair (s, y) enters the L-BFGS history only if
                               s.y > curvature_tol |s| |y| (default 1e-12, which keeps every H
                               positive definite).  A negative value also admits pairs of
                               negative curvature (-INFINITY: every pair); the descent test then
                               catches an uphill direction, clears the history and takes
                               -P^{-1} grad g.  NaN is rejected (EINVAL). */
} npfem_options;

/* Material and time step of one mesh type.  Element weights follow the
 * projective-dynamics reading of the paper's energies: w_strain = k_strain *
 * rest area, w_area = k_area * rest area (per triangle), w_bend = k_bend (per
 * interior edge), w_vol = k_vol (per cell).
 * Rayleigh damping (Supp. Sec. 2.1, Eq. (Newton2nd); the paper's parameter
 * table uses alpha = 0, beta = 0.01): C = rayleigh_alpha M + rayleigh_beta L
 * with L = sum_i w_i A_i^T A_i (volume term included), the constant stiffness
 * of the quadratic energies.  Both >= 0; zero (the default of a zeroed
 * struct) is the undamped step.  A damped type keeps Mt^{-1} beside P^{-1}
 * and applies it once per step for the predictor, in FP64 (FP64 form), TF32,
 * or BF16 split into high and low parts (BF16 form, whatever refine_split). */
typedef struct {
    double k_strain, k_area, k_bend, k_vol;
    double dt;              /* h */
    double rayleigh_alpha, rayleigh_beta;
} npfem_material;

/* Per-step counters of the last completed npfem_step (summed over cells). */
typedef struct {
    int64_t cell_iterations;   /* cells x K */
    int64_t backtracks;        /* line-search halvings */
    int64_t capped_searches;   /* searches that hit max_backtracks */
    int64_t fallbacks;         /* non-descent directions replaced by -P^{-1} grad g */
    int64_t refine_sweeps;     /* refinement sweeps applied (mixed forms) */
    double max_refine_residual;/* largest final |q - P z|/|q| seen (mixed forms) */
    double energy_sum;         /* sum over cells of g(x_{n+1}) */
    int64_t launches_per_step; /* kernels one npfem_step launches */
    int64_t contacts;          /* vertices that found a colliding neighbour (pik_radius > 0) */
} npfem_step_stats;

/* Kernel classes of the per-kernel timing (npfem_profile_read). */
#define NPFEM_K_PREDICT 0        /* inertial predictor + first local step */
#define NPFEM_K_ITERATE 1        /* fused L-BFGS + line search + local steps */
#define NPFEM_K_FALLBACK 2       /* the same kernel over non-descent cells */
#define NPFEM_K_GEMM 3           /* global-step apply z = P^{-1} q */
#define NPFEM_K_GEMM_REFINE 4    /* refinement correction applies */
#define NPFEM_K_RESIDUAL 5       /* FP64 refinement residuals */
#define NPFEM_K_FALLBACK_APPLY 6 /* P^{-1} grad for non-descent cells */
#define NPFEM_K_FILTER 7         /* force median filter, velocity cap, PBD damping */
#define NPFEM_K_CONTACT 8        /* particle-in-kernel search and collision targets */
#define NPFEM_KCLASSES 9

typedef struct {
    double ms[NPFEM_KCLASSES];         /* summed CUDA-event time per class */
    int64_t launches[NPFEM_KCLASSES];  /* launches timed per class */
} npfem_kernel_times;

/* Fill *opt with the defaults listed above. */
void npfem_default_options(npfem_options *opt);

/* Create a context on opt->device.  opt may be NULL (defaults).
 * Errors: EINVAL (bad option values), ECUDA, ENOMEM. */
int npfem_create(const npfem_options *opt, npfem_ctx **out);

/* Release every resource of the context (NULL is ignored). */
void npfem_destroy(npfem_ctx *ctx);

/* Register a mesh type: a closed, consistently oriented (outward CCW)
 * triangle surface with its rest shape, lumped vertex masses and material.
 *   nV, rest_xyz : nV x 3 rest positions (the rest state of every cell of the type)
 *   nT, tris     : nT x 3 vertex indices
 *   vertex_mass  : nV masses, or NULL for 1/nV each (total mass 1; Supp. Sec. 2.1
 *                  lumps the cell mass on its vertices)
 * Builds the type's element constants and P (Supp. Sec. 2.1, the Hessian
 * approximation "of quadratic form"), inverts P once on the GPU in FP64 and
 * keeps P^{-1} (and its TF32/BF16 copy in the mixed forms).
 * Errors: EINVAL (nV < 4, index out of range, open or non-manifold mesh,
 * inconsistent orientation, degenerate triangle, inward orientation,
 * non-positive mass or dt, negative or non-finite damping), ENOTSPD, ENOMEM, ECUDA, ESTATE (after cells were
 * added to a graph-captured context the call is still allowed; the graph is
 * rebuilt on the next step). */
int npfem_create_mesh_type(npfem_ctx *ctx, int nV, const double *rest_xyz,
                           int nT, const int32_t *tris, const double *vertex_mass,
                           const npfem_material *mat, int *type_id);

/* Append n_cells cells of type type_id with initial positions x0 and
 * velocities v0 (NULL = zero), both n_cells x nV x 3 doubles.  The new cells
 * follow all earlier cells in the public layout; *first_cell (may be NULL)
 * receives the index of the first new cell.
 * Errors: EINVAL (unknown type, n_cells < 0), ENONFINITE, ENOMEM, ECUDA. */
int npfem_add_cells(npfem_ctx *ctx, int type_id, int n_cells, const double *x0,
                    const double *v0, int64_t *first_cell);

/* Number of doubles of one per-cell array over all cells (sum of 3 nV). */
size_t npfem_num_dofs(const npfem_ctx *ctx);

/* Advance every cell by one time step of its type's h under the external
 * forces f_ext (npfem_num_dofs doubles, public layout).  f_ext_on_device != 0
 * means f_ext is a device pointer read on the context's stream (no copy): the
 * caller's writes of it must be complete before that stream reaches the step
 * (e.g. the same stream, or an event the stream waits on), and it must stay
 * valid and unchanged until the step has run (npfem_sync, or an event recorded
 * on the stream after the call).  Otherwise it is host memory, copied to the
 * device in the call; for page-locked memory that copy runs asynchronously, so
 * keep the buffer unchanged until the next synchronising call.  Unless a force
 * filter, the collision search or a damped type reads the forces first, the
 * copy goes in four pieces on a second stream of the library's while the
 * predictor starts on the cells whose forces are in (the step's results are
 * the same bits as with device forces).
 * The call enqueues the work and returns; device errors are reported by the
 * next call that synchronises (get_*, stats, npfem_sync).
 * Errors: EINVAL, ESTATE (no cells), ECUDA. */
int npfem_step(npfem_ctx *ctx, const double *f_ext, int f_ext_on_device);

/* Wait for the context's stream; report device-side errors (ENONFINITE with
 * the cell index, ETIMEOUT) raised since the last synchronising call. */
int npfem_sync(npfem_ctx *ctx);

/* Copy the current positions / velocities (n_doubles must equal
 * npfem_num_dofs) into out: host memory, or device memory when
 * out_on_device != 0.  Synchronises the stream.  Errors: EINVAL, ECUDA and
 * pending device errors. */
int npfem_get_positions(npfem_ctx *ctx, double *out, size_t n_doubles, int out_on_device);
int npfem_get_velocities(npfem_ctx *ctx, double *out, size_t n_doubles, int out_on_device);

/* Replace the state of all cells (checkpoint resume).  v may be NULL (zero).
 * Errors: EINVAL, ENONFINITE, ECUDA. */
int npfem_set_state(npfem_ctx *ctx, const double *x, const double *v, size_t n_doubles);

/* Counters of the last completed step (synchronises). */
int npfem_stats(npfem_ctx *ctx, npfem_step_stats *out);

/* Global-step building block: z = P^{-1} q for n_cols right-hand sides of
 * mesh type type_id, through the same apply (and, in the mixed forms, the
 * same refinement) as npfem_step.  q, z: device pointers, n_cols x nV
 * doubles (one column = one component of one cell, vertex contiguous), read
 * and written on the context's stream: q must be complete before that stream
 * reaches the call.  The call synchronises the stream before it returns, so z
 * is complete on return (this holds for npfem_apply_pinv_noalloc too).
 * Errors: EINVAL, ENOMEM, ECUDA. */
int npfem_apply_pinv(npfem_ctx *ctx, int type_id, const double *q, double *z, int n_cols);

/* Allocation-free variant of npfem_apply_pinv, for callers that cannot let
 * the library allocate device memory: code whose GPU memory is entirely owned
 * by another allocator (a framework's caching allocator that has reserved the
 * device, a fixed memory budget), and latency-critical loops where the
 * implicit device synchronisation of cudaMalloc/cudaFree would stall the
 * pipeline.  No counterpart in the paper: it is a deployment convenience.
 *
 * Same arguments, result and refinement as npfem_apply_pinv; the caller still
 * provides q and z (device pointers, n_cols x nV doubles).  The temporaries
 * live in one static device array (16 x NPFEM_NOALLOC_MAX_ELEMS bytes + 1 MiB, about 33 MB)
 * that every GPU which loads the library holds until the process exits; no
 * call allocates or frees memory.
 *  - Limit: 3 * ceil(n_cols / 3) * nVp <= NPFEM_NOALLOC_MAX_ELEMS (2^21)
 *    scratch elements, nVp = nV rounded up to 8 (e.g. 3236 columns of a
 *    642-vertex type); larger requests fail with NPFEM_EINVAL and a message
 *    naming the limit (use npfem_apply_pinv for them).
 *  - The first call on a device resolves the array's device address
 *    (cudaGetSymbolAddress) and caches it; make that first call before any
 *    stream capture.
 *  - All calls in the process share the one array, which keeps the last
 *    call's contents (the call clears what must start at zero).  Calls whose
 *    device work overlaps (other streams, other contexts, other threads on
 *    the same device) race on it: serialise them.
 * Errors: EINVAL, ECUDA. */
#define NPFEM_NOALLOC_MAX_ELEMS (1 << 21)
int npfem_apply_pinv_noalloc(npfem_ctx *ctx, int type_id, const double *q, double *z, int n_cols);

/* Lattice of a fluid velocity field for npfem_ibm_forces: nx x ny x nz nodes at
 * (x0 + i dx, y0 + j dx, z0 + k dx); fields are component-major [3][nz][ny][nx]
 * doubles (x fastest). */
typedef struct {
    int nx, ny, nz;
    double dx, x0, y0, z0;
} npfem_lattice;

/* Immersed-boundary forces on every vertex of every cell by multi-direct
 * forcing (supplementary IBM section, after Wang et al. and Ota et al.), the
 * producer of F_ext in the coupled method.  The Lagrangian points are the
 * vertices at the current state: positions X and velocities U (those of the last
 * step), areas A = a third of the incident triangles' areas.  With Peskin's
 * four-point function phi4 (support 4 dx per axis):
 *   u(X) = sum_x u(x) phi4 phi4 phi4,   spread F(x) = sum_k f_k phi4 phi4 phi4 / dx^2
 *   f_0 = (U - u*(X)) A / dt;  per cycle: F = spread(f), f += (U - (u* + F dt)(X)) A / dt
 *   F_imm = spread(f_cycles)
 * (a point stands for the shell volume A dx; lattice nodes outside the lattice
 * are left out of every sum).
 *   u_fluid : device, 3 nx ny nz doubles, the fluid velocity u*
 *   dt      : > 0;  cycles >= 0
 *   f_lagr  : device, npfem_num_dofs doubles (public layout), receives f_cycles
 *   f_grid  : device, 3 nx ny nz doubles, receives F_imm (also the call's scratch)
 * Enqueued on the context's stream (FP64; the spreading uses atomic additions,
 * so F's last bits depend on their order); device errors surface at the next
 * synchronising call.  The call keeps each point's stencil (about 108 bytes per
 * vertex) in context memory for reuse by later calls.
 * Errors: EINVAL (null pointer, empty lattice, dx or dt not > 0, cycles < 0),
 * ESTATE (no cells), ENOMEM, ECUDA. */
int npfem_ibm_forces(npfem_ctx *ctx, const npfem_lattice *lat, const double *u_fluid, double dt, int cycles,
                     double *f_lagr, double *f_grid);

/* Self-check of device failure detection: enqueues one kernel that waits, through
 * the same bounded mbarrier wait as the tensor-core kernels, on a barrier that
 * nothing arrives on (no copy is in flight) for limit_ms milliseconds (1..2000),
 * then records an expired wait in the context's error word.  The next
 * synchronising call (npfem_sync, get_*, stats) returns NPFEM_ETIMEOUT and clears
 * the word; the context stays usable.  Errors: EINVAL, ECUDA. */
int npfem_check_wait(npfem_ctx *ctx, int limit_ms);

/* Per-kernel timing: when enabled, every kernel launch of a step is
 * bracketed by CUDA events on the context stream (recorded into the step's
 * graph) and npfem_step waits for the step to finish to accumulate the
 * elapsed times per kernel class.  Enabling or disabling rebuilds the graph.
 * Errors: ECUDA. */
int npfem_profile(npfem_ctx *ctx, int enable);

/* Copy the accumulated per-class times and launch counts; reset != 0 zeroes
 * them afterwards. */
int npfem_profile_read(npfem_ctx *ctx, npfem_kernel_times *out, int reset);

/* Message of the last failure of this context (never NULL); with ctx = NULL,
 * the message of this thread's last failed npfem_create. */
const char *npfem_last_error(const npfem_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NPFEM_H */
