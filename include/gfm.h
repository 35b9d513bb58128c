/*
 * gfm.h -- C ABI of libgfm: the Ghost Fluid Method dynamic-pressure equation
 * (assembly + iterative solve + adjoint) on one GB300 GPU.
 *
 * The method is that of Sec. 3.1 of Vukcevic, Roenby, Gatin & Jasak, "A sharp
 * free surface finite volume method applied to gravity wave flows": the
 * continuity equation (Eq. 1) turned into a pressure equation for the dynamic
 * pressure p_d = p - rho g.x (Eq. 3), discretised on a face-addressed
 * finite-volume mesh (Sec. 3, owner P / neighbour N, area vector S_f, centre
 * distance d_f) with the ghost-fluid interface treatment of Eqs. 12-20 and the
 * jump conditions Eqs. 7-8.
 *
 * General rules for every call:
 *  - Array arguments are DEVICE pointers (memory of the current CUDA device,
 *    e.g. allocated by PyTorch) unless the comment says host.  They stay owned
 *    by the caller.  The library owns only the opaque handle and its workspace.
 *  - Arrays are structure-of-arrays FP64 unless noted: a 3-vector field over
 *    m items is laid out [3][m] (all x, then all y, then all z).
 *  - Cell arrays are indexed by the caller's cell numbering, face arrays by
 *    the caller's internal-face numbering.  Any internal renumbering is
 *    invisible to the caller.
 *  - Work is stream-ordered on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  A call returns once the work is enqueued, except where noted.
 *  - Every call returns a gfm_status; no C++ exception or process exit ever
 *    crosses this boundary.  gfm_last_error(h) describes the last failure.
 *  - Inputs are never modified.  Outputs may not alias inputs unless noted.
 *  - A handle is not thread-safe: one host thread and one stream at a time.
 */
#ifndef GFM_H
#define GFM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GFM_OK = 0,
    GFM_ERR_ARG = 1,           /* invalid argument (host-checked)                          */
    GFM_ERR_CUDA = 2,          /* a CUDA runtime call failed                               */
    GFM_ERR_NOMEM = 3,         /* device or host allocation failed                         */
    GFM_ERR_NOT_CONVERGED = 4, /* max_iters / max_refine reached; p holds the last iterate */
    GFM_ERR_BREAKDOWN = 5,     /* CG breakdown (p^T A p <= 0 or not finite)                */
    GFM_ERR_TIMEOUT = 6,       /* a grid-barrier wait exceeded its time budget             */
    GFM_ERR_INCOMPATIBLE = 7,  /* unpinned system with an incompatible right-hand side     */
    GFM_ERR_STATE = 8          /* call out of order (e.g. solve before assemble)           */
} gfm_status;

typedef struct gfm_ctx *gfm_handle;
typedef void *gfm_stream; /* cudaStream_t */

/*
 * Face-addressed mesh (Sec. 3, Fig. "polyhedral control volume").
 *  n_cells, n_faces : number of cells and of INTERNAL faces (> 0).  Boundary
 *                     faces are walls: zero flux, zero-gradient p_d, and are
 *                     not listed.
 *  owner, neighbour : int32 [n_faces], 0 <= owner[f] < neighbour[f] < n_cells.
 *  Sf               : [3][n_faces] face area vectors pointing owner -> neighbour.
 *  C                : [3][n_cells] cell centres (absolute coordinates: the
 *                     jump source uses g.x_Gamma with x absolute, Eq. 7).
 *  V                : [n_cells] cell volumes, or NULL (not used by the solve).
 * The arrays are read during gfm_create only (the handle keeps its own copy).
 */
typedef struct {
    int32_t n_cells;
    int32_t n_faces;
    const int32_t *owner;
    const int32_t *neighbour;
    const double *Sf;
    const double *C;
    const double *V;
} gfm_mesh;

/*
 * Physics of one problem (host struct).
 *  rho_w, rho_a : heavy (water, "+") and light (air, "-") densities, Eq. 4;
 *                 0 < rho_a <= rho_w.
 *  g            : gravitational acceleration vector (Eq. 3).
 *  ref_cell     : cell whose p_d is pinned to ref_value (caller numbering),
 *                 or -1 for no pin (then the right-hand side must be
 *                 compatible, sum(b) ~ 0, else GFM_ERR_INCOMPATIBLE at solve).
 *                 The pin doubles that cell's diagonal and adds
 *                 diag * ref_value to its source, so A stays symmetric
 *                 positive definite; a compatible system's solution does not
 *                 depend on the pin's size.
 */
typedef struct {
    double rho_w;
    double rho_a;
    double g[3];
    int32_t ref_cell;
    double ref_value;
} gfm_phys;

typedef enum {
    GFM_FP64 = 0,  /* Jacobi-PCG entirely in FP64                                       */
    GFM_MIXED = 1  /* FP32 inner Jacobi-PCG (FP64-accurate dot sums) inside FP64
                      iterative refinement: true residual, correction and the jump
                      source stay FP64                                                  */
} gfm_mode;

/*
 * Solver options (host struct; gfm_default_opts fills sensible values).
 *  rtol       : stop when ||b - A p||_2 <= rtol ||b||_2, the TRUE FP64 residual.
 *  inner_rtol : MIXED only: relative residual reduction of each FP32 inner solve.
 *  max_iters  : cap on CG iterations (inner iterations summed, MIXED).
 *  max_refine : MIXED: cap on refinement steps; FP64: cap on restarts from the
 *               true residual.
 *  use_x0     : 1 = start from the p passed in, 0 = start from zero.
 *  info_on_device : 1 = `info` is a DEVICE pointer written by the solve, and
 *               the call returns without synchronising (graph-capturable);
 *               0 = `info` is a host pointer (or NULL) and the call
 *               synchronises `stream` to fill it and to return the status.
 *  timeout_ms : budget of ONE grid-barrier wait inside the persistent kernel;
 *               on expiry the kernel records GFM_ERR_TIMEOUT and all CTAs
 *               return (the device stays usable).
 */
typedef struct {
    int32_t mode;
    double rtol;
    double inner_rtol;
    int32_t max_iters;
    int32_t max_refine;
    int32_t use_x0;
    int32_t info_on_device;
    double timeout_ms;
} gfm_solve_opts;

/* Result of a solve.  iters = CG iterations (summed over refinements),
 * refinements = outer steps (MIXED) or true-residual checks (FP64),
 * status = a gfm_status, rel_res_l2 = final ||b - A p||_2 / ||b||_2 (FP64),
 * rel_res_l1 = OpenFOAM-style normalised L1 residual of the same p. */
typedef struct {
    int32_t iters;
    int32_t refinements;
    int32_t status;
    int32_t reserved;
    double rel_res_l2;
    double rel_res_l1;
} gfm_solve_info;

/* Launch shape of the persistent solver kernels (autotuned or set). */
typedef struct {
    int32_t threads;     /* threads per CTA (multiple of 32, <= 512)        */
    int32_t ctas_per_sm; /* co-resident CTAs per SM (grid = SMs x this)     */
    int32_t form;        /* GFM_MIXED iteration form: 1 = two passes and two
                          * grid all-reduces per FP32 iteration (default);
                          * 2 = one fused pass and one all-reduce (single
                          * meshes only); see gfm_set_tuning              */
} gfm_tuning;

/* Timings of the last call, recorded with CUDA events on the launching
 * stream when profiling is on (gfm_set_profiling); launch counts always. */
typedef struct {
    float ms_assemble;   /* face + cell assembly kernels             */
    float ms_solve;      /* the persistent solver kernel alone       */
    float ms_total;      /* everything enqueued by the last call     */
    int32_t launches;    /* kernels launched by the last call        */
    int32_t grid;        /* CTAs of the persistent kernel            */
    int32_t threads;     /* threads per CTA of the persistent kernel */
    int32_t launches_total; /* kernels launched since gfm_create         */
} gfm_profile;

/* Fill `opts` with defaults: FP64, rtol 1e-10, inner_rtol 1e-4, max_iters 1e6,
 * max_refine 30, use_x0 0, info_on_device 0, timeout_ms 2000. */
gfm_status gfm_default_opts(gfm_solve_opts *opts);

/*
 * Build a handle for one mesh.  Validates indices on the host (the index
 * arrays are copied to the host once), renumbers cells for locality
 * (renumber: 0 = keep the caller's order, 1 = reverse Cuthill-McKee,
 * 2 = Morton order of the cell centres) and builds the sliced-ELL
 * cell-to-face tables.  Synchronises `stream`.  Errors: GFM_ERR_ARG (bad
 * sizes, owner >= neighbour, index out of range, NULL arrays),
 * GFM_ERR_NOMEM, GFM_ERR_CUDA.
 */
gfm_status gfm_create(const gfm_mesh *mesh, int32_t renumber, gfm_stream stream, gfm_handle *out);

/*
 * Batched handle: n_tanks (<= 128) independent meshes ("tanks", e.g. many
 * wave tanks of uneven size) solved together by ONE persistent launch.  All
 * later cell and face arrays are the tanks' arrays concatenated in tank
 * order; gfm_assemble's `phys` is then a host array of n_tanks entries, each
 * ref_cell numbered within its tank and >= 0.  gfm_solve runs GFM_MIXED only:
 * every tank keeps its own CG scalars, residual replacements and stopping
 * test, and `info` points to n_tanks records (the returned status is the
 * last failing tank's).  The launch needs at least one CTA per tank.  When
 * tanks finish, their CTAs are handed to the tanks still iterating.  A tank
 * that asks for an FP64 residual replacement keeps iterating in FP32 until
 * the next replacement round (at most 32 iterations later), so its iteration
 * count can run a little above a single-mesh solve's.  Results are
 * bit-reproducible from run to run.  The adjoint and the host-buffer entry
 * point take single-mesh handles.  Each tank gets its own coarse space (up
 * to its 2 largest one-phase regions, see gfm_set_coarse).  Errors as
 * gfm_create.
 */
gfm_status gfm_create_batched(const gfm_mesh *meshes, int32_t n_tanks, int32_t renumber, gfm_stream stream,
                              gfm_handle *out);

/* Release the handle and its device workspace (synchronises the device). */
gfm_status gfm_destroy(gfm_handle h);

/*
 * Assemble the GFM pressure equation A p = b (Sec. 3.1) for volume fraction
 * alpha [n] (Eq. 10) and predicted face flux phi [F] (the Rhie-Chow flux of
 * the momentum predictor, oriented owner -> neighbour):
 *   wet cell: alpha >= 0.5; interface face: wet owner != wet neighbour;
 *   lambda_W = (alpha_W - 0.5)/(alpha_W - alpha_D) from the wet cell (Eq. 13);
 *   gamma_f = c_f / (lambda_W rho_w + (1 - lambda_W) rho_a), c_f = S.S/S.d
 *     (Eqs. 16-18, 20 collapsed; lambda := 1 or 0 off the interface);
 *   H_f = (rho_w - rho_a) g.(x_W + lambda_W (x_D - x_W))   (Eqs. 7, 12);
 *   J_f = +H_f if the owner is wet, -H_f if dry, 0 elsewhere;
 *   A_ii = sum gamma_f, A_{o,nb} = -gamma_f; b_i = -sum s_if (phi_f + gamma_f J_f).
 * Face quantities and the per-cell sums (ascending face order) are computed
 * in FP64 with every operation rounded as written (bit-reproducible).
 * Errors: GFM_ERR_ARG (NULL, rho_a <= 0, rho_w < rho_a, ref_cell out of range).
 */
gfm_status gfm_assemble(gfm_handle h, const double *alpha, const double *phi, const gfm_phys *phys,
                        gfm_stream stream);

/*
 * Copy the assembled system out (for tests and diagnostics).  Any pointer may
 * be NULL.  lambda, gamma, jump: [F] face order; diag, b: [n] cell order, with
 * the pin applied.  Errors: GFM_ERR_STATE before gfm_assemble.
 */
gfm_status gfm_export_system(gfm_handle h, double *lambda, double *gamma, double *jump, double *diag, double *b,
                             gfm_stream stream);

/*
 * Solve A p = b.  p [n]: in = x0 when opts->use_x0, out = p_d.  phi_corr [F]
 * (nullable): corrected face flux phi_f - gamma_f (p_nb - p_own - J_f), zero in
 * still water (balanced force, Sec. 3.1).  info: see info_on_device.
 * Returns GFM_OK, GFM_ERR_NOT_CONVERGED, GFM_ERR_BREAKDOWN, GFM_ERR_TIMEOUT,
 * GFM_ERR_INCOMPATIBLE (when synchronising), GFM_ERR_STATE before assemble,
 * GFM_ERR_ARG.  With info_on_device = 1 the solve status is only in info.
 */
gfm_status gfm_solve(gfm_handle h, const gfm_solve_opts *opts, double *p, double *phi_corr, gfm_solve_info *info,
                     gfm_stream stream);

/*
 * Reverse mode of p = A(alpha)^{-1} b(alpha, phi): given p (the solution of
 * the last assembled system) and dL/dp [n], solve the adjoint system A mu =
 * dL/dp (A is symmetric) and return
 *   dL_dphi [F]   = -(mu_own - mu_nb),
 *   dL_dalpha [n] = sum over interface faces of dL/dlambda_f * dlambda_f/dalpha,
 * through gamma_f(lambda_f) and J_f(lambda_f) (Eqs. 13, 18, 7, 12); wet/dry
 * flags and the pin's size are held fixed.  mu [n] nullable.  Same options
 * and errors as gfm_solve.
 */
gfm_status gfm_solve_adjoint(gfm_handle h, const gfm_solve_opts *opts, const double *p, const double *dL_dp,
                             double *dL_dphi, double *dL_dalpha, double *mu, gfm_solve_info *info, gfm_stream stream);

/*
 * End-to-end call on HOST buffers: copies alpha [n] and phi [F] to the
 * device, assembles, solves and copies p [n] back, all on `stream`, and
 * synchronises.  Host buffers should be page-locked for the copies to run
 * asynchronously.  p_host is x0 when opts->use_x0.  info is a host pointer.
 */
gfm_status gfm_solve_host(gfm_handle h, const double *alpha_host, const double *phi_host, const gfm_phys *phys,
                          const gfm_solve_opts *opts, double *p_host, gfm_solve_info *info, gfm_stream stream);

/*
 * Dynamic-pressure gradient of the momentum equation and cell velocities
 * (Sec. 3.1: Eq. 20 and the paragraph after it, which carries the ghost
 * values into the pressure gradient of Eq. 2; Eq. 8).  After gfm_assemble,
 * for a p_d [n] (e.g. gfm_solve's), caller order throughout:
 *   grad [3][n] (nullable): (1/rho grad p_d)_P by the Gauss theorem, linear
 *        cell-to-face interpolation, the neighbour's value replaced at an
 *        interface face by its ghost value in P's fluid (Eq. 20 from the wet
 *        side, the analogous extrapolation from the dry side); zero-gradient
 *        walls.  The ghost values collapse onto the assembled coefficients:
 *          grad_P = 1/V_P sum_f (1 - w_P) (p_N - p_P - s_Pf J_f)/rho_f s_Pf S_f,
 *        rho_f = lambda_f rho_w + (1 - lambda_f) rho_a, s_Pf = +1 (P owns f) or -1,
 *        1 - w_P = S_f.(x_f - x_P)/S_f.(x_N - x_P).  Zero in still water.
 *   U [3][n] (nullable; needs phi [F]): cell velocity from the face flux phi
 *        (e.g. gfm_solve's corrected flux), U_P = 1/V_P sum_f s_Pf phi_f (x_f - x_P),
 *        exact for a uniform velocity.
 *   V  [n]     cell volumes (required).
 *   xf [3][F]  face centres, or NULL for the midpoints of the two cell centres
 *              (exact on uniform hex meshes).
 * Works on batched handles (densities per tank).  One kernel launch, FP64.
 * Errors: GFM_ERR_ARG (NULL p or V, both outputs NULL, U without phi),
 * GFM_ERR_STATE (grad before gfm_assemble), GFM_ERR_CUDA.
 */
gfm_status gfm_gradient(gfm_handle h, const double *p, const double *V, const double *xf, double *grad,
                        const double *phi, double *U, gfm_stream stream);

/*
 * Real pressure-equation inputs (Sec. 3: the pressure equation comes from
 * continuity with the Rhie-Chow flux, and its Laplacian is discretised by
 * the Gauss theorem with an explicit over-relaxed non-orthogonal correction).
 *
 * gfm_set_rau: rau [F] (DEVICE, copied; NULL = 1 everywhere) is the face
 * value of 1/a_P, the inverse diagonal of the momentum equation.  From the
 * next gfm_assemble on, gamma_f = (c_f / rho_f) * rau_f: the equation is
 * div(rau beta grad p_d) = div(phi*), with the jump source scaled alike.
 * Errors: GFM_ERR_NOMEM, GFM_ERR_CUDA.
 *
 * gfm_nonorth_correct: after gfm_assemble, splits each area vector into
 * Delta_f = (S.S)/(S.d) d (the implicit two-point part already assembled)
 * and k_f = S_f - Delta_f, and adds the explicit part
 *   corr_f = rau_f k_f . (w_o G_own + (1 - w_o) G_nb),  G = (1/rho) grad p_d
 * of the given p [n] (gfm_gradient's ghost-value gradient; continuous across
 * the interface by Eq. 8) to the source: the next gfm_solve solves with
 * phi* - corr, and its corrected flux is phi* - corr - gamma (p_nb - p_own - J).
 * Calling it again replaces the correction (deferred correction: solve,
 * correct from the new p_d, solve again with use_x0).  The next gfm_assemble
 * clears it.  V [n] volumes (required), xf [3][F] face centres or NULL
 * (midpoints), corr [F] (nullable) receives the correction flux.  Zero on
 * orthogonal meshes.  The adjoint treats the correction as a fixed source.
 * Errors: GFM_ERR_ARG (NULL p or V), GFM_ERR_STATE (before gfm_assemble),
 * GFM_ERR_NOMEM, GFM_ERR_CUDA.
 */
gfm_status gfm_set_rau(gfm_handle h, const double *rau, gfm_stream stream);
gfm_status gfm_nonorth_correct(gfm_handle h, const double *p, const double *V, const double *xf, double *corr,
                               gfm_stream stream);

/*
 * Solve without device allocation.  The paper has no counterpart: this is an
 * entry point for callers that cannot call cudaMalloc -- code running inside
 * a host program that owns the GPU's memory (a CFD code or plugin drawing
 * from the host's pool or held under a memory cap, where a cudaMalloc would
 * be refused or fragment the pool) and loops that must not call
 * cudaMalloc/cudaFree because those can synchronise the device.  It needs no
 * handle (gfm_create allocates) and allocates nothing, on the device or
 * through any library.
 *
 * Solves A x = b by FP64 Jacobi-preconditioned CG for a symmetric positive
 * definite A in CSR form, all DEVICE pointers owned by the caller:
 *   row_ptr [n+1], col [nnz], val [nnz] (int32, int32, FP64); every row
 *   holds a positive diagonal entry.  nnz is the length of col and val.
 *   The kernel checks the structure before it gathers through it:
 *   0 <= row_ptr[i] <= row_ptr[i+1] <= nnz and 0 <= col[e] < n, else the
 *   record's status is GFM_ERR_ARG and nothing else is read or written
 *   beyond x's start vector.  The GFM system of gfm_assemble is
 *   A_ii = diag_i, A_{own,nb} = A_{nb,own} = -gamma_f (gfm_export_system).
 *   b [n] the right-hand side, x [n] the solution (in: the start vector when
 *   use_x0 = 1).  x may not alias the other arrays.
 * Stops when the TRUE residual ||b - A x||_2 <= rtol ||b||_2, after
 * max_iters CG iterations, or after 30 restarts from the true residual.
 * timeout_ms bounds each grid-barrier wait as in gfm_solve_opts.  info
 * (nullable) is a DEVICE pointer to one record, written by the kernel
 * (status GFM_OK, GFM_ERR_NOT_CONVERGED, GFM_ERR_BREAKDOWN, GFM_ERR_TIMEOUT,
 * or GFM_ERR_ARG for a bad CSR structure or a row without a positive
 * diagonal).  The call only enqueues work on `stream` and never
 * synchronises.
 *
 * Scratch: the CG vectors, the per-CTA partial sums and the barrier counter
 * live in one fixed array in the library's device code, 8.05 MiB for
 * n <= GFM_NOALLOC_MAX_CELLS; every GPU that loads the library's device code
 * holds it until the process exits.  n beyond that limit returns
 * GFM_ERR_ARG before anything is enqueued.  The first call on a device looks
 * up the array's address and the co-resident grid size for that device
 * (cudaGetSymbolAddress, with the caller's current device); make that first
 * call before any stream capture.  All calls on a device share the array:
 * the barrier block is cleared on `stream` at every call, and the rest is
 * written before it is read, but two calls whose work overlaps on the GPU
 * (different streams or host threads) race on it and corrupt each other.
 * Returns GFM_OK once enqueued, GFM_ERR_ARG (n out of range, nnz < n, NULL
 * array, rtol <= 0, max_iters < 0, timeout_ms <= 0), GFM_ERR_CUDA.
 */
#define GFM_NOALLOC_MAX_CELLS 262144
gfm_status gfm_solve_csr_noalloc(int32_t n, int32_t nnz, const int32_t *row_ptr, const int32_t *col,
                                 const double *val, const double *b, double *x, double rtol, int32_t max_iters,
                                 int32_t use_x0, double timeout_ms, gfm_solve_info *info, gfm_stream stream);

/*
 * Split the tanks of a batch across n_ranks GPUs (one process each).  The
 * tanks are independent problems (each its own pressure equation of
 * Sec. 3.1 with its own pin), so the split needs no data exchange: each
 * rank builds a batched handle of its tanks and only per-tank records are
 * gathered afterwards.  Balances cells per rank by longest-processing-time
 * list scheduling (descending cells, ties by tank index; each tank to the
 * least-loaded rank, ties to the lower rank), so every rank computes the
 * same table from the same counts.  The busiest rank holds at most
 * total/n_ranks + (1 - 1/n_ranks) * largest cells.
 *  cells        : host int64 [n_tanks], cells of each tank (>= 1).
 *  rank_of_tank : host int32 [n_tanks], out: the rank of each tank.
 *  rank_cells   : host int64 [n_ranks] or NULL, out: cells per rank.
 * Host only; needs no GPU.  Errors: GFM_ERR_ARG (NULL, n_tanks or n_ranks
 * < 1, a tank with no cells).
 */
gfm_status gfm_partition_tanks(const int64_t *cells, int32_t n_tanks, int32_t n_ranks, int32_t *rank_of_tank,
                               int64_t *rank_cells);

/*
 * The pressure part of one time step of the segregated solver (Sec. 3,
 * flow chart: SIMPLE outer iterations around PISO correctors; Sec. 4.1.1
 * uses 6 outer iterations with 2 pressure correctors each), enqueued as one
 * stream-ordered sequence that a CUDA graph can capture and replay:
 *   for k = 0 .. n_solves-1:
 *     gfm_assemble(alpha, phi_star + k F)    the corrector's predicted flux
 *     gfm_solve into p, warm-started from the previous corrector's p_d
 *       (k = 0: from p when opts->use_x0), info + k (DEVICE records)
 *     n_nonorth times: gfm_nonorth_correct from the new p_d, solve again
 *   then, for the last corrector: phi_corr [F] (nullable) = corrected flux,
 *   grad [3][n] (nullable) = (1/rho) grad p_d, U [3][n] (nullable, needs
 *   phi_corr) = cell velocity from phi_corr (gfm_gradient).
 * alpha [n] is the step's volume fraction (one advection per time step),
 * phi_star [n_solves][F] the predicted fluxes (the momentum predictor's
 * Rhie-Chow fluxes, produced outside this library), phys as gfm_assemble.
 * opts->info_on_device must be 1: the call never synchronises; info holds
 * n_solves records (n_solves x n_tanks on a batched handle).  V [n] and xf
 * [3][F] (nullable) as gfm_gradient; V is required for n_nonorth > 0, grad
 * or U.  Errors: those of the calls it makes, GFM_ERR_ARG.
 */
gfm_status gfm_piso_step(gfm_handle h, const gfm_solve_opts *opts, int32_t n_solves, int32_t n_nonorth,
                         const double *alpha, const double *phi_star, const gfm_phys *phys, double *p, double *phi_corr,
                         const double *V, const double *xf, double *grad, double *U, gfm_solve_info *info,
                         gfm_stream stream);

/*
 * isoAdvector advection step (Sec. 3.2) on the handle's mesh: the volume of
 * heavy fluid each face passes during [t, t + dt] and the volume-fraction
 * update,
 *   dV_f = phi_f int_0^dt alpha_f+(tau) dtau                     (Eq. dV)
 *   alpha_P(t + dt) = alpha_P(t) - 1/V_P sum_f s_Pf dV_f,
 * alpha_f+ being the submerged fraction of the face (Eq. alphaf).  In the
 * upwind cell U of face f (owner when phi_f >= 0) the interface is the
 * isoface plane through xS [3][n] (column U) with unit normal nS [3][n]
 * pointing away from the heavy fluid, moving at normal speed UnS [n]
 * (= U_S.n_S); it reaches a point x at t + (x - x_S).n_S / UnS (Eq. tv).
 * The face surface is the union of the triangles (xf, v_k, v_k+1) over its
 * polygon, fv_xyz [3][nvt] columns fv_ptr[f] .. fv_ptr[f+1]-1 (in order
 * round the face; fv_ptr int32 [F+1]).  Each triangle is swept in the
 * paper's way: vertex times in order, the cut point x4 (Eq. x_41), the two
 * quadratic pieces of the swept fraction (Eqs. aplus1, aplus2) and their
 * exact time integrals (Eq. intaplus).  UnS < 0 (interface moving into the
 * heavy fluid): the submerged fraction is the complement of the swept one;
 * UnS = 0: a static plane.  A face whose upwind cell has has_iso [n]
 * (int8) = 0 carries alpha_U throughout.  The isofaces (the reconstruction
 * step) are inputs.  Outputs: dV [F]; integral [F] (nullable) the time
 * integrals; alpha_new [n] (nullable; needs V [n]).  Face arrays in the
 * caller's face order, cell arrays in the caller's cell order.  FP64, one
 * thread per face, then one per cell summing its faces in ascending order.
 * Errors: GFM_ERR_ARG (NULL, dt < 0, nvt < 3), GFM_ERR_CUDA.
 */
gfm_status gfm_iso_advect(gfm_handle h, const double *alpha, const double *phi, double dt, const int32_t *fv_ptr,
                          const double *fv_xyz, int32_t nvt, const double *xf, const int8_t *has_iso,
                          const double *xS, const double *nS, const double *UnS, const double *V, double *integral,
                          double *dV, double *alpha_new, gfm_stream stream);

/*
 * Operator-table format of the streamed mixed-precision pass.  When a
 * CTA's slice tables do not fit in shared memory, the operator pass streams
 * them every iteration; the full form is 8 bytes per slot (neighbour index,
 * FP32 coefficient).  The compact form is 4 bytes: the neighbour as a signed
 * 16-bit offset from the slot's own cell and a 16-bit code of the
 * coefficient -- off the interface, one of the two values (c_f/rho_w,
 * c_f/rho_a) of the face's class of bit-identical c_f = S.S/S.d, looked up
 * in a dictionary staged in shared memory; at an interface face an escape
 * code sends the pass to the FP32 coefficient in global memory.  Both forms
 * give bit-identical results.  The compact form is usable when every
 * neighbour offset fits 16 bits (after renumbering) and the faces fall into
 * at most 2047 classes; it is not used while a face Rhie-Chow coefficient
 * is set (gfm_set_rau), which makes every coefficient distinct.
 * gfm_set_table: compact = 1 uses it when usable, 0 (default) never;
 * force_stream = 1 streams the tables even when they would fit in shared
 * memory (for tests and tuning; default 0).  Takes effect at the next solve.
 * The compact form halves the streamed bytes, but the operator pass of the
 * meshes measured here is bound by gather latency rather than by its share
 * of HBM bandwidth, and interface slots add a dependent load: it was slower
 * on the 3D box and the 64-tank batch, hence off by default.
 * gfm_get_table (host pointers, any may be NULL): whether the compact form
 * is usable for this mesh, its number of classes, and whether the last
 * assembly wrote it.
 */
gfm_status gfm_set_table(gfm_handle h, int32_t compact, int32_t force_stream);
gfm_status gfm_get_table(gfm_handle h, int32_t *compact_usable, int32_t *n_classes, int32_t *compact_valid);

/* Launch shape of the persistent kernels (threads a multiple of 32, at most
 * 512) and the form of the mixed-precision iteration.  A zero field keeps
 * the current value.  Both forms run the same preconditioned CG recurrences
 * of the pinned system of Sec. 3.1 (the paper names no solver) with the same
 * FP64 residual replacement and stopping rules.  Form 1 applies each FP32
 * iteration as an operator pass (p = u + beta p, s = A p, p.s) and an update
 * pass (x, r, u; r.u, r.r), each closed by a grid all-reduce.  Form 2 keeps
 * per cell (q = D^{-1} r, t = D^{-1} s, p) and folds the update into the
 * next operator pass, every neighbour's new direction recomputed from its
 * gathered state; r.u of the next step follows from q.D q, t.D q and t.D t
 * (summed with p.s in the same all-reduce), so an iteration closes with ONE
 * all-reduce.  Form 2 suits meshes whose iteration is bound by all-reduce
 * latency; the results agree within the solver tolerance, not bit for bit.
 * Errors: GFM_ERR_ARG if the shape is out of range or cannot be co-resident,
 * or form 2 is asked of a batched handle. */
gfm_status gfm_set_tuning(gfm_handle h, const gfm_tuning *t);
gfm_status gfm_get_tuning(gfm_handle h, gfm_tuning *t);

/*
 * Autotuner: on the assembled system, time `trials` solves (median, CUDA
 * events on `stream`) with opts for each launch shape of the persistent
 * kernel ({512,1}, {256,2}, {128,4}, {384,1}, {256,1} threads x CTAs per
 * SM, where co-resident), and for a single mesh in GFM_MIXED mode with both
 * iteration forms (gfm_set_tuning).  For a batched handle it also tries the tank->CTA
 * table weighted by the iterations each tank took (tanks that iterate longer
 * get more CTAs).  The fastest shape and table are kept for later solves and
 * returned in *chosen and *best_ms (either may be NULL).  The paper has no
 * counterpart; tuning changes how the work is split, not what is computed.
 * The trial solutions go to the handle's own workspace; synchronises
 * `stream`.  Errors: GFM_ERR_STATE before gfm_assemble, GFM_ERR_ARG (bad
 * opts, trials outside [1, 64]), GFM_ERR_NOT_CONVERGED when no shape solved
 * the system (the previous shape is kept), GFM_ERR_CUDA.
 */
gfm_status gfm_autotune(gfm_handle h, const gfm_solve_opts *opts, int32_t trials, gfm_tuning *chosen, float *best_ms,
                        gfm_stream stream);

/*
 * Two-level preconditioner.  With a density ratio of 1000 the ghost-fluid
 * Laplacian (Sec. 3.1) couples each connected region of one phase to the rest
 * only through its interface faces, and Jacobi-PCG stalls for thousands of
 * iterations on the near-constant modes of the large regions.  Every
 * assembly finds the connected regions of each phase (cells joined by
 * non-interface faces) and keeps the up-to-max_vectors largest with at least
 * min_size cells as coarse space Z; the preconditioner is then
 * D^{-1} + Z (Z^T A Z)^{-1} Z^T.  max_vectors = 0 gives plain Jacobi.
 * Defaults: 8 vectors, 64 cells.  Takes effect at the next gfm_assemble.
 * The coarse space needs a pin (ref_cell >= 0); unpinned systems use Jacobi.
 * On a batched handle each tank keeps up to min(max_vectors, 2) regions of
 * its own (default 2).  gfm_get_coarse reports (host pointers, synchronises
 * `stream`) the vectors in use (summed over the tanks of a batch), the
 * regions of at least min_size cells, and the sizes [8] of the first kept ones.
 */
gfm_status gfm_set_coarse(gfm_handle h, int32_t max_vectors, int32_t min_size);
gfm_status gfm_get_coarse(gfm_handle h, int32_t *n_vectors, int32_t *n_regions, int32_t *sizes, gfm_stream stream);

/* Profiling: on = 1 records CUDA events around every kernel of each call. */
gfm_status gfm_set_profiling(gfm_handle h, int32_t on);
gfm_status gfm_get_profile(gfm_handle h, gfm_profile *out);

/* Sizes: cells, internal faces, tanks, and the internal cell order
 * (perm[i] = internal index of caller cell i), perm may be NULL (host). */
gfm_status gfm_get_sizes(gfm_handle h, int32_t *n_cells, int32_t *n_faces, int32_t *n_tanks);
gfm_status gfm_get_permutation(gfm_handle h, int32_t *perm_host);

const char *gfm_status_string(gfm_status s);
const char *gfm_last_error(gfm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* GFM_H */
