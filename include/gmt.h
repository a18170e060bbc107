/*
 * gmt.h — C ABI of the B300 periodic-homogenization library (libgmt.so).
 *
 * The library solves the periodic cell problems of a binary voxel cell with a matrix-free
 * geometric-multigrid V-cycle on a sparse active-voxel hierarchy and returns the
 * homogenized tensor. Problem statement: Sec. 3.1 of the paper (eq. generic_cell,
 * linear_system; Example 1 linear elasticity with six unit macro-strain modes, Example 2
 * steady heat conduction with three unit gradients) and App. F (element matrices, C^H and
 * kappa^H energy averages). Hierarchy: Sec. 4.1 (sparse voxels, octant features,
 * conservative coarsening, eq. gmgcoarsenode). Solver: Sec. 3.2 (Alg. 1, Galerkin
 * operators), Sec. 4.6 (element-by-element operator, smoothing, local Galerkin
 * projection), App. E (matrix-free trilinear transfers).
 *
 * Conventions shared by every call
 *   - Voxels: N^3 uint8, index x + N*y + N^2*z (x fastest); nonzero = solid.
 *   - Levels are numbered 0 (finest, the voxel grid) .. L-1 (coarsest); level l has
 *     N_l = N / 2^l voxels per side.
 *   - Node order ("canonical"): active nodes of a level sorted by x + N_l*y + N_l^2*z.
 *   - Field layout: double[node][component][case], i.e. value (n, i, m) at
 *     n*D*M + i*M + m, with D = 3, M = 6 (elasticity; cases in Voigt order
 *     xx, yy, zz, yz, xz, xy, engineering shear) or D = 1, M = 3 (heat; cases x, y, z).
 *   - Sign: fields u solve K u = +f with f = sum_e A_e^T K_e x0, so u = -chi and the total
 *     field on an element is x0 - u_e (App. F.1).
 *   - Pointers documented "device" must be CUDA device (or managed) memory on the
 *     device that was current at gmt_build_hierarchy; "host" pointers are ordinary host
 *     memory. The caller owns every pointer it passes; the library owns the hierarchy,
 *     its operators and all scratch, and frees them in gmt_free_hierarchy.
 *   - Every call returns a gmt_status and never aborts, traps or exits. On an error the
 *     outputs are unspecified and gmt_last_error() describes the failure (thread-local).
 *   - All work is issued on the stream given to gmt_build_hierarchy (or gmt_set_stream);
 *     calls that return host values synchronize that stream.
 *   - A hierarchy is not thread-safe: one host thread at a time per hierarchy.
 */
#ifndef GMT_H
#define GMT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmt_hierarchy gmt_hierarchy;

typedef enum { GMT_ELASTIC = 0, GMT_HEAT = 1 } gmt_physics;

typedef enum {
  GMT_OK = 0,
  GMT_ERR_ARG = 1,          /* invalid argument (null pointer, bad level, bad option) */
  GMT_ERR_RES = 2,          /* resolution not a multiple of 4 / not divisible by 2^(L-1) */
  GMT_ERR_EMPTY = 3,        /* the cell has no solid voxel */
  GMT_ERR_OOM = 4,          /* device allocation failed */
  GMT_ERR_CUDA = 5,         /* a CUDA call failed */
  GMT_NOT_CONVERGED = 6,    /* iteration caps reached; best field written, info filled */
  GMT_DIVERGED = 7,         /* residual grew by > 1e4 or became NaN; best field written */
  GMT_ERR_STATE = 8         /* call needs gmt_prepare / gmt_solve to have run first */
} gmt_status;

/* Precision of a solve's inner V-cycle. GMT_PREC_FP32: FP32 vectors and arithmetic;
   GMT_PREC_BF16: the V-cycle's vectors stored in BF16 on every level (its input rounded
   from the FP32 Krylov residual, its result widened back), arithmetic in FP32; both with
   FP32 Krylov vectors and a float-float solution. GMT_PREC_FP64: everything in FP64. The
   per-step calls (gmt_apply ... gmt_vcycle) take FP64 or FP32. */
typedef enum { GMT_PREC_FP64 = 0, GMT_PREC_FP32 = 1, GMT_PREC_BF16 = 2 } gmt_precision;
typedef enum { GMT_SMOOTH_JACOBI = 0, GMT_SMOOTH_CHEBYSHEV = 1, GMT_SMOOTH_GS8 = 2 } gmt_smoother;
/* Multigrid cycle of Sec. 5's schedules: V (one coarse correction per level), W (two),
   F (one F-cycle then one V-cycle on the next level). */
typedef enum { GMT_CYCLE_V = 0, GMT_CYCLE_W = 1, GMT_CYCLE_F = 2 } gmt_cycle;

/* Solver options. gmt_default_options fills the defaults given in brackets. */
typedef struct {
  int levels;          /* [0] number of levels L; 0 = smallest L with coarsest <= coarsest_max */
  int coarsest_max;    /* [8] automatic level rule: coarsest grid side at most this */
  int smoother;        /* [GMT_SMOOTH_JACOBI] damped block-Jacobi, Chebyshev, or 8-colour
                          Gauss-Seidel (Sec. 4.6 "Parallel Smoothing": nodes coloured by the
                          parity of (x, y, z); one sweep updates the 8 colours in turn, each
                          with the damped block-Jacobi step on the latest values) */
  int nu_pre;          /* [1] pre-smoothing sweeps on level 0 (Chebyshev: polynomial degree) */
  int nu_post;         /* [1] post-smoothing sweeps on level 0 */
  double omega;        /* [0.6] Jacobi damping */
  double cheb_ratio;   /* [30] Chebyshev interval [lmax/cheb_ratio, cheb_upper*lmax] */
  double cheb_upper;   /* [1.1] */
  int precision;       /* [GMT_PREC_FP32] precision of the inner V-cycle / Krylov loop
                          (gmt_precision); GMT_PREC_FP64 = plain all-FP64 solve */
  int krylov;          /* [1] 1: conjugate gradients preconditioned by the V-cycle;
                          0: stationary V-cycle iteration (the paper's GMG loop) */
  double inner_tol;    /* [0.03] mixed precision: the true residual is recomputed (and replaces the
                          iterated one) whenever the iterated residual fell by this factor
                          (0.03 was 5 % faster than 0.1 on the 128^3 batch at the same
                          V-cycle count; 0.3 was 9 % slower) */
  int max_inner;       /* [40] with max_outer: at most max_inner * max(1, max_outer) V-cycles */
  int max_outer;       /* [40] (1600 V-cycles: spinodal cells of wavenumber 9-10 at 128^3
                          need 560-1100, in FP64 as in mixed precision) */
  int cycle;           /* [GMT_CYCLE_V] */
  int fp64_fallback;   /* [1] when the mixed-precision solve diverges, gmt_solve solves the
                          cell again in plain FP64 (gmt_info.fp64_fallback reports it) */
  int nu_coarse;       /* [2] pre- and post-smoothing sweeps on levels >= 1; 0: nu_pre and
                          nu_post on every level. The defaults (1 on the fine level, 2 on
                          the coarse ones) were the fastest of the sweeps measured on the
                          128^3 elasticity batch; heat conduction on the same cells and
                          elasticity at 512^3 ran faster with nu_pre = nu_post = 2 */
  int graphs;          /* [1] gmt_solve replays its V-cycles from CUDA graphs captured on the
                          hierarchy's stream (not on the legacy default stream, not while
                          tracing, not inside a caller's own stream capture, and not while
                          another host thread is inside a call of this library: graph
                          operations concurrent with other threads' kernel launches
                          crashed the driver). Kernels that the caller launches from other
                          threads itself are not covered: such a caller sets 0. */
  int coarse_fp16;     /* [0] mixed precision: the stored per-node stencils of levels >= 1
                          in FP16 (scaled per level, FP32 arithmetic), half the bytes the
                          coarse sweeps read; the V-cycle becomes a slightly different
                          preconditioner (the solve's accuracy is unchanged) */
  int warm_sweeps;     /* [0] with a given initial field u0: this many damped-Jacobi sweeps
                          on level 0 (omega) smooth it before the iteration starts, removing
                          the rough part of a predicted field's error that the V-cycle
                          preconditioned iteration would otherwise carry (0..16) */
} gmt_options;

/* Per-solve report. rel_residual[m] = ||f_m - K u_m|| / ||f_m|| of the returned field,
   computed by the library's outer residual (0 for a case whose load cancels exactly). */
typedef struct {
  int outer;             /* outer refinements performed */
  int inner_total;       /* V-cycles applied in total */
  int cases;             /* number of load cases (6 or 3) */
  double rel_residual[6];
  double t_setup_ms;     /* operator setup for this material (0 if cached) */
  double t_solve_ms;     /* solve time (host wall clock around the device work) */
  int fp64_fallback;     /* 1 if the mixed-precision solve diverged and FP64 took over */
} gmt_info;

void gmt_default_options(gmt_options* opts);

const char* gmt_status_string(gmt_status s);

/* Thread-local description of the last failure in this thread ("" if none). */
const char* gmt_last_error(void);

/* Build the sparse hierarchy (Sec. 4.1): active elements and nodes, octant masks,
   canonical numbering, conservative coarsening, brick tables. Geometry only; operators
   are built by gmt_prepare (or implicitly by gmt_solve).
   voxels: N^3 bytes, host memory if voxels_on_device == 0, else device memory; read only
   during the call. res: N, a positive multiple of 4 with N divisible by 2^(L-1).
   opts: nullable (defaults). stream: a cudaStream_t (nullable = legacy default stream).
   out: receives the new hierarchy (library-owned; release with gmt_free_hierarchy).
   Errors: GMT_ERR_ARG, GMT_ERR_RES, GMT_ERR_EMPTY, GMT_ERR_OOM, GMT_ERR_CUDA. */
gmt_status gmt_build_hierarchy(const uint8_t* voxels, int res, int voxels_on_device,
                               const gmt_options* opts, void* stream, gmt_hierarchy** out);

void gmt_free_hierarchy(gmt_hierarchy* h);

gmt_status gmt_set_stream(gmt_hierarchy* h, void* stream);
gmt_status gmt_set_options(gmt_hierarchy* h, const gmt_options* opts);  /* solver fields only */

int gmt_num_levels(const gmt_hierarchy* h);
int gmt_level_res(const gmt_hierarchy* h, int level);
int64_t gmt_num_nodes(const gmt_hierarchy* h, int level);
int64_t gmt_num_elements(const gmt_hierarchy* h, int level);
int64_t gmt_num_bricks(const gmt_hierarchy* h, int level);   /* 4^3-node bricks (0 = dense) */
int64_t gmt_device_bytes(const gmt_hierarchy* h);            /* library-owned device memory */

/* Canonical node list of a level (Sec. 4.1): xyz_out device int32[n][3] (x, y, z);
   mask_out device uint8[n] octant masks (bit o set when the element whose local vertex o
   is this node is active), nullable. */
gmt_status gmt_node_coords(const gmt_hierarchy* h, int level, int32_t* xyz_out,
                           uint8_t* mask_out);

/* Active elements of a level, sorted by linear index: xyz_out device int32[ne][3];
   child_mask_out device uint8[ne] (levels >= 1: bit c set when child 2X + c is active;
   level 0: 0), nullable. */
gmt_status gmt_element_coords(const gmt_hierarchy* h, int level, int32_t* xyz_out,
                              uint8_t* child_mask_out);

/* Transfer stencil tuples of App. E.2 between level and level+1: for every active node
   of `level` (canonical order) the 8 coarse canonical indices and weights; zero-weight
   slots hold index -1 and weight 0. idx_out device int32[n][8], w_out device double[n][8]. */
gmt_status gmt_transfer_stencil(const gmt_hierarchy* h, int level, int32_t* idx_out,
                                double* w_out);

/* Build the operators for one material (App. F element matrices; Sec. 4.6 element-local
   Galerkin coarse operators; coarsest dense generalized inverse; smoother data).
   physics GMT_ELASTIC uses E > 0 and -1 < nu < 0.5; GMT_HEAT uses k > 0. Cached: a
   repeat call with the same arguments does no work. */
gmt_status gmt_prepare(gmt_hierarchy* h, gmt_physics physics, double E, double nu, double k);

/* y = K_level u on canonical fields of `level` (device double[n][D][M]) for the prepared
   material, computed in `precision` (FP64 or FP32 arithmetic). Level 0 is the
   matrix-free operator of Sec. 4.6; levels >= 1 are the Galerkin operators. */
gmt_status gmt_apply(gmt_hierarchy* h, int level, int precision, const double* u, double* y);

/* `sweeps` smoothing steps of the configured smoother on K_level u = f, in place on u
   (device canonical fields). zero_init != 0 means u is taken as 0 on entry. */
gmt_status gmt_smooth(gmt_hierarchy* h, int level, int precision, const double* f,
                      double* u, int sweeps, int zero_init);

/* f_coarse = P^T r_fine (restriction, App. E.2, gather form) from `level` to level+1. */
gmt_status gmt_restrict(gmt_hierarchy* h, int level, int precision, const double* r_fine,
                        double* f_coarse);

/* u_fine += P u_coarse (prolongation and correction, App. E.2) from level+1 to `level`. */
gmt_status gmt_prolong(gmt_hierarchy* h, int level, int precision, const double* u_coarse,
                       double* u_fine);

/* Coarsest-level solve: u = zero-mean solution of K_{L-1} u = f (device canonical). */
gmt_status gmt_coarse_solve(gmt_hierarchy* h, const double* f, double* u);

/* One V-cycle (Alg. 1) on K_0 u = f at `precision`; u holds the initial guess on entry
   (zero_init != 0: taken as 0) and the result on exit. */
gmt_status gmt_vcycle(gmt_hierarchy* h, int precision, const double* f, double* u,
                      int zero_init);

/* One V-cycle with injected coarse corrections (Alg. 2): as gmt_vcycle, except that on the
   way down the coarse unknown of each level l >= 1 starts from the correction e[l] instead
   of zero and is pre-smoothed from there. e: n_e = gmt_num_levels(h) pointers, e[l] a
   device canonical field of level l ([node][comp][case] doubles, gmt_num_nodes(h, l)
   nodes) or NULL for that level's zero start; e[0] is not read (u is the fine level's
   start), nor is the coarsest level's entry (that level is solved exactly). Read during
   the call. GMT_ERR_ARG for a W- or F-cycle schedule. */
gmt_status gmt_vcycle_inject(gmt_hierarchy* h, int precision, const double* f, double* u,
                             int zero_init, const double* const* e, int n_e);

/* Largest number of hierarchies one gmt_vcycle_batch call takes. */
#define GMT_BATCH_MAX 64

/* One FP32 V-cycle (Alg. 1) on each of n (1..GMT_BATCH_MAX) distinct prepared hierarchies
   at once: hs[i], f[i], u[i] as for gmt_vcycle(hs[i], GMT_PREC_FP32, f[i], u[i], zero_init)
   (device canonical FP64 fields, u[i] the initial guess unless zero_init, the result on
   exit), and every u[i] is bitwise what that call returns. Each phase of the cycle
   (smoothing sweep, residual, restriction, coarsest solve, prolongation) runs as one launch
   over the bricks of all n lattices, so the small coarse levels of many cells fill the GPU
   together and the launch count does not grow with n. The hierarchies must share the
   material (physics and parameters of gmt_prepare), have no element densities, use the
   damped-Jacobi smoother and the V-cycle with the same omega, nu_pre, nu_post, nu_coarse
   and coarse_fp16, and run on the same device and stream; otherwise GMT_ERR_ARG
   (GMT_ERR_STATE if one is not prepared). Sizes and level counts may differ: at each
   level the lattices whose
   coarsest level it is take their coarsest solve in one launch, the others go on down.
   The launches go to that stream and the call returns after it has finished them. */
gmt_status gmt_vcycle_batch(gmt_hierarchy* const* hs, int n, const double* const* f,
                            double* const* u, int zero_init);

/* Largest eigenvalue estimate of D^-1 K at `level` used by the Chebyshev smoother
   (host double out). */
gmt_status gmt_lambda_max(gmt_hierarchy* h, int level, double* out);

/* Solve the cell problems to max_m r_m <= tol (Sec. 5 metric r, Sec. 3.1).
   u0: device canonical initial guess, nullable (zero). u_out: device canonical field,
   nullable (the library keeps its own copy for gmt_homogenize). info: host, nullable.
   Returns GMT_OK, GMT_NOT_CONVERGED or GMT_DIVERGED (field and info still written) or
   an error. Fields are gauge-fixed: zero mean over active nodes per component/case. */
gmt_status gmt_solve(gmt_hierarchy* h, gmt_physics physics, double E, double nu, double k,
                     double tol, const double* u0, double* u_out, gmt_info* info);

/* Number of option sets gmt_autotune tries. */
#define GMT_AUTOTUNE_CANDIDATES 13

/* Solver-schedule autotuner: solves this hierarchy's cell problems to tol once per
   candidate and keeps the fastest. Candidate i (0..11) sets nu_pre = nu_post = 1 + i / 6,
   nu_coarse = 1 + (i / 2) % 3, coarse_fp16 = i % 2 (with GMT_PREC_FP64 the FP16 candidates
   are skipped); candidate 12 is the fastest of those with inner_tol = 0.003 (mixed
   precision, when the hierarchy's inner_tol is larger; else skipped); the other options
   stay the hierarchy's.
   Each solve starts from zero and is timed with CUDA events on the hierarchy's stream,
   after one untimed solve and after the lazily built operators of every candidate exist.
   The fastest candidate that returned GMT_OK is set on the hierarchy and written to best
   (nullable); times_ms (nullable, GMT_AUTOTUNE_CANDIDATES entries) receives each
   candidate's time in ms, infinity for a skipped or unconverged one. The 4^3 brick and
   the kernels' tile shapes are fixed by the data layout and are not tuned.
   GMT_NOT_CONVERGED if no candidate converged (the options are then unchanged). */
gmt_status gmt_autotune(gmt_hierarchy* h, gmt_physics physics, double E, double nu, double k,
                        double tol, gmt_options* best, double* times_ms);

/* Solves the cell problems of n (1..GMT_BATCH_MAX) distinct hierarchies together, each
   exactly as gmt_solve(hs[i], physics, E, nu, k, tol, u0[i], u_out[i], &info[i]) would:
   every field, gmt_info and stored solution is bitwise what that call returns, including
   the FP64 fallback of a diverging cell. One host thread per hierarchy runs its solve on
   the hierarchy's own stream; the mixed-precision V-cycles of all lattices still iterating
   run as one batched V-cycle (as gmt_vcycle_batch) on a stream of the call's own, so the
   small coarse levels of all cells share each launch. The hierarchies must be on one
   device and use mixed precision (GMT_PREC_FP32), the damped-Jacobi smoother and the
   V-cycle with the same omega, nu_pre, nu_post, nu_coarse and coarse_fp16, without
   element densities;
   their sizes and level counts may differ. u0 and u_out are arrays of n device pointers,
   or NULL (entries may be NULL: zero start / no copy out, as for gmt_solve); info and
   status, if not NULL, receive n entries. Returns GMT_OK when every lattice returned
   GMT_OK, else the first lattice's other status (gmt_last_error names the lattice). */
gmt_status gmt_solve_batch(gmt_hierarchy* const* hs, int n, gmt_physics physics, double E,
                           double nu, double k, double tol, const double* const* u0,
                           double* const* u_out, gmt_info* info, gmt_status* status);

/* Homogenized tensor (App. F.1 C^H, App. F.2 kappa^H): CH_out host double[M][M]
   row-major = 1/N^3 sum_e (x0^I - u_e^I)^T K_e (x0^J - u_e^J). u: device canonical field,
   or NULL for the field of the last gmt_solve on this hierarchy. That stored field stays
   as the solve left it through later calls on the hierarchy (per-level steps in either
   precision, residuals, C^H or sensitivities of other fields); a new material, new
   densities or another solve replace or discard it. */
gmt_status gmt_homogenize(gmt_hierarchy* h, gmt_physics physics, double E, double nu,
                          double k, const double* u, double* CH_out);

/* Element densities of the SIMP interpolation (App. F.3): element e of level 0 (canonical
   element order, gmt_element_coords) gets the material C_e = (rho_min + rho_e^p) C0
   (kappa_e likewise). rho: double[n_elems] with every rho_e in [0, 1], host memory if
   rho_on_device == 0, else device memory; read during the call. rho_min >= 0, simp_p > 0,
   and every coefficient rho_min + rho_e^p must be positive. rho == NULL returns to the binary
   design (every active element C0). The densities stay with the hierarchy; the operators of
   Sec. 4.6 (level-0 operator, element-local Galerkin products) are rebuilt with them on the
   next gmt_prepare / gmt_solve, and gmt_homogenize / gmt_sensitivities use them. The stored
   solution is discarded. With densities the level-0 operator is applied from stored
   per-node stencils (as the coarse levels are) instead of being formed from the octant
   masks. Errors: GMT_ERR_ARG (bad values), GMT_ERR_OOM, GMT_ERR_CUDA. */
gmt_status gmt_set_densities(gmt_hierarchy* h, const double* rho, int rho_on_device,
                             double rho_min, double simp_p);

/* Inverse-homogenization sensitivities (App. F.3): for the SIMP interpolation
   C_e = (rho_min + rho_e^p) C0, dC^H_IJ / d rho_e = p rho_e^(p-1) / |Omega|
   (x0^I - u_e^I)^T K0 (x0^J - u_e^J), u the solution for the current densities (the binary
   design, rho_e = 1 and factor p / N^3, when none are set). simp_p: the penalisation p
   (> 0; with densities it must equal the p given to gmt_set_densities). u: device canonical
   field, or NULL for the field of the last gmt_solve. dCH_out: device, caller-owned
   double[n_elems][M][M] in canonical element order (gmt_element_coords, level 0), symmetric
   in (I, J). Summed over the elements of the binary design it equals p C^H. */
gmt_status gmt_sensitivities(gmt_hierarchy* h, gmt_physics physics, double E, double nu,
                             double k, double simp_p, const double* u, double* dCH_out);

/* Relative residuals ||f_m - K u_m|| / ||f_m|| of a device canonical field u (host out[M]),
   with the solver's outer residual (precision FP32: float-float difference form;
   FP64: native FP64). */
gmt_status gmt_residual(gmt_hierarchy* h, int precision, const double* u, double* out);

/* ---- allocation-free homogenization --------------------------------------------------
   The paper has no counterpart to this call. It serves callers that cannot allocate device
   memory (an application whose memory manager owns the device and forbids side
   allocations, a fixed-budget embedded or sandboxed process, a latency-bound loop that
   cannot pay for an allocation's implicit device synchronisation). It computes the same
   energy average as gmt_homogenize, in FP64, for a nodal field the caller already holds,
   without a hierarchy and without any allocation: the working memory is a 352 KB array
   inside the library that each GPU using the library keeps until the process exits.
   voxels: device uint8[N^3] (x fastest). u_dense: device double[N^3][D][M], the field at
   every node site x + N*y + N^2*z (values at sites without an active element are
   ignored). CH: device double[M][M] written row-major. res: N, at most 512 (larger values
   are rejected with GMT_ERR_ARG). stream: cudaStream_t (nullable); the call is
   asynchronous on it and does not synchronise.
   The first call on a device looks up the array's device address (once per device, with
   that device current); make that first call before any stream capture. All calls share
   the array: calls that overlap on the GPU (other streams or host threads) race with each
   other and must be serialised by the caller. */
gmt_status gmt_homogenize_dense_noalloc(const uint8_t* voxels, int res, gmt_physics physics,
                                        double E, double nu, double k, const double* u_dense,
                                        double* CH, void* stream);

/* ---- tracing (measurement support; not part of the method) -----------------------------
   When enabled, the library records a CUDA event pair on its stream around every launch of
   the kernels below and accumulates, per category, the launch count, the summed device time
   and the algorithmic bytes (the bytes the operation must move per active node, times the
   active nodes: vectors read + written, counted once; no halo re-reads).
   Categories: 0 level-0 smoother sweep (Jacobi / Chebyshev stencil), 1 level-0 residual in the
   V-cycle, 2 level-0 operator apply (CG), 3 outer residual (float-float or FP64), 4 level-0
   first smoothing step (diagonal), 5 level-1 stencils (smoother, residual, first step),
   6 restriction, 7 prolongation, 8 coarsest solve, 9 C^H energy reduction, 10 vector /
   reduction kernels, 11 hierarchy build, 12 operators (element matrices, Galerkin products,
   block-diagonal inverses, node stencils), 13 coarsest matrix and its inverse, 14 stencils
   of levels >= 2, 15 whole V-cycles of gmt_solve (one event pair around each, its bytes 0).
   on == 2 records category 15 alone, without the per-launch events inside the V-cycles. */
#define GMT_TRACE_CATEGORIES 16
gmt_status gmt_trace_enable(gmt_hierarchy* h, int on);   /* on != 0 enables; resets totals */
/* Totals since enabling (synchronizes the stream): launches, device milliseconds, bytes. */
gmt_status gmt_trace_query(gmt_hierarchy* h, int category, int64_t* launches, double* ms,
                           double* bytes);
const char* gmt_trace_name(int category);
/* Kernels launched by this process through the library so far (all hierarchies). */
int64_t gmt_launch_count(void);

/* ---- device memory pool -----------------------------------------------------------------
   Device memory of hierarchies, operators and solver buffers comes from a process-wide
   caching pool: gmt_free_hierarchy returns it to the pool instead of the driver, so that
   the next cell reuses it without cudaMalloc / cudaFree. gmt_release_cached_memory hands
   every cached (unused) block back to the driver; a failed allocation does so first and
   retries. gmt_cached_bytes reports the bytes held unused by the pool. Thread-safe. */
void gmt_release_cached_memory(void);
int64_t gmt_cached_bytes(void);

/* ---- learned initializer (Sec. 4.2-4.3, Alg. 2) -------------------------------------------
   A sparse 3D convolutional U-Net over levels 0-2 of a hierarchy predicts the fine-level
   field from the geometry; gmt_solve then refines it as its warm start u0, and the plain
   V-cycles run on until the tolerance is met (the fallback). The paper's initializer is a
   transformer; this network is a convolutional U-Net of about 2M parameters with the same
   role (input: the octant masks; output: the fine field; trained on solved fields).
   Activations are FP32 [node][channel] over the canonical active nodes of a level. Every
   convolution has 27 taps, tap t = (dz+1)*9 + (dy+1)*3 + (dx+1); a missing neighbour adds 0:
     same-level  z[n] = b + sum_t W[t]^T x[node n + d_t]            (periodic wrap)
     down l->l+1 z[q] = b + sum_t W[t]^T x[fine node 2q + d_t]
     up l+1->l   z[p] = b + sum_t W[t]^T x[coarse node q, p = 2q + d_t]
   y = relu(z + skip). Twelve layers for widths (w0, w1, w2) and cout outputs:
     0 same@0 8->w0, 1 same@0 w0->w0, 2 down w0->w1, 3 same@1 w1->w1, 4 down w1->w2,
     5 and 6 same@2 w2->w2, 7 up w2->w1 + skip(act 4), 8 same@1 w1->w1,
     9 up w1->w0 + skip(act 2), 10 same@0 w0->w0, 11 same@0 w0->cout without relu.
   (activation 0 is the input, activation i+1 the output of layer i). Input channels: the
   node's octant mask bits. Output: cout = D*M channels = the field in canonical
   [node][D][M] order divided by `scale`. Parameters: FP32, per layer W [27][cin][cout] then
   b [cout], layers in order. Losses against a solved canonical field u:
     GMT_UNET_LOSS_MSE     mean over nodes and channels of (y - u/scale)^2;
     GMT_UNET_LOSS_ENERGY  (e^T K e) / (u^T K u), e = scale*y - u, summed over the load
                           cases: the relative energy norm of the warm start's error, the
                           norm conjugate gradients minimise (K: the level-0 operator of the
                           material prepared on the graph's hierarchy, applied in FP32).
   Optimizer: AdamW with bias-corrected moments and decoupled weight decay. */
#define GMT_UNET_LOSS_MSE 0
#define GMT_UNET_LOSS_ENERGY 1
typedef struct gmt_unet gmt_unet;
typedef struct gmt_netgraph gmt_netgraph;
typedef struct {
  double lr, beta1, beta2, eps, weight_decay;
} gmt_adamw;

/* Parameter count for out_channels and widths[3]; -1 for a bad shape. */
int64_t gmt_unet_param_count(int out_channels, const int* widths);
/* Layer table, host int32[12][6]: kind (0 same, 1 down, 2 up), output level, input
   activation, skip activation (-1 none), cin, cout. */
gmt_status gmt_unet_layers(int out_channels, const int* widths, int32_t* layers_out);
/* New network on the current device with parameters copied from `params` (host or device
   float[gmt_unet_param_count]); the initial values are the caller's (random draws are
   inputs). AdamW moments start at zero. Release with gmt_unet_free. */
gmt_status gmt_unet_create(int out_channels, const int* widths, const float* params,
                           gmt_unet** out);
void gmt_unet_free(gmt_unet* net);
int64_t gmt_unet_num_params(const gmt_unet* net);
/* Copy the parameters out / in (host or device float[P]); set also zeroes the moments. */
gmt_status gmt_unet_get_params(const gmt_unet* net, float* dst);
gmt_status gmt_unet_set_params(gmt_unet* net, const float* src);

/* Neighbour tables and input features of a hierarchy with at least 3 levels (GMT_ERR_RES
   otherwise), on the hierarchy's stream at build time; owns the activation buffers of the
   last network shape used with it. Release with gmt_netgraph_free (the hierarchy may be
   freed first). */
gmt_status gmt_netgraph_build(gmt_hierarchy* h, gmt_netgraph** out);
void gmt_netgraph_free(gmt_netgraph* g);
int64_t gmt_netgraph_nodes(const gmt_netgraph* g, int level);   /* level 0..2, else -1 */
/* Tables of `level` (host or device int32, each nullable): same [n_l][27] canonical
   neighbours; for level < 2, down [n_{l+1}][27] fine nodes 2q + d_t and up [n_l][27]
   coarse nodes q with p = 2q + d_t; -1 where none. */
gmt_status gmt_netgraph_tables(const gmt_netgraph* g, int level, int32_t* same_out,
                               int32_t* down_out, int32_t* up_out);

/* u_out (device double[n_0][cout]) = scale * network output: the predicted canonical field,
   ready to pass to gmt_solve as u0. */
gmt_status gmt_unet_forward(gmt_unet* net, gmt_netgraph* g, double scale, double* u_out);

/* Inference on the 5th-generation tensor cores: with on != 0, gmt_unet_forward runs every
   layer as an implicit-GEMM gather convolution with FP16 operands (weights and the gathered
   activations rounded to FP16 per call) and FP32 accumulation in tensor memory; the
   prediction then differs from the FP32 forward by FP16 rounding (about 1e-3 relative).
   Training (gmt_unet_gradient, gmt_unet_train_step) always runs in FP32. Off by default.
   GMT_ERR_CUDA from gmt_unet_forward if a bounded wait inside the kernel ran out. */
gmt_status gmt_unet_set_tensor_cores(gmt_unet* net, int on);
/* Loss against the canonical field u_target (device double[n_0][cout]) and its gradient
   with respect to every parameter (grad_out: host or device float[P], nullable; loss_out:
   host, nullable). The parameters do not change. h: the hierarchy the graph was built
   from, with a material prepared whose values per node equal cout (GMT_ERR_STATE if none);
   used by GMT_UNET_LOSS_ENERGY only (nullable for GMT_UNET_LOSS_MSE). */
gmt_status gmt_unet_gradient(gmt_unet* net, gmt_netgraph* g, gmt_hierarchy* h, int loss_kind,
                             const double* u_target, double scale, float* grad_out,
                             double* loss_out);
/* One training step: forward, loss, backward, AdamW update of the parameters. loss_out
   (host, nullable): the loss before the update. h and loss_kind as for gmt_unet_gradient. */
gmt_status gmt_unet_train_step(gmt_unet* net, gmt_netgraph* g, gmt_hierarchy* h, int loss_kind,
                               const double* u_target, double scale, const gmt_adamw* hp,
                               double* loss_out);

#ifdef __cplusplus
}
#endif

#endif /* GMT_H */
