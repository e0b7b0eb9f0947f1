/*
 * mgar.h - C ABI of the GB300 (sm_103a) library for multigrid-assisted
 * reanalysis (MGAR) heat-transfer topology optimisation.
 *
 * The operations follow Yin, Wang, Guo, Li, "An efficient topology
 * optimization based on multigrid assisted reanalysis for heat transfer
 * problem" (arXiv 2210.00947).  Each entry point cites the passage that
 * defines what it computes.
 *
 * Conventions shared by every call
 *   - Grid: nx x ny (x nz) unit elements; nz = 0 selects 2D bilinear (Q4)
 *     elements, nz > 0 3D trilinear (H8) elements.  Nodes and elements are
 *     numbered x-fastest: node(i,j,k) = i + (nx+1)*(j + (ny+1)*k),
 *     elem(i,j,k) = i + nx*(j + ny*k).  n = number of nodes, E = number of
 *     elements.
 *   - Arrays named "device" are CUDA device pointers owned by the caller;
 *     the library never frees them and keeps no reference after the call
 *     returns.  Arrays named "host" are plain host memory, read during the
 *     call only.
 *   - Every call is ordered on the CUDA stream given to mgar_create (or
 *     mgar_set_stream).  A call that returns a scalar through a host
 *     pointer synchronises that stream before returning.
 *   - Return value: MGAR_OK (0) or a negative MGAR_ERR_* code;
 *     mgar_last_error() then describes the failure.  A handle is not
 *     thread-safe: use one handle per host thread.
 *   - Fixed (Dirichlet, T = 0) nodes are eliminated: the operator is
 *     A = Z K Z + (I - Z), Z = diag(free nodes).
 */
#ifndef MGAR_H_
#define MGAR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGAR_OK 0
#define MGAR_ERR_ARG (-1)       /* invalid argument or size */
#define MGAR_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define MGAR_ERR_NOT_SPD (-3)   /* a Cholesky factorisation met a non-positive pivot */
#define MGAR_ERR_MAXIT (-4)     /* MGCG stopped at cg_max without reaching eps2 */
#define MGAR_ERR_NONFINITE (-5) /* a NaN/Inf appeared in a solver scalar */
#define MGAR_ERR_STATE (-6)     /* call out of order (e.g. MGAR before any MGCG) */
#define MGAR_ERR_TOO_LARGE (-7) /* input beyond a fixed internal capacity */

#define MGAR_FP64 0  /* every step in FP64 */
#define MGAR_MIXED 1 /* FP32 multigrid preconditioner, FP64 elsewhere */

#define MGAR_GUESS_PREVIOUS 0 /* Eq. 17 as printed: V-cycle initial guess r_{i-1} */
#define MGAR_GUESS_ZERO 1     /* V-cycle from a zero initial guess */

typedef struct mgar_ctx* mgar_t;

/* Problem and solver parameters (Sections 2.1-2.2, 3.2).  All fields are
 * read at mgar_create. */
typedef struct mgar_params {
  int32_t nx, ny, nz;   /* elements per axis; nz = 0 for 2D */
  double k0, kmin;      /* solid / void conductivity (Eq. 4) */
  double penal;         /* SIMP exponent p (Eq. 4) */
  double rmin;          /* density-filter radius in element lengths (Eq. 6-8) */
  int32_t nl;           /* multigrid levels incl. the finest, >= 2 (Section 3.2) */
  int32_t m;            /* MGAR basis size, 1..8 (Eq. 14) */
  double eps1;          /* MGAR acceptance threshold on Res (Eq. 28) */
  double eps2;          /* MGCG relative residual tolerance (Section 3.2) */
  int32_t cg_max;       /* MGCG iteration cap (Section 3.2) */
  double omega;         /* damped-Jacobi weight (Section 2.2) */
  int32_t nu_pre, nu_post; /* smoothing sweeps before / after the coarse correction */
  int32_t precision;    /* MGAR_FP64 or MGAR_MIXED */
  int32_t basis_guess;  /* MGAR_GUESS_PREVIOUS or MGAR_GUESS_ZERO (Eq. 17) */
  int32_t n_on;         /* MGAR activation cycle N_on (Section 3.1) */
  double volfrac;       /* volume fraction of the OC update */
  double move;          /* OC move limit */
  /* Continuous filter radius (Section 2.3, Eq. 22-23): design cycle k of
   * mgar_step / mgar_run filters with r^(k) = max(rmin, eta r^(k-1)),
   * r^(0) = filter_alpha * filter_L, eta = exp((ln rmin - ln r^(0)) /
   * filter_lp).  Off when filter_alpha <= 0 (the filter keeps rmin); with
   * filter_L <= 0 the longest side in elements is used.  The largest radius
   * must leave at most 3072 filter offsets (about r <= 31 in 2D, 9 in 3D),
   * else mgar_create fails with MGAR_ERR_ARG. */
  double filter_alpha;
  int32_t filter_lp;
  double filter_L;
} mgar_params;

/* Per-cycle report of mgar_step. */
typedef struct mgar_step_info {
  double compliance;  /* f = q^T t (Eq. 5) */
  double res;         /* MGAR residual Res (Eq. 28), NaN when MGAR did not run */
  double relres;      /* MGCG final relative residual, NaN when MGCG did not run */
  double lambda;      /* OC multiplier */
  int32_t used_mgcg;  /* 1 when MGCG produced t (N_on or Eq. 28 rejection) */
  int32_t accepted;   /* 1 when the MGAR solution was accepted */
  int32_t cg_iters;   /* MGCG iterations of this cycle */
  int32_t status;     /* MGAR_OK, or MGAR_ERR_MAXIT when MGCG hit cg_max */
  double compliance_mgar; /* q^T t~ of the MGAR reduced solution (Eq. 5, 21) whether
                             Eq. 28 accepted it or not; NaN when MGAR did not run */
} mgar_step_info;

/* Fill *p with the defaults of the paper's experiments (Section 3.2): k0 1,
 * kmin 1e-3, p 3, rmin 1.5, nl 4, m 2, eps1 0.5, eps2 1e-8, cg_max 200,
 * omega 0.9, one pre- and post-sweep, FP64, Eq. 17 as printed, n_on 0,
 * volfrac 0.4, move 0.2.  The grid size is left zero. */
void mgar_default_params(mgar_params* p);

/* Create a handle for one design domain (Eq. 3-5).
 *   fixed_mask: host, n bytes, non-zero marks a T = 0 node.
 *   q:          host, n doubles, nodal heat load (entries on fixed nodes
 *               are ignored and treated as zero).
 *   stream:     cudaStream_t to order all work on (NULL = legacy default).
 * Allocates all device workspaces; the caller's arrays are copied.
 * Errors: MGAR_ERR_ARG on bad sizes/parameters (nl too deep for the grid,
 * m out of range), MGAR_ERR_CUDA on allocation failure. */
int mgar_create(mgar_t* out, const mgar_params* p, const uint8_t* fixed_mask, const double* q,
                void* stream);

/* Release every device allocation of the handle.  h may be NULL. */
int mgar_destroy(mgar_t h);

/* Change the stream later calls are ordered on. */
int mgar_set_stream(mgar_t h, void* stream);

/* Text of the last error on this handle (never NULL). */
const char* mgar_last_error(mgar_t h);

/* Density filter, Eq. 6-8 (transpose = 0): out_e = sum_i w_ei in_i /
 * sum_i w_ei with w_ei = max(0, rmin - |c_e - c_i|) over in-domain
 * elements.  transpose = 1 applies the adjoint used by the chain rule of
 * Eq. 9 and 11: out_j = sum_e w_ej in_e / sum_i w_ei.
 *   in, out: device, E doubles, must not overlap. */
int mgar_filter(mgar_t h, const double* in, double* out, int transpose);

/* Set the current design.  rho: device, E doubles.  is_physical = 0
 * filters rho first (Eq. 6); 1 takes rho as the physical density rho~.
 * The element conductivities k_e = kmin + (k0-kmin) rho~^p (Eq. 4) are
 * derived here; the multigrid hierarchy is not touched. */
int mgar_set_density(mgar_t h, const double* rho, int is_physical);

/* Replace the nodal heat load q of Eq. 3 (the right-hand side of every
 * later MGCG / MGAR solve, the compliance of Eq. 5 and the Res of Eq. 28).
 *   q: device, n doubles, copied; entries on fixed nodes are treated as zero.
 * A solve for another right-hand side, such as the difference solve
 * (K + dK) dt = -dK t of a finite-difference check, sets its load here and
 * the original one back afterwards.  Errors: MGAR_ERR_ARG when q is NULL or
 * zero on every free node. */
int mgar_set_load(mgar_t h, const double* q);

/* y = A(rho~) x for the current design (Eq. 3, fixed nodes eliminated).
 *   x, y: device, n doubles, must not overlap. */
int mgar_apply_K(mgar_t h, const double* x, double* y);

/* Build the multigrid hierarchy of the current design and make it the
 * reference ("factorised") matrix K0 of Eq. 12 (Table 1 operators, Galerkin
 * coarse levels A_{l+1} = P^T A_l P, coarsest level factorised). */
int mgar_build_hierarchy(mgar_t h);

/* One V-cycle x <- MG(K0, b, x, P) on the reference hierarchy (Table 1).
 *   b: device, n doubles; x: device, n doubles, initial guess in, result
 *   out.  Errors: MGAR_ERR_STATE if no hierarchy was built yet. */
int mgar_vcycle(mgar_t h, const double* b, double* x);

/* MGCG solve of A(rho~) T = q for the current design (Section 3.2): the
 * hierarchy is rebuilt from the current design (K0 <- K), then CG
 * preconditioned by one V-cycle runs until ||r||/||q|| <= eps2 or cg_max
 * iterations.
 *   T: device, n doubles, warm start in, solution out.
 *   iters, relres: host, may be NULL.
 * Returns MGAR_ERR_MAXIT (T still written) when cg_max was reached,
 * MGAR_ERR_NONFINITE on breakdown. */
int mgar_solve_mgcg(mgar_t h, double* T, int* iters, double* relres);

/* MGAR reanalysis (Eq. 17-21 and 28) of the current design on the reference
 * hierarchy K0: basis from t_prev by V-cycles, Gram-Schmidt, reduced
 * m x m Cholesky solve, Res = ||K R~ y - q|| / ||q||.
 *   T_prev: device, n doubles (r_1 of Eq. 15); T: device, n doubles, the
 *   reduced solution t~ = R~ y.  T may alias T_prev.
 *   res, accepted: host, may be NULL; accepted = (Res <= eps1).
 * No fallback inside: the caller decides what to do on rejection.
 * Errors: MGAR_ERR_STATE if no hierarchy exists. */
int mgar_solve_mgar(mgar_t h, const double* T_prev, double* T, double* res, int* accepted);

/* Compliance and design sensitivities (Eq. 5, 9-11) for the current design
 * and temperatures T:
 *   dc_j = sum_e w_ej/sum_i w_ei * (-p (k0-kmin) rho~_e^(p-1) t_e^T k0 t_e).
 *   T: device n doubles; dc: device E doubles (may be NULL);
 *   dv: device E doubles (may be NULL), gradient of mean(rho~);
 *   compliance: host (may be NULL), q^T T. */
int mgar_sensitivity(mgar_t h, const double* T, double* dc, double* dv, double* compliance);

/* Projection-based boundary post-processing (Section 2.3, Eq. 24-27), run
 * once after the optimisation: the element sensitivities of the design
 * (Eq. 10, magnitude) are projected onto the nodes with the filter's weights
 * (radius rmin); an element is solid when all its nodes exceed the level,
 * void when all are below it, and otherwise gets the share of a 5 x 5
 * (x 5) lattice of points over the element at which the bilinear /
 * trilinear interpolation of the nodal values exceeds the level (Eq. 25-27);
 * the level is bisected so that the mean density is the largest attainable
 * at or below volfrac.
 *   rho: device E doubles, the design (filtered inside); T: device N
 *   doubles, its temperatures; rho_out: device E doubles (densities in
 *   [0, 1], multiples of 1/25 or 1/125).  level, volume: host (may be NULL).
 *   Errors: MGAR_ERR_ARG on null pointers or volfrac outside (0, 1). */
int mgar_postprocess(mgar_t h, const double* rho, const double* T, double volfrac, double* rho_out,
                     double* level, double* volume);

/* Optimality-criteria update (not in the paper; the classical SIMP
 * framework it names): rho <- clamp(rho sqrt(-dc/(lambda dv)), rho-move,
 * rho+move, [0,1]) with lambda by bisection so that mean(F rho) = volfrac.
 *   rho: device E doubles, updated in place; dc: device E doubles.
 *   lambda, change: host (may be NULL); change = max |rho_new - rho|. */
int mgar_oc_update(mgar_t h, double* rho, const double* dc, double volfrac, double move,
                   double* lambda, double* change);

/* One design cycle of the MGAR-based loop (Section 3.1, Figure 5): filter,
 * then MGCG when cycle < n_on or no reference exists, else MGAR with MGCG
 * fallback when Res > eps1; then compliance, sensitivities and the OC
 * update of rho.
 *   rho: device E doubles (design, updated in place); T: device n doubles
 *   (previous temperatures in, this cycle's out); cycle: 1-based.
 *   info: host, may be NULL. */
int mgar_step(mgar_t h, double* rho, double* T, int cycle, mgar_step_info* info);

/* Sizes of the handle's grid: nodes, elements. */
int mgar_sizes(mgar_t h, int64_t* n_nodes, int64_t* n_elems);

/* A whole optimisation run from host memory (Section 3.1, Figure 5): copy
 * rho_host (E doubles, pinned or pageable) to the device, start from zero
 * temperatures and no reference matrix, run design cycles 1..cycles of
 * mgar_step, then copy the final design to rho_out_host (E doubles) and one
 * mgar_step_info per cycle to info_host (cycles entries, may be NULL).
 * Device work buffers are allocated on the first call and kept. */
int mgar_run(mgar_t h, const double* rho_host, int cycles, double* rho_out_host,
             mgar_step_info* info_host);

/* Instrumentation (no counterpart in the paper).  Kernel classes whose
 * launches can be timed with CUDA events on the handle's stream: */
#define MGAR_KC_APPLY64 1 /* finest-level K x of the outer CG and the MGAR projection:
                             FP64, or double-float (df64) in the mixed path (on 3D
                             grids the mixed path's CG iterations use MGAR_KC_APPLY32
                             and its residuals MGAR_KC_RESID64) */
#define MGAR_KC_SMOOTH0 2 /* finest-level smoothing passes of the V-cycle (any precision) */
#define MGAR_KC_RESID0 3  /* finest-level residual inside the V-cycle */
#define MGAR_KC_OC 4      /* OC bisection pass */
#define MGAR_KC_GALERKIN0 5 /* Galerkin element matrices of level 1 */
#define MGAR_KC_FILTER 6  /* density filter / its transpose */
#define MGAR_KC_SENS 7    /* element sensitivities (Eq. 10) */
#define MGAR_KC_APPLY32 8 /* mixed path, 3D: FP32 direction update + K p + p.Kp of a CG iteration */
#define MGAR_KC_RESID64 9 /* mixed path, 3D: df64 residual q - K x of the CG (its start and
                             every reliable update) */
#define MGAR_KC_TIMELINE 100 /* every launch site: device time between consecutive launches */

/* Start timing every launch of one kernel class (0 stops).  Each launch
 * is bracketed by two CUDA events; at most 65536 launches are recorded. */
int mgar_profile_start(mgar_t h, int kernel_class);
/* Stop, synchronise the stream, and return the summed duration (ms) and
 * the number of timed launches.  With MGAR_KC_TIMELINE an event follows
 * every launch site (and graph replay); the device time between two
 * consecutive events is charged to the later site, and the per-site totals
 * become available through mgar_profile_report. */
int mgar_profile_stop(mgar_t h, double* total_ms, int64_t* launches);

/* Text table (site, launches, ms, share) of the last MGAR_KC_TIMELINE
 * session, written to buf (host, len bytes, NUL-terminated). */
int mgar_profile_report(mgar_t h, char* buf, int64_t len);

/* Number of kernels this library has launched in this process (all
 * handles), for accounting in benchmarks. */
int64_t mgar_kernel_launches(void);

/* Batched MGCG over many independent 2D designs (Section 3.2's solve with
 * the Table 1 V-cycle as preconditioner), each design a handle of its own
 * (its grid, sink, load, density and parameters).  A batch holds no copy of
 * the designs' data, only device tables of their sizes and buffers: every
 * step of the solve is one launch over all designs (one per V-cycle level
 * and operation), the outer CG runs in double-float arithmetic (FP64
 * accuracy on the FP32 pipe; FP64 scalars) around the FP32 V-cycle, and
 * the solve after the hierarchy builds is one CUDA graph that iterates while
 * any design is unconverged.  The V-cycle kernels' block sizes come from an
 * autotuner at the first solve (mgar_batch_report lists its timings and
 * choices); no choice changes a result, and each design's result does not
 * depend on the other designs in the batch. */
typedef struct mgar_batch_ctx* mgar_batch_t;

/* Create a batch over `count` handles (host array), all 2D and created with
 * MGAR_MIXED; a handle may appear once.  The handles must outlive the batch
 * and must not be used by other calls while a batch call runs.  Batch calls
 * run one at a time per process (calls from several host threads wait for
 * each other: concurrent batches gave differing results and once an illegal
 * address in an experiment).  Work is
 * ordered on `stream` (cudaStream_t, NULL = legacy default).
 * Errors: MGAR_ERR_ARG (bad arguments, 3D or FP64 handles), MGAR_ERR_CUDA. */
int mgar_batch_create(mgar_batch_t* out, const mgar_t* handles, int count, void* stream);

/* Release the batch (not its handles).  b may be NULL. */
int mgar_batch_destroy(mgar_batch_t b);

/* Text of the batch's last error (b = NULL: of the last failed create). */
const char* mgar_batch_last_error(mgar_batch_t b);

/* Solve A(rho~_d) T_d = q_d for every design d of the batch at its current
 * density (mgar_set_density), as mgar_solve_mgcg does for one handle: each
 * handle's hierarchy is rebuilt from its design (K0 <- K), then the
 * preconditioned CG runs until the design's ||r|| / ||q|| <= eps2 or its
 * cg_max, designs finishing independently.
 *   T: host array of `count` device pointers, each n_d doubles: warm start
 *      in, solution out.
 *   iters, relres, status: host arrays of `count` entries, each may be NULL;
 *      status[d] is MGAR_OK, MGAR_ERR_MAXIT or MGAR_ERR_NONFINITE.
 * Returns MGAR_OK, or the worst per-design status (solutions still written),
 * or MGAR_ERR_NOT_SPD when a coarsest factorisation failed.  Synchronises
 * the stream. */
int mgar_batch_solve_mgcg(mgar_batch_t b, double* const* T, int* iters, double* relres,
                          int* status);

/* One design cycle of Figure 5 with MGCG for every design of the batch
 * (Eq. 6-8 filter and Eq. 4 SIMP, the batched solve of Eq. 3, the
 * compliance of Eq. 5, the sensitivities of Eq. 9-11 and the OC update), as
 * mgar_step does for one handle with n_on past the cycle.  All of it runs on
 * the batch's stream, ordered after what each handle's stream holds: every
 * design's filter, SIMP and hierarchy as one CUDA graph of per-design
 * branches, the solve graph, every design's update as one graph, then one
 * read of all outcomes.  The per-design graphs are kept while the pointers,
 * volume fractions and move limit passed stay the same, and captured again
 * otherwise.  When a handle times a kernel class or runs without graphs, the
 * same launches are issued on the handles' own streams instead.
 *   rho:     host array of `count` device pointers, each ne_d doubles: the
 *            design in, the updated design out.
 *   T:       host array of `count` device pointers, each n_d doubles: warm
 *            start in, this cycle's temperatures out.
 *   volfrac: host array of `count` volume fractions in (0, 1).
 *   move:    OC move limit (> 0), the same for every design.
 *   info:    host array of `count` reports (may be NULL): compliance, CG
 *            iterations, relative residual, lambda, status per design.
 * Returns as mgar_batch_solve_mgcg.  Errors: MGAR_ERR_ARG (null pointers,
 * volfrac or move out of range, a handle with the continuation filter
 * schedule of filter_alpha, which follows mgar_step's cycle count).
 * Synchronises the batch's stream (and with it all the work of the call). */
int mgar_batch_cycle(mgar_batch_t b, double* const* rho, double* const* T, const double* volfrac,
                     double move, mgar_step_info* info);

/* The autotuner's timings and choices as text (empty before the first
 * solve), written to buf (host, len bytes, NUL-terminated). */
int mgar_batch_report(mgar_batch_t b, char* buf, int64_t len);

/* Design sensitivities dc, as mgar_sensitivity computes them, for callers
 * that cannot allocate device memory (no counterpart in the paper): code
 * whose device memory is owned by a host framework's pool, or that must not
 * grow the process's device footprint after start-up.  No handle and no
 * allocation: the per-element intermediate lives in a static device array
 * of 2^20 doubles (8 MiB) that every GPU loading the library keeps until
 * the process exits.
 *   p:        host; nx, ny, nz, k0, kmin, penal, rmin and filter_alpha are
 *             read.  The filter is the fixed-radius one of radius rmin; a
 *             continuation schedule (filter_alpha > 0, Eq. 22-23) is refused
 *             with MGAR_ERR_ARG: pass the radius wanted as rmin instead.
 *   rho_phys: device, E doubles, the physical (filtered) density.
 *   T:        device, n doubles; dc: device, E doubles (output).
 *   stream:   cudaStream_t the two kernels are queued on.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call outside any
 * stream capture.  The address is kept for the life of the process, so a
 * device reset (cudaDeviceReset) after the first call is not supported.  All calls share the array, so calls whose work overlaps
 * on the GPU (other streams or host threads) race; each call writes every
 * entry it reads, so nothing needs clearing between calls.
 * Errors: MGAR_ERR_ARG (null pointer, bad grid, rmin > 8 or filter_alpha > 0),
 * MGAR_ERR_TOO_LARGE (more than 2^20 elements), MGAR_ERR_CUDA (symbol lookup
 * or launch failed).  Returns without synchronising the stream. */
int mgar_sensitivity_noalloc(const mgar_params* p, const double* rho_phys, const double* T,
                             double* dc, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MGAR_H_ */
