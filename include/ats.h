/*
 * ats.h -- C ABI of the GB300 (sm_103a) per-level implicit diffusion solver.
 *
 * The operation: one backward-Euler step of the heat / flux-limited-diffusion
 * operator restricted to one AMR level (Commerçon, Debout & Teyssier 2014,
 * Sect. 3.1, Eq. Er_imp and Eq. Er_imp1),
 *
 *     (1 + s_i + sum_f w_f C_f) E_i - sum_{f same-level leaf} C_f E_j = b_i,
 *
 * with C_f = factor * dt / dx^2 * (K_i + K_j) / 2 (factor 1 for a same-level
 * or restricted finer neighbour, 2/3 for a coarser neighbour, Sect. 3.1), the
 * interface rows of Sect. 3.2 (Dirichlet: w = 1, b += C E_nb; Neumann: w = 0,
 * b += F; Robin: w = alpha, b += alpha C E_nb + (1 - alpha) F), solved by
 * conjugate gradient with a diagonal preconditioner and the stopping rule of
 * Sect. 3.3.4.  The right-hand side is b_i = E^n_i + src_i + interface terms.
 *
 * Geometry (all arrays in "level order"):
 *   a level is a list of n_oct octs of 2x2x2 cells; oct o has integer oct
 *   coordinates (ox, oy, oz); its cell c = ix + 2 iy + 4 iz has the level
 *   cell coordinates (2 ox + ix, 2 oy + iy, 2 oz + iz) and the cell index
 *   8 o + c.  N = 8 n_oct.  Octs in Morton order give the best locality; any
 *   order is correct.  Face directions: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z.
 *   A cell is an unknown ("leaf") when its bit in leaf_mask is set.  A leaf
 *   face whose neighbour is not a same-level leaf (missing oct, refined cell)
 *   is an interface face: it takes the condition of its descriptor, or is a
 *   zero-flux wall when it has none.
 *
 * Memory and ownership: the library owns every device buffer it allocates.
 * Arguments marked "host" are read (or written) during the call only and stay
 * the caller's.  Per-step arrays may be host or device pointers, as the
 * caller's `mem` field says (ATS_MEM_HOST / ATS_MEM_DEVICE); device pointers
 * are borrowed for the call and used in stream order on the context's stream.
 * A host x that the device can address (pinned or registered memory) may be
 * written by the device during a solve call, as each solve ends; the call
 * returns (also on an error) only after every such write.
 *
 * Errors: every entry point returns an ats_status; 0 is success, < 0 an
 * error, > 0 a warning.  No C++ exception crosses this boundary.
 * ats_last_error() gives a message for the calling thread's last failure.
 * Threads: one context per thread; a context's objects are not thread-safe.
 */
#ifndef ATS_H
#define ATS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ats_status;
#define ATS_OK 0
#define ATS_ERR_INVALID_ARG (-1)   /* bad argument or level description      */
#define ATS_ERR_OOM (-2)           /* device allocation failed                */
#define ATS_ERR_OVER_BUDGET (-3)   /* the context's memory budget is spent    */
#define ATS_ERR_NOT_CONVERGED (-4) /* iteration / refinement cap reached      */
#define ATS_ERR_BREAKDOWN (-5)     /* CG breakdown: p.Ap <= 0 or non-finite  */
#define ATS_ERR_TIMEOUT (-6)       /* a bounded wait ran out                  */
#define ATS_ERR_CUDA (-7)          /* a CUDA runtime call failed              */
#define ATS_ERR_NO_DEVICE (-8)     /* no usable CUDA device                   */
#define ATS_ERR_BAD_INPUT (-9)     /* non-finite value or K <= 0 on a leaf    */
#define ATS_WARN_NEGATIVE 1        /* the solve succeeded but its result has a  */
                                   /* negative energy (the failure mode Sect. 4.2 */
                                   /* reports with Neumann interfaces); checked  */
                                   /* at the copy-out (not by ats_solve_noalloc) */

/* face kinds (Sect. 3.2) */
#define ATS_FACE_DIRICHLET 0
#define ATS_FACE_NEUMANN 1
#define ATS_FACE_ROBIN 2
/* face relations (Sect. 3.1): distance factor of the face coefficient */
#define ATS_REL_SAME 0    /* physical wall, ghost value at distance dx: 1    */
#define ATS_REL_COARSER 1 /* fine-to-coarse (Sect. 3.3.1): 2/3               */
#define ATS_REL_FINER 2   /* coarse-to-fine, restricted finer cell: 1        */

#define ATS_MEM_HOST 0
#define ATS_MEM_DEVICE 1

/* stopping rules (Sect. 3.3.4) */
#define ATS_STOP_RESIDUAL 0  /* ||r_j||_2 <= tol ||r_0||_2 (the paper's L2 rule)  */
#define ATS_STOP_CERTIFIED 1 /* ||b - A x||_2 <= tol ||x||_2; since the level      */
                             /* matrix has lambda_min >= 1 this bounds the        */
                             /* relative error of x by tol                          */
#define ATS_STOP_PAPER 2     /* L2 rule AND max_i |x_j - x_{j-1}| / |x_{j-1}| < tol */

/* precision of the CG bulk (vectors, stencil); dots are always FP64 */
#define ATS_PREC_FP64 0  /* FP64 everywhere                                    */
#define ATS_PREC_MIXED 1 /* FP32 vectors and stencil, FP64 dots, FP64 iterative */
                         /* refinement r = b - (I + dt A) x on FP64 K, b and x  */

typedef struct ats_context ats_context;
typedef struct ats_level ats_level;
typedef struct ats_batch ats_batch;

/* Topology of one level (host arrays, read during ats_level_create only). */
typedef struct {
  int64_t n_oct;
  const int32_t *oct_xyz;   /* host [n_oct * 3] oct coordinates, |coord| < 2^20 */
  const uint8_t *leaf_mask; /* host [n_oct] bit c = cell c is a leaf; NULL = all */
  double dx;                /* cell size of the level, > 0                       */
  int64_t n_face;           /* interface-face descriptors                        */
  const int32_t *face_cell; /* host [n_face] leaf cell index 8 o + c             */
  const int8_t *face_dir;   /* host [n_face] 0..5                                */
  const int8_t *face_kind;  /* host [n_face] ATS_FACE_*                          */
  const int8_t *face_rel;   /* host [n_face] ATS_REL_*                           */
  const double *face_alpha; /* host [n_face] Robin weight in [0,1]; NULL = 1     */
} ats_level_desc;

/* Per-step values of a level operator (Sect. 3.1-3.2, Sect. 3.3.4). */
typedef struct {
  double dt;            /* time step of the level, > 0                           */
  int mem;              /* ATS_MEM_HOST or ATS_MEM_DEVICE for the arrays below   */
  const double *K;      /* [N] cell diffusion coefficient, > 0 on leaf cells    */
  const double *E_old;  /* [N] E^n                                              */
  const double *s;      /* [N] diagonal shift (linearised coupling) or NULL     */
  const double *src;    /* [N] extra right-hand side or NULL                     */
  const double *face_K; /* [n_face] neighbour K of each descriptor, NULL = K_i   */
  const double *face_E; /* [n_face] neighbour value E_nb, NULL = 0              */
  const double *face_F; /* [n_face] imposed flux F (energy per unit volume into  */
                        /* the cell over the step), NULL = 0                     */
  int integrator;       /* ATS_INTEGRATOR_* (0 = backward Euler)                 */
} ats_coef_desc;

/* time integrator of a level step (ats_coef_desc.integrator) */
#define ATS_INTEGRATOR_BACKWARD_EULER 0 /* Eq. Er_imp1: (I + dt A) E^{n+1} = E^n + ...      */
#define ATS_INTEGRATOR_CRANK_NICOLSON 1 /* second order (Sect. 3.3.5 names it): the      */
        /* operator is built for dt/2 with F and src at half weight (they stay amounts  */
        /* over the full step), and every solve of the level returns 2 x' - E^n, where */
        /* x' solves that backward-Euler half step and E^n is the build's E_old; this  */
        /* equals the Crank-Nicolson step (I + dt/2 A) E^{n+1} = (I - dt/2 A) E^n + .. */
        /* An initial guess x on entry is a guess of E^{n+1}: the solve starts from   */
        /* (x + E^n) / 2.  The solve statistics, ats_level_get_rhs and               */
        /* ats_level_apply refer to the half-step system.  Not with a shift s         */
        /* (ATS_ERR_INVALID_ARG); device E_old must stay unchanged until the solve.   */
        /* Hierarchy substeps (ats_level_advance) integrate with backward Euler.    */

typedef struct {
  double tol;        /* stopping tolerance (default 1e-10)                    */
  int stop_rule;     /* ATS_STOP_*                                            */
  int precision;     /* ATS_PREC_*                                            */
  int max_iter;      /* cap on CG iterations per solve (0 = 20000)            */
  int max_refine;    /* cap on FP64 residual passes (0 = 40)                 */
  double inner_rtol; /* mixed: residual reduction per inner FP32 solve (0 = 1e-6) */
  int tile_octs;     /* octs per work item, multiple of 32 (0 = the size rule: */
                     /* about one item per CTA of the stencil kernel's grid, */
                     /* 256..1024; ats_batch_autotune tunes it per batch)    */
  int check_every;   /* ticks between host convergence polls (0 = 16)       */
  int use_graph;     /* 1 = each poll interval of check_every ticks is one CUDA graph, the host polls between intervals; 2 = the whole tick loop is one graph (a WHILE conditional node over one interval, ended on the device when no solve is active), the host waits once (with profiling on, 2 runs as 1); 3 = as 2 for a solve, and for ats_level_advance the whole step as one graph (see there) */
  int mem;           /* ATS_MEM_HOST / ATS_MEM_DEVICE for x (and rhs)        */
  int x0;            /* ATS_X0_*: where the initial guess comes from          */
  int sched;         /* ATS_SCHED_*: tick path or resident solver (0 = AUTO)  */
  int res_threads;   /* resident solver: threads per CTA, 256 or 512          */
                     /* (0 = 512 for ATS_PREC_MIXED, 256 for ATS_PREC_FP64)   */
  int res_cluster;   /* resident solver: CTAs per thread-block cluster, 1..16 */
                     /* (0 = 4)                                              */
  int res_cta_octs;  /* resident solver: a level of at most this many octs is */
                     /* solved by one CTA alone (0 = 2048, < 0 = never)      */
  int res_max_octs;  /* ATS_SCHED_AUTO: levels above this many octs take the  */
                     /* whole-GPU form or the tick path (see ATS_SCHED_AUTO) */
                     /* (0 = 16384 for ATS_PREC_MIXED, 2048 for              */
                     /* ATS_PREC_FP64)                                       */
  int cg_scalars;    /* resident solver, mixed precision: the CG step's alpha,  */
                     /* beta and inner convergence test from the error-free   */
                     /* dot totals, 0 = rounded to FP32 (the tick path's form, */
                     /* default), 1 = in FP64                                 */
  int res_state;     /* resident solver, mixed precision: where each CTA     */
                     /* keeps K, z and p of its octs: 0 = shared memory      */
                     /* (neighbours read from the owning CTA through          */
                     /* distributed shared memory; default), 1 = global      */
                     /* memory (L2).  The FP64 bulk always uses global.      */
  int res_cluster_big; /* resident solver: CTAs per cluster for the levels    */
                     /* whose runs on res_cluster_mid CTAs would not fit     */
                     /* their shared memory, or whose estimated work         */
                     /* exceeds res_big_work (0 = 16; < 0 = none)           */
  int res_big_work;  /* resident solver: a level of more than res_cta_octs   */
                     /* octs also takes the larger clusters when its        */
                     /* estimated work n_oct min(sqrt(1 + 8 h), 4 n_oct^(1/3)),*/
                     /* h = dt / (2 dx^2), exceeds this (0 = no work rule)   */
  int res_cluster_mid; /* resident solver: CTAs per cluster for the levels    */
                     /* whose runs on res_cluster CTAs would not fit their   */
                     /* shared memory but whose runs on this many would     */
                     /* (0 = 8; < 0 = none: they take res_cluster_big);     */
                     /* used only between res_cluster and res_cluster_big   */
  int cg_form;       /* resident solver, mixed precision: how each CG step    */
                     /* forms q = (I + dt A) p (Sect. 3.3.4).  1 = from the   */
                     /* new p, after a group barrier that makes every CTA's   */
                     /* p visible; 2 = by the recurrence                      */
                     /* q = (I + dt A) z + beta q_prev (equal in exact         */
                     /* arithmetic, since p = z + beta p_prev): z is final at */
                     /* the previous step's group sum, so the step needs no   */
                     /* barrier -- two group synchronisations per step        */
                     /* instead of three.  0 = the default (2)                */
} ats_solve_opts;

/* scheduling of a solve (ats_solve_opts.sched).  Which path a level takes
 * depends on that level and the options alone, so a level gives bitwise the
 * same result solved alone and in any batch with the same options.
 *   Tick path: every solve still running advances one CG step per "tick" (a
 *   stencil kernel, a refinement kernel and an update kernel over the active
 *   work items of all solves), ticks replayed as CUDA graphs, host or device
 *   polling between intervals; one solve spreads over the whole GPU.
 *   Resident solver: a solve runs from its first residual pass to its
 *   certificate inside one persistent launch, on one thread-block cluster of
 *   res_cluster CTAs (per-step sums exchanged through distributed shared
 *   memory, steps ordered by the hardware cluster barrier); a level whose
 *   runs on res_cluster CTAs would not fit their shared memory takes the
 *   smallest of res_cluster_mid and res_cluster_big CTAs whose runs fit (or
 *   res_cluster_big when its estimated work exceeds res_big_work, when
 *   set); a level of at most res_cta_octs octs runs on one CTA; clusters and CTAs take solves from work queues ordered
 *   by estimated work (largest first; after a completed run of a batch, by
 *   the measured durations); the cluster sizes and the single CTAs run as
 *   concurrent launches sharing the SMs in proportion to their queues'
 *   estimated work (after a completed run, their measured SM-time).  Not for the paper stopping rule (ATS_STOP_PAPER
 *   takes the tick path). */
#define ATS_SCHED_AUTO 0     /* resident solver for levels up to res_max_octs octs; */
        /* above it, FP32 bulk: the whole-GPU form (see ATS_SCHED_GRID) for a level */
        /* of at most 1 100 octs per CTA of that form (167 200 octs on 152 SMs),    */
        /* the tick path for larger levels and for FP64                             */
#define ATS_SCHED_TICK 1     /* the tick path for every level                    */
#define ATS_SCHED_RESIDENT 2 /* the resident solver for every level              */
#define ATS_SCHED_GRID 3     /* as AUTO, and every level above res_max_octs (FP32  */
        /* bulk) on the whole-GPU form of the resident solver: one cooperative     */
        /* launch, one CTA per SM, each CTA's run of octs with its CG arrays in     */
        /* shared memory, the faces across runs and the per-step sums through       */
        /* global memory, steps ordered by a grid barrier whose waits give up after */
        /* a bounded number of polls (the solve then ends with ATS_ERR_TIMEOUT);    */
        /* such levels run one after another, after the other resident solves.     */

/* initial guess of a solve (ats_solve_opts.x0) */
#define ATS_X0_GIVEN 0 /* x_inout holds the initial guess on entry (default) */
#define ATS_X0_E_OLD 1 /* start from E^n given to the level's last operator  */
                       /* build (the paper's initial guess, Sect. 3.3.4):     */
                       /* x_inout is output only.  Device E^n arrays must be  */
                       /* unchanged from the build to the end of the solve;   */
                       /* host E^n is kept in the library's staging copy.     */

typedef struct {
  int status;          /* ATS_OK or ATS_ERR_NOT_CONVERGED / _BREAKDOWN      */
  int iterations;      /* CG iterations (all inner passes)                   */
  int refinements;     /* FP64 true-residual passes                          */
  int ticks;           /* device steps taken                                 */
  double r0_norm;      /* ||b - A x_0||_2 (FP64)                             */
  double res_norm;     /* final ||b - A x||_2 (FP64, true residual)          */
  double x_norm;       /* ||x||_2                                            */
  double err_bound;    /* res_norm / x_norm: bound on the relative error     */
} ats_solve_stats;

/* ---- context ------------------------------------------------------------ */
/* Create a context on CUDA device `device` with a device-memory budget in
 * bytes (0 = no limit).  The context creates its own non-blocking stream. */
ats_status ats_context_create(int device, size_t mem_budget_bytes, ats_context **out);
ats_status ats_context_destroy(ats_context *ctx);
/* Use the caller's cudaStream_t (passed as void*) for all later work; NULL =
 * the context's own stream. */
ats_status ats_context_set_stream(ats_context *ctx, void *stream);
/* Bytes currently allocated by the context, and its budget. */
ats_status ats_context_memory(const ats_context *ctx, size_t *used, size_t *budget);

/* ---- level (Sect. 3.1: the grid of one AMR level) ------------------------ */
/* Build the oct neighbour table, the interface records and upload the
 * topology.  Errors: ATS_ERR_INVALID_ARG for duplicate octs, descriptors on
 * interior faces or non-leaf cells, duplicate descriptors, bad enums. */
ats_status ats_level_create(ats_context *ctx, const ats_level_desc *desc, ats_level **out);
ats_status ats_level_destroy(ats_level *lvl);
ats_status ats_level_size(const ats_level *lvl, int64_t *n_oct, int64_t *n_cell, int64_t *n_face);

/* Build the level operator for one step (kernel: coefficients, face
 * coefficients, diagonal extras and the right-hand side b, Sect. 3.1-3.2).
 * Errors: ATS_ERR_BAD_INPUT if K <= 0 on a leaf or any value is not finite. */
ats_status ats_level_build_operator(ats_level *lvl, const ats_coef_desc *coef);

/* Copy the assembled right-hand side b (FP64, [N]) out (mem = host/device). */
ats_status ats_level_get_rhs(ats_level *lvl, double *b, int mem);

/* y = (I + dt A) x in FP64 for a built level (x, y: [N], mem = host/device). */
ats_status ats_level_apply(ats_level *lvl, const double *x, double *y, int mem);

/* Cell coefficient model of the nonlinear equilibrium test (Sect. 4.2):
 * K[i] = K0 * E[i]^p for i < n, on the context's stream (not waited for).
 * E, K: device arrays of n FP64 values (may alias).  The lagged-coefficient
 * step builds the level operator from K(E^n).  E[i] <= 0 with a non-integer
 * p gives NaN, which the next operator build reports as ATS_ERR_BAD_INPUT.
 * Errors: ATS_ERR_INVALID_ARG (NULL context or arrays, n < 0), ATS_ERR_CUDA. */
ats_status ats_power_law_K(ats_context *ctx, int64_t n, const double *E, double K0, double p, double *K);

/* ---- solve (Sect. 3.3.4: diagonal-preconditioned CG) ---------------------- */
/* Solve (I + dt A) x = b for one built level.  rhs_or_null: NULL = the b of
 * ats_level_build_operator, else [N] replaces it for this call.  x_inout:
 * [N] initial guess in, solution out (non-leaf entries are kept).  opts may
 * be NULL (defaults).  stats may be NULL. */
ats_status ats_solve(ats_level *lvl, const double *rhs_or_null, double *x_inout,
                     const ats_solve_opts *opts, ats_solve_stats *stats);

/* ---- batched launch: many independent level solves ------------------------ */
/* Plan a batch over n built levels (one work list, one CUDA graph per poll
 * interval).  The levels must stay alive while the batch exists. */
ats_status ats_batch_create(ats_context *ctx, ats_level *const *levels, int n,
                            const ats_solve_opts *opts, ats_batch **out);
/* Solve all levels of the batch; x_inout[k] is solve k's [N_k] vector
 * (initial guess in, solution out), host or device per opts->mem. stats: [n]
 * or NULL.  Returns the first error status of any solve, else the first
 * warning (ATS_WARN_NEGATIVE), else ATS_OK. */
ats_status ats_batch_solve(ats_batch *batch, double *const *x_inout, ats_solve_stats *stats);
ats_status ats_batch_destroy(ats_batch *batch);
/* Build the operators of every level of the batch in one kernel launch
 * (same computation as ats_level_build_operator, Sect. 3.1-3.2): coefs[k]
 * describes level k.  Errors as ats_level_build_operator; ATS_ERR_BAD_INPUT
 * is reported per solve by the next ats_batch_solve. */
ats_status ats_batch_build_operators(ats_batch *batch, const ats_coef_desc *coefs);
/* Pipelining of host inputs: copy the host arrays of coefs (the next step's
 * operators) on a copy stream of the batch into its second staging set, and
 * return without waiting, so that the copies overlap a solve the caller runs
 * meanwhile (host<->device links carry both directions at once; use pinned
 * host memory, pageable copies do not overlap).  The next
 * ats_batch_build_operators with the same host arrays (same pointers) builds
 * from the copies instead of copying again; with other arrays the prefetch
 * is dropped.  The host arrays must not change until that build returns.
 * Device arrays are not copied (nothing to prefetch).  Errors: as
 * ats_batch_build_operators. */
ats_status ats_batch_prefetch_operators(ats_batch *batch, const ats_coef_desc *coefs);
/* One-shot form: create, solve and destroy. */
ats_status ats_batch_run(ats_context *ctx, ats_level *const *levels, int n, double *const *x_inout,
                         const ats_solve_opts *opts, ats_solve_stats *stats);
/* Kernel timing of the last ats_batch_solve, when profiling is on: CUDA
 * events around every tick kernel (also inside the replayed graphs), summed
 * per kernel, with the algorithmic bytes each moved (compulsory traffic of
 * the vectors and coefficients the kernel must read and write once).  A
 * profiled solve is scheduled like an unprofiled one (one poll interval
 * queued ahead, the events in two alternating sets; with use_graph = 2 it
 * runs as use_graph = 1, a conditional graph body holding no events), and
 * the times include every interval enqueued, the no-op one still queued when
 * the last solve finished included. */
typedef struct {
  double op_ms, op_bytes;    /* CG op kernel: p = z + beta p, q = A p, p.q        */
  double ref_ms, ref_bytes;  /* FP64 refinement residual kernel                  */
  double upd_ms, upd_bytes;  /* update kernel: e, z, dots; x += e after refinement */
  int launches;              /* tick-kernel launches                              */
  int ticks;                 /* ticks enqueued                                    */
  double res_ms, res_bytes;  /* resident solver launch (all its steps) and the    */
                             /* method's minimal traffic over them: 10 words per  */
                             /* cell and CG iteration, 5 FP64 words per cell and  */
                             /* refinement pass (most of it stays on chip)        */
  int res_launches;          /* resident-solver launches (with their hold kernels) */
  int res_solves;            /* solves taken by the resident solver               */
  double res_span_ms;        /* first resident solve's start to the last one's end */
  double res_longest_ms;     /* the longest resident solve                         */
  double res_occupancy;      /* CTA-time inside solves / (span x the launch's CTAs) */
  int res_longest;           /* index of the longest resident solve (-1: none)     */
  int res_grid;              /* CTAs of the resident launches                      */
  double res_end_ms[3];      /* end of the last big-cluster / cluster / one-CTA    */
                             /* solve, from the first resident solve's start       */
  int res_grids[3];          /* CTAs of the big- and middle-cluster, cluster and    */
                             /* one-CTA launches                                  */
} ats_kernel_stats;
ats_status ats_batch_set_profiling(ats_batch *batch, int on);
ats_status ats_batch_kernel_stats(const ats_batch *batch, ats_kernel_stats *out);

/* Autotuner of the batched launch (not in the paper, whose solver is one CPU
 * CG per level): times ats_batch_solve on the batch's own levels and
 * operators for every candidate and keeps the fastest, together with the
 * options the batch was created with.  The candidates: for a batch with
 * tick-path solves, every pair (work-item size tile_octs, poll interval
 * check_every); for a batch with resident solves, eight resident shapes
 * (res_threads, res_cluster, res_cta_octs, res_cluster_big):
 * (512, 4, 2048, 16) (512, 8, 2048, 16) (512, 8, 2048, none)
 * (256, 4, 2048, 16) (512, 4, 1024, 16) (512, 2, 2048, 16) (512, 4, 2048, 8)
 * (512, 16, 2048, none); each varies those options only.  tiles[n_tiles]: octs per work item, 0 = the
 * library's size rule (see ats_solve_opts.tile_octs), others
 * rounded up to a multiple of 32; NULL / 0 = {0, 128, 256, 384, 512}.
 * checks[n_checks]: ticks per CUDA graph and host poll; NULL / 0 = {8, 16,
 * 32}.  reps (>= 1): timed solves per candidate after one warm-up solve (the
 * fastest counts).  x_inout as in ats_batch_solve: with x0 = ATS_X0_GIVEN
 * every trial starts from the caller's x (kept in a scratch copy); on return
 * it holds the solution of one more solve with the chosen configuration, whose
 * plan the batch keeps.  Results are valid solutions for every candidate but
 * differ between tile sizes in the last bits (a solve's reduction order
 * follows its work items, a resident solve's its shape).  out: the choice,
 * its time and the time of the batch's original options (may be NULL).  Errors: ATS_ERR_INVALID_ARG for a
 * NULL batch or x, a negative tile or an unbuilt level; the first failing
 * solve's status otherwise (the batch then keeps its original plan). */
typedef struct {
  int tile_octs;     /* chosen octs per work item (0 = the size rule)      */
  int check_every;   /* chosen ticks per graph / poll interval             */
  double ms;         /* fastest solve time of the chosen configuration     */
  double ms_default; /* fastest solve time of the batch's original options */
  int candidates;    /* configurations timed                               */
  int res_threads;   /* chosen resident shape: threads per CTA, CTAs per   */
  int res_cluster;   /* cluster, one-CTA level limit (0 = the default)     */
  int res_cta_octs;
  ats_solve_opts chosen; /* the options the batch keeps                    */
} ats_tune_result;
ats_status ats_batch_autotune(ats_batch *batch, double *const *x_inout, const int *tiles, int n_tiles,
                              const int *checks, int n_checks, int reps, ats_tune_result *out);

/* ---- AMR hierarchy and the level substep driver (Sect. 2.2, 3.3) ----------- */
/* A hierarchy of levels l = 0 .. n_levels-1, dx halving per level; an oct at
 * level l+1 with oct coordinates (x, y, z) refines cell (x, y, z) of level l,
 * which must be marked non-leaf there.  Interface faces are derived from the
 * geometry: a leaf next to a refined cell of its level gets a Dirichlet face
 * with the restriction (mean of the 8 children) of that cell (coarse-to-fine,
 * Sect. 3.3.2, factor 1); a leaf next to a coarser leaf gets a Dirichlet face
 * with the coarse value (fine-to-coarse, Sect. 3.3.1, factor 2/3); faces on
 * the domain's outer boundary (no cell beyond them at any level) are
 * zero-flux walls unless wall_kind makes a side Dirichlet: then every leaf of
 * every level on that side gets a Dirichlet face holding wall_E in a ghost
 * cell one cell width of its level away (relation ATS_REL_SAME), with ghost
 * coefficient wall_K.  2:1 balance is required (ATS_ERR_INVALID_ARG
 * otherwise). */
typedef struct ats_hierarchy ats_hierarchy;
#define ATS_ORDER_FINE_FIRST 0   /* the paper: finer levels first, coarse value held at E^n   */
#define ATS_ORDER_COARSE_FIRST 1 /* coarse step first, fine ghosts linear in time over it   */
typedef struct {
  int n_levels;
  const ats_level_desc *levels; /* per level: n_oct, oct_xyz, leaf_mask, dx; face fields ignored */
  int order;                    /* ATS_ORDER_*                                                   */
  const int8_t *wall_kind;      /* [6] or NULL (all zero flux): per side -x,+x,-y,+y,-z,+z,     */
                                /* -1 zero flux or ATS_FACE_DIRICHLET                            */
  const double *wall_E;         /* [6] ghost value of each Dirichlet side (host)                 */
  const double *wall_K;         /* [6] ghost diffusion coefficient of each Dirichlet side, > 0   */
} ats_hierarchy_desc;
ats_status ats_hierarchy_create(ats_context *ctx, const ats_hierarchy_desc *desc, ats_hierarchy **out);
ats_status ats_hierarchy_destroy(ats_hierarchy *h);
/* Row of the coarse-to-fine faces (Sect. 3.3.1 - 3.3.2).  After every solve
 * of a level, the energy its fine-to-coarse faces moved into the coarser
 * cells is stored per coarse-to-fine face of the coarser level (energy per
 * unit coarse-cell volume, C (E_fine - E_coarse) / 8 with the 2/3 factor of
 * Sect. 3.3.1, summed over the fine steps: the Delta t-weighted mean flux of
 * Eq. mean_flux times the coarse step).  The coarser level's next solve uses
 * it and clears it:
 *   ATS_FACE_DIRICHLET  the restriction of the refined cell (default; the
 *                       stored energy is not used);
 *   ATS_FACE_NEUMANN    the stored energy as the imposed flux F: the total
 *                       energy of a closed hierarchy is conserved;
 *   ATS_FACE_ROBIN      alpha (Dirichlet part) + (1 - alpha) stored flux,
 *                       alpha in [0, 1].
 * Fine-to-coarse faces stay Dirichlet with the coarse value held at E^n.
 * Neumann and Robin need ATS_ORDER_FINE_FIRST (the stored energy must exist
 * before the coarse solve); ATS_ERR_INVALID_ARG otherwise or for a bad kind
 * or alpha.  Clears the stores. */
ats_status ats_hierarchy_set_interface(ats_hierarchy *h, int kind, double alpha);
/* The ats_level of one hierarchy level (owned by the hierarchy). */
ats_status ats_hierarchy_level(ats_hierarchy *h, int level, ats_level **out);
/* Set E and K ([N] of that level, host or device per mem); E is E^n. */
ats_status ats_hierarchy_set_state(ats_hierarchy *h, int level, const double *E, const double *K, int mem);
/* Radiation-matter mode (Sect. 2.1, flux-limited diffusion): per level the gas
 * density rho and temperature T ([N], host or device per mem) and the opacity
 * constant k0.  Once every level has them, each level solve first computes,
 * on its leaf cells from rho, T and E^n: rho kappa_R = k0 rho^2 / T (kappa_R
 * = kappa_P = k0 rho / T per unit mass), R = |grad E| / (rho kappa_R E) with
 * central (one-sided at a missing neighbour) differences over same-level
 * cells, the Levermore-Pomraning limiter lambda = (2 + R) / (6 + 3R + R^2),
 * K = c lambda / (rho kappa_R); and the linearised gas coupling sigma = dt
 * kappa_P rho c, mu = 4 a_R T^3 / (rho c_v), diagonal shift s = sigma / (1 +
 * sigma mu), source s a_R T^4; after the solve T = T + sigma (E - a_R T^4) /
 * (rho c_v (1 + sigma mu)).  Units c = a_R = c_v = 1.  K of the level is set
 * from the current E immediately. */
/* Power-law coefficient mode (the nonlinear equilibrium test, Sect. 4.2):
 * before every level solve, K = K0 E^a on the level's leaf cells from its
 * E^n (refined cells keep the mean of their children's K), held over the
 * step.  K0 > 0; a = 0 gives the constant K0.  Not with the radiation-matter
 * mode (ATS_ERR_INVALID_ARG). */
ats_status ats_hierarchy_set_power_law(ats_hierarchy *h, double K0, double a);
ats_status ats_hierarchy_set_fld(ats_hierarchy *h, int level, const double *rho, const double *T, double k0,
                                 int mem);
ats_status ats_hierarchy_get_temperature(ats_hierarchy *h, int level, double *T, int mem);
/* Copy E of a level out; refined cells carry the restriction of their children. */
ats_status ats_hierarchy_get_state(ats_hierarchy *h, int level, double *E, int mem);
/* Advance `level` by dt: with ATS_ORDER_FINE_FIRST the finer levels first take
 * two substeps of dt/2 each (recursively), then this level is solved; with
 * ATS_ORDER_COARSE_FIRST this level is solved first, then the finer levels
 * take their substeps with this level's value linear in time.  Every solve is
 * ats_solve with opts; stats accumulates iterations over all solves and keeps
 * the worst status and residuals.
 * opts->use_graph = 2: every level solve's tick loop is one graph launch and
 * no solve is waited for; the step's result records are read once at its end.
 * opts->use_graph = 3: the whole step -- restriction, ghost gathers, operator
 * builds, the level solves with their device loops, flux stores and the
 * copy of the result records -- is one graph: one launch and one host wait
 * per step.  A call takes the step as with 2 and then captures it when no
 * graph is held for the same level, dt and options, or when the hierarchy's
 * configuration (set_interface, set_fld, set_power_law) or the context's
 * device allocations changed since the capture; every other call replays the
 * graph.  The results are bitwise those of use_graph = 2.  A step whose
 * solves fail is not captured; a failure in a replayed step is reported as
 * with 2.  If the capture itself fails, the step has still been taken and the
 * call returns ATS_ERR_CUDA. */
ats_status ats_level_advance(ats_hierarchy *h, int level, double dt, const ats_solve_opts *opts,
                             ats_solve_stats *stats);
/* The step graph of use_graph = 3: *held = 1 while a captured step is kept;
 * *captures / *replays: steps captured / replayed since the hierarchy was
 * created.  Any output pointer may be NULL. */
ats_status ats_hierarchy_graph_stats(ats_hierarchy *h, int *held, int64_t *captures, int64_t *replays);
/* Host-only (no device): the interface faces the hierarchy derives for one
 * level.  Call with NULL arrays to get n_face first.  rel is ATS_REL_FINER
 * (src_cell = refined cell of the same level), ATS_REL_COARSER (src_cell =
 * leaf of level - 1) or, on a Dirichlet side of the domain, ATS_REL_SAME
 * (src_cell = the side, 0..5). */
ats_status ats_hierarchy_plan_faces(const ats_hierarchy_desc *desc, int level, int64_t *n_face,
                                    int32_t *face_cell, int8_t *face_dir, int8_t *face_rel,
                                    int32_t *src_cell);

/* ---- serving: continuous batching of level solves ---------------------------- */
/* A server owns a private context on `device` and a scheduler thread.  Any
 * thread submits level solves; the scheduler admits queued requests in arrival
 * order whenever a slot, enough work items and the device-memory budget allow
 * (an estimate of the request's resident bytes), builds them on the device and
 * joins them to the solves already in flight; every device tick advances all
 * resident solves one step (one CUDA graph of `check_every` ticks); finished
 * solves are copied back and their memory released.  A solve's arithmetic
 * involves no other solve: its result is the same alone and in any mix.
 * Requests whose estimate exceeds the whole budget fail with
 * ATS_ERR_OVER_BUDGET.  All ats_server_* calls are thread-safe. */
typedef struct ats_server ats_server;
typedef struct {
  ats_solve_opts solve; /* precision, max_iter, inner_rtol, check_every, tile (tol/stop per request) */
  int max_slots;        /* resident solves at most (0 = 1024)                                   */
  int max_items;        /* work-item pool (0 = 65536)                                          */
} ats_server_opts;
typedef struct {
  const ats_level_desc *level; /* host topology, copied at submit                          */
  const ats_coef_desc *coef;   /* host per-step values (mem = ATS_MEM_HOST), copied at submit */
  const double *x0;            /* host [N] initial guess or NULL (= E_old)                   */
  double tol;                  /* stopping tolerance of this request (0 = 1e-10)             */
  int stop_rule;               /* ATS_STOP_RESIDUAL or ATS_STOP_CERTIFIED                     */
} ats_request;
typedef struct {
  ats_status status;
  ats_solve_stats stats;
  double latency_us; /* submit to result ready                      */
  double queue_us;   /* submit to admission                          */
} ats_result;
typedef struct {
  uint64_t completed, queued;
  int64_t ticks;
  int peak_resident;
  size_t resident_bytes;
} ats_server_counters;
ats_status ats_server_create(int device, size_t mem_budget_bytes, const ats_server_opts *opts, ats_server **out);
/* Stops after the queued and resident solves are done, then frees everything. */
ats_status ats_server_destroy(ats_server *server);
ats_status ats_server_submit(ats_server *server, const ats_request *req, uint64_t *ticket);
/* Wait for a ticket (timeout_us < 0: forever); x_out: host [N] or NULL. */
ats_status ats_server_wait(ats_server *server, uint64_t ticket, int64_t timeout_us, double *x_out, ats_result *res);
ats_status ats_server_stats(ats_server *server, ats_server_counters *out);

/* ---- allocation-free solve ------------------------------------------------- */
/* The paper has no counterpart to this entry point: it is a service for
 * callers that cannot allocate device memory -- plug-ins confined to a memory
 * pool owned by their host program, and processes whose device memory belongs
 * to another runtime's allocator (a framework's caching allocator) that must
 * not be bypassed.  It solves one level like ats_solve with ATS_PREC_FP64 and
 * ATS_STOP_RESIDUAL, but calls no cudaMalloc or cudaFree: its CG vectors,
 * partial sums, work list and scalars live in one fixed device array inside
 * the library (about 19 MB, held by every GPU that loads the library until
 * the process exits).
 *
 * Arguments (all arrays are DEVICE pointers, FP64, read in stream order on
 * `stream`, a cudaStream_t or NULL for the default stream; K, xd, b and x
 * start on a 32-byte boundary, as every cudaMalloc block does):
 *   n_oct     octs of the level, 1 <= 8 n_oct <= ATS_NOALLOC_MAX_CELLS;
 *   nbr       [6 n_oct] oct neighbour table (ats_layout_neighbors gives it);
 *   K         [8 n_oct] cell K on leaf cells, a negative value on cells that
 *             are not unknowns of the level (their x is left as it is);
 *   xd        [8 n_oct] extra diagonal per cell (a coupling shift plus the
 *             diagonal terms of interface faces), or NULL for none;
 *   h         dt / dx^2 / 2, so an interior face has C = h (K_i + K_j);
 *   b         [8 n_oct] right-hand side;
 *   x         [8 n_oct] initial guess in, solution out;
 *   tol       ||r_j|| <= tol ||r_0||; max_iter: CG cap (<= 0: 20000).
 * The call is synchronous: it synchronises `stream` and polls the solve from
 * the host, so `stream` must not be under stream capture (a capturing stream
 * is rejected with ATS_ERR_INVALID_ARG before anything is enqueued).
 * Returns ATS_ERR_INVALID_ARG for sizes above ATS_NOALLOC_MAX_CELLS, a
 * misaligned array or a capturing stream.  The first call on each device
 * looks up the array's device address with that device current.  Every call
 * reuses the same array (its contents are the last call's; what must start
 * at zero is cleared by each call), so calls that overlap on the GPU race:
 * serialise them. */
#define ATS_NOALLOC_MAX_CELLS 262144
ats_status ats_solve_noalloc(int device, void *stream, int64_t n_oct, const int32_t *nbr,
                             const double *K, const double *xd, double h, const double *b,
                             double *x, double tol, int max_iter, ats_solve_stats *stats);

/* ---- misc ------------------------------------------------------------------ */
void ats_default_opts(ats_solve_opts *opts);
const char *ats_status_string(ats_status s);
const char *ats_last_error(void);
/* Host-only layout helper (no device needed): the oct neighbour table of a
 * level, nbr[6 o + dir] = neighbour oct index or -1. */
ats_status ats_layout_neighbors(const ats_level_desc *desc, int32_t *nbr);
/* Bounds-checked build (the library compiled with ATS_BOUNDS_CHECK=1): every
 * index a kernel gathers through (neighbour oct, interface record, face
 * descriptor, work item, work-list entry) is tested against the length of
 * the array it indexes; an index out of range is counted on the device and
 * its access skipped, so a corrupt table gives wrong results and a count,
 * never an access outside a buffer.  *count (host) receives the number of
 * such indices met on `device` since the previous call, which resets it;
 * the call synchronises the device.  The default build has no checks and
 * sets *count = -1.  Errors: ATS_ERR_INVALID_ARG (null count), ATS_ERR_CUDA. */
ats_status ats_bounds_violations(int device, long long *count);
/* Self-test of the whole-GPU resident solver's grid barrier (the wait every
 * CTA of its cooperative launch passes between CG steps): `ctas` CTAs (0 =
 * one per SM) wait for ctas + extra arrivals.  extra = 0: every wait ends
 * normally; extra > 0: no wait can end normally, and each must give up by
 * itself after its bounded number of polls (about 0.2 s) and raise the
 * solver's give-up flag -- the path that ends a solve with ATS_ERR_TIMEOUT
 * instead of hanging the GPU.  *n_normal / *n_gave_up count the CTAs by how
 * their wait ended, *ms is the launch's device time.  Errors:
 * ATS_ERR_INVALID_ARG (null outputs, negative counts, more CTAs than SMs),
 * ATS_ERR_CUDA (also when the flag disagrees with the waits). */
ats_status ats_grid_barrier_selftest(int device, int ctas, int extra, int *n_normal, int *n_gave_up, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* ATS_H */
