// Internal declarations of the sm_103a level-solve library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ats.h"

namespace ats {

constexpr int kThreads = 128;          // threads per CTA of the tick kernels (one oct each)
constexpr int kNumPartials = 4;        // FP64 partial sums per work item

// Phases of the per-solve state machine advanced by each device "tick"
// (one op kernel + one update kernel).
enum Phase : int {
  kRefine = 0,  // FP64 true residual r = b - A (x + e), z = D^-1 r
  kInner = 1,   // one CG iteration on the correction e
  kDone = 2,
};

// Static description of one solve, read-only on the device during a run.
struct SolveDev {
  const int32_t *nbr;   // [n_oct*6]
  const int32_t *xrec;  // [n_oct] record of the diagonal extras or -1
  const double *K64;    // [N]  K on leaves, -1 on non-leaf cells
  const void *KT;       // [N]  K in the bulk precision (alias of K64 in FP64 mode)
  const double *xd64;   // [n_rec*8] s_i + sum of interface w C
  const void *xdT;      // same in the bulk precision
  const double *b64;    // [N]
  double *x64;          // [N]  the FP64 iterate
  void *e;              // [N]  correction (bulk precision)
  void *z;              // [N]  preconditioned residual (bulk precision)
  void *p0;             // [N]  search direction, ping
  void *p1;             // [N]  search direction, pong
  const double *C64;    // [n_oct][3][8] h (K_i + K_j) of each cell's +x, +y, +z face (0 off the leaves)
  const double *cn_base;  // Crank-Nicolson: E^n; the copy-out returns 2 x - E^n (else null)
  void *q;              // [N]  (I + dt A) p of the current direction (k_op)
  void *dg;             // [N]  diagonal D = 1 + xd + sum C (k_ref; 1 off the leaves)
  double h;             // dt / dx^2 / 2, so an interior C = h (K_i + K_j)
  double tol;
  double inner_rtol;
  double final_safety;  // inner target = max(inner_rtol r, final_safety * tol * ref)
  int32_t n_oct;
  int32_t item_begin;
  int32_t n_items;
  int32_t stop_rule;
  int32_t max_iter;
  int32_t max_refine;
  int32_t inner_max;    // iterations per inner pass before a restart
  int32_t n_xd;         // records in xd64 / xdT (bounds of xrec)
};

// Per-solve scalars (device).  Double-buffered by tick parity: the kernels of
// a tick read S[parity] and the CTA that owns a solve's first work item
// writes the solve's next state into S[parity ^ 1]; a finished solve's last
// state also goes to a separate final array.
struct SolveScalars {
  int32_t phase;
  int32_t first;        // the next CG iteration starts a new direction (p = z)
  int32_t pcur;         // which p buffer holds the current direction
  int32_t iters;
  int32_t inner_iters;
  int32_t refines;
  int32_t status;
  int32_t final_pass;   // the next refinement pass ends the solve
  int32_t ticks;
  float inner_t2;        // inner_target^2 in FP32 (the FP32 convergence test)
  double rz;            // r.z of the newest residual that is not yet a direction
  double r0;
  double inner_target;
  double rnorm;         // last FP64 true residual norm
  double xnorm;
  double maxchg;
};

struct WorkItem {
  int32_t solve;
  int32_t oct_begin;
  int32_t n_oct;
  int32_t pad;
};

// Active work lists, one per (parity, phase): k_op walks the CG-phase list,
// k_ref the refinement-phase list and k_upd both; the last CTA of each solve
// that stays active appends that solve's items to the next parity's list of
// its new phase; the last CTA of k_upd flips the parity.
struct TickCtl {
  int32_t parity;
  int32_t count[2][2];  // [parity][phase]
  int32_t cta_done;
};

// ---- launchers (kernels.cu) ----
struct CoefArgs {
  int64_t n_oct;
  const uint8_t *leaf;
  const int32_t *frec;      // [n_oct] face record or -1
  const int32_t *rec_face;  // [n_rec*48] descriptor id per (cell, dir) or -1
  const int32_t *xrec;      // [n_oct] diagonal-extra record or -1
  const int8_t *face_kind;
  const int8_t *face_rel;
  const double *face_alpha;
  const double *face_K;
  const double *face_E;
  const double *face_F;
  const double *K;
  const double *E_old;
  const double *s;
  const double *src;
  double h;
  double *K64;
  float *K32;
  double *xd64;
  float *xd32;
  double *b64;
  int *err_flag;
  const int32_t *nbr;   // for the face coefficients
  double *C64;          // [n_oct][3][8] written by the face-coefficient pass
  double src_scale;     // weight of src and face F (1; 1/2 for a Crank-Nicolson half step)
  int64_t n_rec;        // face records (bounds of frec)
  int64_t n_xd;         // diagonal-extra records (bounds of xrec)
  int64_t n_face;       // interface descriptors (bounds of rec_face entries)
};
// K, diagonal extras, b and the FP64 face coefficients C64, one thread per cell.
cudaError_t launch_coef_build(const CoefArgs &a, cudaStream_t st);
// One launch for many levels after zeroing the levels' error flags (flags:
// device array of device pointers): block b of kCoefThreads threads builds
// cells of level blk_level[b], starting at (b - blk_first[level]) * kCoefThreads.
constexpr int kCoefThreads = 256;
cudaError_t launch_coef_build_batch(const CoefArgs *args, const int32_t *blk_level, const int32_t *blk_first,
                                    int n_blocks, int n, int *const *flags, cudaStream_t st);
// FP64 face coefficients C64[(3 o + a) 8 + c] = h (K_i + K_j) between cell i =
// 8 o + c and its +a neighbour j when both are leaves (K >= 0), else 0.
cudaError_t launch_face_coef(int64_t n_oct, const int32_t *nbr, const double *K64, double h, double *C64,
                             cudaStream_t st);
cudaError_t launch_gather_flags(const int *const *flags, int n, int *out, cudaStream_t st);

// Device state of a planned batch, passed by value to the tick kernels.
// Cells processed, counted when profiling: [0] k_op CG items after the first
// iteration of an inner solve, [1] k_ref, [2] k_upd CG items, [3] x += e at
// the end of an inner solve, [4] k_op CG items in a first iteration.
constexpr int kCellCounters = 5;

struct TickArgs {
  const SolveDev *solves;
  SolveScalars *sbuf;       // [2][n_solves]
  SolveScalars *final_sc;   // [n_solves] state of every finished solve
  const WorkItem *items;
  int32_t *lists;           // [2 parities][2 phases][n_items]
  int n_items;
  int n_solves;
  TickCtl *ctl;
  double *p_op;             // [n_items][kNumPartials] partials of k_op / k_ref
  double *p_upd;            // [2][n_items][kNumPartials] partials of k_upd by parity
  int *n_active;
  unsigned long long *cells;  // [kCellCounters] cells per kernel / phase, or null
};

// One tick = k_op (CG items) and k_ref (refinement residual of the solves in
// their refinement phase), which touch disjoint solves, then k_upd (all items;
// a solve that leaves its inner solve folds x += e there).  With fj->aux set,
// k_ref is launched first on fj->aux, forked from st, then k_op on st, and
// both join before k_upd, so the two overlap; otherwise all three run on st.
// tt (null, or timing): after each kernel an event is recorded on a side
// stream that waits for that kernel and that nothing else waits for, so the
// timestamps stay off the kernels' dependency chain; ev[0] after k_op, ev[1]
// after k_ref, ev[2] after k_upd.  `capture` says whether st is being
// captured.
struct TickStreams {
  cudaStream_t aux;
  cudaEvent_t fork, join;  // created with cudaEventDisableTiming
};
struct TickTiming {
  cudaStream_t side;
  cudaEvent_t mark;  // ordering marker, cudaEventDisableTiming
  cudaEvent_t *ev;   // [kTickEvents] timing events of this tick
};
constexpr int kTickEvents = 3;
// Record `ev` on tt->side once the work queued so far on `from` is done.
cudaError_t record_after(const TickTiming &tt, cudaEvent_t ev, cudaStream_t from, bool capture);
// grids: [0] k_op, [1] k_ref, [2] k_upd (each kernel strides over its list).
cudaError_t launch_tick(bool fp64, bool paper, const TickArgs &a, const int grids[3], cudaStream_t st,
                        const TickStreams *fj, const TickTiming *tt, bool capture);
// Resident grid of each tick kernel on `device` (its CTAs per SM under its
// register and shared-memory use, times the SM count), in launch_tick order.
void tick_grids(bool fp64, bool paper, int device, int grids[3]);

// Resident solver (kernels.cu): whole solves inside one launch.  The
// launch's clusters take the solves of cq[0, n_cq), then its CTAs take
// single-CTA solves from tq[0, n_tq); *cq_head / *tq_head are the next
// positions of the two queues (zero before the launch; several launches of a
// plan share the CTA queue and its head).  A finished solve writes its state
// to final_sc.  With cells set, the cells processed per step kind are added
// as the tick kernels count them (kCellCounters).
struct ResArgs {
  const SolveDev *solves;
  SolveScalars *final_sc;
  const int32_t *cq;
  const int32_t *tq;
  int n_cq, n_tq, n_solves;
  int cg_scalars;  // FP32 bulk: 0 = step decisions in FP32 from the rounded totals, 1 = in FP64
  int q_recur;     // FP32 bulk: 1 = q = (I + dt A) z + beta q_prev (no barrier), 0 = q = (I + dt A) p
  int *cq_head;
  int *tq_head;
  unsigned long long *cells;
  unsigned long long *t_solve;  // [n_solves][2] %globaltimer at a solve's start and end (profiling), or null
  int cap;                      // shared-memory form: octs per CTA kept in shared memory (0: none)
  // whole-GPU form (launch_resident_grid): every CTA of one cooperative
  // launch works on gq[0], gq[1], ... in turn; gbar[0] = the arrivals at
  // its grid barriers so far (zeroed before the launch; gbar[1] unused),
  // gpart = [2][grid + 1][3] (hi, lo) pairs: per buffer, each CTA's partial
  // sums (the last row unused); *gerr set when a barrier wait gave up
  const int32_t *gq;
  int n_gq;
  unsigned *gbar;
  float *gpart;
  int *gerr;
  int g_expect;  // arrivals a grid barrier waits for (0: every CTA of the launch)
  // FP32-bulk kernels: where each solve's result goes (x, or 2 x' - E^n for
  // Crank-Nicolson), written by the solve's own CTAs when it ends; null for
  // the solves whose result k_final writes.  neg[s] is set when a written
  // value is negative.
  double *const *x_out;
  int *neg;
};
// One resident launch on st of the FP64 solver (CG state in global memory):
// clusters of `cluster` CTAs of `threads` threads (256 or 512), `grid` CTAs
// in all (a multiple of `cluster`) when the cluster queue is not empty, else
// `grid` single CTAs.  fp64 = false: cudaErrorInvalidValue (the FP32-bulk
// solver is launch_resident_smem).
cudaError_t launch_resident(bool fp64, int threads, int cluster, int grid, const ResArgs &a, cudaStream_t st,
                            bool cta_only = false);
// Clusters of that shape resident at once on the current device (0: none).
int resident_max_clusters(bool fp64, int threads, int cluster);
// CTAs of the single-CTA kernel resident per SM.
int resident_cta_blocks(bool fp64, int threads);
// The resident solver of FP32-bulk solves with each CTA's K, z, p in shared
// memory: a.cap octs per CTA (resident_smem_cap gives the largest that fits;
// 0 keeps every array in global memory, with the same arithmetic), one CTA
// per SM; the same queue and grid conventions as launch_resident.
// cta_only: the single-CTA kernel only (the CTA queue), e.g. on the SMs a
// concurrent cluster launch leaves free.  priority: the launch's scheduling
// priority (cudaLaunchAttributePriority; lower numbers first, 0 = default).
cudaError_t launch_resident_smem(int threads, int cluster, int grid, const ResArgs &a, cudaStream_t st,
                                 bool cta_only = false, int priority = 0);
int resident_smem_clusters(int threads, int cluster, int cap);
int resident_smem_cap(int threads, int device);
// The whole-GPU form of the shared-memory solver (FP32 bulk, 512-thread CTAs
// only): one cooperative launch of `grid` CTAs (at most resident_grid_ctas,
// 0 for other CTA sizes) solves gq[0, n_gq) one
// level at a time, each level split into `grid` contiguous runs; sums and
// steps go through global memory and a grid barrier whose waits end after a
// bounded number of polls (then *gerr is set and the solve ends with
// ATS_ERR_TIMEOUT).
cudaError_t launch_resident_grid(int threads, int grid, const ResArgs &a, cudaStream_t st);
// A one-thread kernel on st that returns after about ns nanoseconds (bounded
// by a fixed number of clock reads): the work queued behind it on st starts
// that much later.
cudaError_t launch_hold(unsigned long long ns, cudaStream_t st);
int resident_grid_ctas(int threads, int device);
// Octs per CTA up to which the shared-memory solver keeps all six CG arrays
// (K, z, p, D, q, e) of a CTA's run in shared memory.
int resident_six_cap();
// One grid barrier of that form alone (cooperative launch of `grid` CTAs of 32
// threads) waiting for a.g_expect arrivals: out[cta] = 1 when its wait ended
// normally, 0 when it gave up (and *a.gerr = 1).  a.gbar, a.gerr zeroed first.
cudaError_t launch_grid_barrier_probe(int grid, const ResArgs &a, int *out, cudaStream_t st);

// Start of a solve: e = 0 on every cell of every item, and x64 = src[solve]
// where src (device array of device pointers) is non-null for that solve.
cudaError_t launch_init(bool fp64, const SolveDev *solves, const WorkItem *items, int n_items,
                        const double *const *src, int grid, cudaStream_t st);
// End of a solve: dst[solve] = x64 (2 x64 - E^n for Crank-Nicolson) where
// dst[solve] is non-null; neg[solve] |= 1 (neg may be null) when a value of
// the result is negative.
cudaError_t launch_final(const SolveDev *solves, const WorkItem *items, int n_items,
                         double *const *dst, int *neg, int grid, cudaStream_t st);

cudaError_t launch_apply64(const SolveDev *solve_host_copy, const double *x, double *y,
                           cudaStream_t st);

int tick_blocks_per_sm(bool fp64, bool paper);

// Flux-limited diffusion coefficients (K, s, src from rho, T, E^n) and the
// gas temperature update after a solve (kernels.cu).
cudaError_t launch_fld_coef(int64_t n_oct, const int32_t *nbr, const uint8_t *leaf, const double *E, const double *rho,
                            const double *T, double dx, double dt, double k0, double *K, double *s, double *src,
                            cudaStream_t st);
cudaError_t launch_fld_temperature(int64_t N, const uint8_t *leaf, const double *E, const double *rho, double *T,
                                   double dt, double k0, cudaStream_t st);
// Serving support (runtime.cpp): the device descriptor of one solve of a
// built level with the given options and work-item range (allocates the
// level's CG vectors of that precision if needed), the work-item tiling, and
// level accessors.
ats_status solve_dev_for(ats_level *L, const ats_solve_opts &o, bool fp64, int item_begin, int n_items,
                         SolveDev *out);
int tile_for(int64_t n_oct, int requested, int grid);
ats_solve_opts normalized_opts(const ats_solve_opts *in);
double *level_x64(ats_level *L);
int64_t level_cells(const ats_level *L);
// Admission of new solves between ticks: append each new solve's items to the
// current tick's refinement list and count it active (kernels.cu).
cudaError_t launch_admit(const TickArgs &a, const int32_t *slots, int n_new, cudaStream_t st);
// Device topology of a level (runtime.cpp): neighbour table and leaf masks.
const int32_t *level_nbr(const ats_level *L);
const uint8_t *level_leaf(const ats_level *L);

// AMR coupling kernels (restriction of children, ghost gather of interface faces).
// Stored interface energy (Sect. 3.3.2): for each face f of the coarse level
// with fine faces gather4[4 f .. 4 f + 3] (fine-to-coarse faces of the finer
// level, -1 = none), store[f] += sum_g C_g (x[fcell[g]] - fE[g]) / 8 with
// C_g = (2/3) h_f (K[fcell[g]] + fK[g]) -- the energy per unit coarse-cell
// volume the fine solve just moved into the coarse cell.
cudaError_t launch_flux_store(int n_face, const int32_t *gather4, const int32_t *fcell, const double *x,
                              const double *K, const double *fK, const double *fE, double h_f, double *store,
                              cudaStream_t st);
// Result record of a solve enqueued without a host wait (device memory):
// its final state, its error flag (bad input) and the tick intervals its
// device-driven loop ran.
struct DeferredRec {
  SolveScalars sc;
  int flag;
  int chunks;
  int neg;  // a negative energy in the result
  int pad;
};
// Enqueue one solve of L on the context stream with the whole tick loop as
// one graph (use_graph = 2 is forced): x_dev is the device initial guess and
// solution, d_rec (device) receives the result.  Nothing waits on the host.
// check_every / max_ticks: the loop's interval and tick bound, for
// deferred_result.  capture: the context stream is under stream capture; the
// level's plan, its device loop and its start state must then be resident
// from an earlier run of the same solve (else ATS_ERR_INVALID_ARG, nothing
// enqueued), and the loop is added to the captured graph.
ats_status level_solve_deferred(ats_level *L, double *x_dev, const ats_solve_opts *opts, DeferredRec *d_rec,
                                int *check_every, int64_t *max_ticks, bool capture = false);
// Status and statistics of a deferred solve from a host copy of its record.
ats_status deferred_result(const DeferredRec &r, int check_every, int64_t max_ticks, ats_solve_stats *out);
// Add to `graph` (standalone, or the graph of a stream under capture), after
// deps[0 .. n_deps), the device-side tick loop: a WHILE conditional node whose
// body runs `interval` (one poll interval of ticks, cloned into the body) and
// then a condition kernel that counts the intervals in *chunks and continues
// while *n_active > 0 and fewer than max_chunks intervals have run.  The
// handle's default value 1 is assigned at every launch of the graph, so the
// body runs once before the first test.  node_out: the conditional node.
cudaError_t add_while_loop(cudaGraph_t graph, const cudaGraphNode_t *deps, size_t n_deps, cudaGraph_t interval,
                           const int *n_active, int *chunks, int max_chunks, cudaGraphNode_t *node_out);
// out[i] = 2 x[i] - E[i] (the Crank-Nicolson step from its backward-Euler half step).
cudaError_t launch_cn_extrapolate(int64_t N, const double *x, const double *E, double *out, cudaStream_t st);
// E^n of a Crank-Nicolson operator build of L (null for backward Euler).
const double *level_cn_base(const ats_level *L);
// Replace the face rows (kind, alpha: host arrays of the level's n_face).
ats_status level_set_face_rows(ats_level *L, const int8_t *kind, const double *alpha);
cudaError_t launch_restrict(int n, const int32_t *cell, const int32_t *child, const double *Ef, const double *Kf,
                            double *Ec, double *Kc, cudaStream_t st);
cudaError_t launch_gather_faces(int n_face, const int8_t *src_rel, const int32_t *src_cell, const double *E_same,
                                const double *K_same, const double *Ec_old, const double *Ec_new,
                                const double *K_coarse, double theta, double *fE, double *fK, const double *wall, cudaStream_t st);

// ---- layout (layout.cpp) ----
struct Layout {
  int64_t n_oct = 0;
  std::vector<int32_t> nbr;       // [n_oct*6]
  std::vector<int32_t> frec;      // [n_oct]
  std::vector<int32_t> rec_face;  // [n_rec*48]
  int64_t n_rec = 0;
};
// Returns "" on success or an error message.
std::string build_layout(const ats_level_desc &d, Layout &out);
// ats_level_create with a layout already built on the host (runtime.cpp).
ats_status level_create_with_layout(ats_context *ctx, const ats_level_desc *desc, const Layout &lay, ats_level **out);

void set_error(const std::string &msg);
// The status of the exception being handled (call only in a catch handler):
// ATS_ERR_OOM for std::bad_alloc, else ATS_ERR_INVALID_ARG; sets the message.
ats_status abi_exception() noexcept;

// Context services for other translation units (runtime.cpp).
ats_status ctx_alloc(ats_context *ctx, size_t bytes, void **out);
void ctx_free(ats_context *ctx, void *p);
cudaStream_t ctx_stream(const ats_context *ctx);
// Counter bumped by every allocation, free and host upload of solve-plan state
// in the context: equal values before and after mean nothing a captured graph
// refers to has moved or been rewritten from the host.
uint64_t ctx_epoch(const ats_context *ctx);
int ctx_device(const ats_context *ctx);

// Interface faces of one level of a hierarchy (hierarchy.cpp): leaf faces whose
// neighbour is a refined cell of the same level (rel = ATS_REL_FINER,
// src_level = l) or a coarser leaf (rel = ATS_REL_COARSER, src_level = l - 1);
// faces on the domain boundary are zero-flux walls (no entry).
struct LevelFaces {
  std::vector<int32_t> cell;
  std::vector<int8_t> dir;
  std::vector<int8_t> rel;
  std::vector<int32_t> src_cell;   // cell index in the source level
  std::vector<int32_t> restrict_cell;   // refined cells of this level ...
  std::vector<int32_t> restrict_child;  // ... and their child oct at level l + 1
};
// wall_kind: [6] or NULL (see ats_hierarchy_desc).
std::string plan_level_faces(const ats_level_desc *levels, int n_levels, int l, LevelFaces &out,
                             const int8_t *wall_kind);
// K = K0 E^a on the leaf cells of a level (all cells when leaf is NULL; bit c
// of leaf[o] marks cell 8 o + c); the other cells keep K.
cudaError_t launch_power_law_K(int64_t n_cell, const uint8_t *leaf, const double *E, double K0, double a,
                               double *K, cudaStream_t st);

}  // namespace ats
