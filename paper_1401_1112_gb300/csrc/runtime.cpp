// Host runtime of the level-solve library: context, levels, operator build,
// solve plans (single and batched), CUDA-graph replay and convergence polling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "ats_internal.h"

namespace ats {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

// Called in the catch handler of an entry point: the status of the exception
// being handled (no C++ exception leaves the library).
ats_status abi_exception() noexcept {
  auto note = [](const char *m) noexcept {
    try {
      g_last_error = m;
    } catch (...) {
    }
  };
  try {
    throw;
  } catch (const std::bad_alloc &) {
    note("out of host memory");
    return ATS_ERR_OOM;
  } catch (...) {
    note("internal error");
    return ATS_ERR_INVALID_ARG;
  }
}

}  // namespace ats

using namespace ats;

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------

struct ats_context {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::unordered_map<void *, size_t> allocs;
  // bumped by every allocation, free and host upload of solve-plan state, so
  // that a graph recorded over plans of this context can tell whether what it
  // captured is still in place
  uint64_t epoch = 0;
};

struct Plan;

struct ats_level {
  ats_context *ctx = nullptr;
  int64_t n_oct = 0, N = 0, n_face = 0, n_rec = 0;
  double dx = 0.0;
  // topology
  int32_t *nbr = nullptr, *frec = nullptr, *rec_face = nullptr, *xrec_dense = nullptr;
  uint8_t *leaf = nullptr;
  int8_t *fkind = nullptr, *frel = nullptr;
  double *falpha = nullptr;
  // operator
  bool built = false;
  bool dense_xd = false;
  double dt = 0.0;
  double *K64 = nullptr, *xd64 = nullptr, *b64 = nullptr;
  double *C64 = nullptr;  // [n_oct][3][8] FP64 face coefficients (+x, +y, +z faces)
  float *K32 = nullptr, *xd32 = nullptr;
  int64_t xd_cap = 0;  // records allocated in xd64/xd32
  int *err_flag = nullptr;
  // host-pointer staging of per-step arrays
  double *stage_cell = nullptr;  // 4 x N : K, E, s, src
  double *stage_face = nullptr;  // 3 x n_face : K, E, F
  // solve vectors: the FP64 iterate, and one set of CG vectors per bulk
  // precision ([0] FP64, [1] FP32), allocated on first use
  double *x64 = nullptr;
  void *e[2] = {nullptr, nullptr}, *z[2] = {nullptr, nullptr};
  void *p0[2] = {nullptr, nullptr}, *p1[2] = {nullptr, nullptr};
  void *q[2] = {nullptr, nullptr}, *dg[2] = {nullptr, nullptr};
  double *rhs_save = nullptr;  // b when a solve overrides it
  const double *E_dev = nullptr;  // device E^n of the last operator build (x0 = E^n)
  const double *cn_base = nullptr;  // E^n when that build was a Crank-Nicolson half step
  Plan *solo = nullptr;        // cached single-solve plan
};

namespace {

struct StatusError {
  ats_status code;
};

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess) {                                                             \
      set_error(std::string("CUDA error: ") + cudaGetErrorString(_e) + " at " #expr);     \
      return ATS_ERR_CUDA;                                                               \
    }                                                                                    \
  } while (0)

ats_status dev_alloc(ats_context *ctx, size_t bytes, void **out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->budget && ctx->used + bytes > ctx->budget) {
    set_error("device memory budget exceeded");
    return ATS_ERR_OVER_BUDGET;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    return ATS_ERR_OOM;
  }
  ctx->allocs[p] = bytes;
  ctx->used += bytes;
  ++ctx->epoch;
  *out = p;
  return ATS_OK;
}

template <typename P>
ats_status dev_alloc_t(ats_context *ctx, size_t count, P **out) {
  void *p = nullptr;
  ats_status s = dev_alloc(ctx, count * sizeof(P), &p);
  *out = (P *)p;
  return s;
}

void dev_free(ats_context *ctx, void *p) {
  if (!p) return;
  ++ctx->epoch;
  auto it = ctx->allocs.find(p);
  if (it != ctx->allocs.end()) {
    ctx->used -= it->second;
    ctx->allocs.erase(it);
  }
  cudaFree(p);
}

cudaMemcpyKind kind_of(int mem, bool to_device) {
  if (mem == ATS_MEM_DEVICE) return cudaMemcpyDeviceToDevice;
  return to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
}

}  // namespace

namespace ats {
ats_status ctx_alloc(ats_context *ctx, size_t bytes, void **out) { return dev_alloc(ctx, bytes, out); }
void ctx_free(ats_context *ctx, void *p) { dev_free(ctx, p); }
cudaStream_t ctx_stream(const ats_context *ctx) { return ctx->stream; }
uint64_t ctx_epoch(const ats_context *ctx) { return ctx->epoch; }
const int32_t *level_nbr(const ats_level *L) { return L->nbr; }
double *level_x64(ats_level *L) { return L->x64; }
const double *level_cn_base(const ats_level *L) { return L->cn_base; }
int64_t level_cells(const ats_level *L) { return L->N; }
const uint8_t *level_leaf(const ats_level *L) { return L->leaf; }
ats_status level_set_face_rows(ats_level *L, const int8_t *kind, const double *alpha) {
  if (!L) return ATS_ERR_INVALID_ARG;
  if (L->n_face == 0) return ATS_OK;
  cudaStream_t st = L->ctx->stream;
  CUDA_TRY(cudaMemcpyAsync(L->fkind, kind, L->n_face, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(L->falpha, alpha, sizeof(double) * L->n_face, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return ATS_OK;
}
int ctx_device(const ats_context *ctx) { return ctx->device; }
}  // namespace ats

// ---------------------------------------------------------------------------
// solve plan: work list, per-solve device descriptors, graph
// ---------------------------------------------------------------------------

struct Plan {
  ats_context *ctx = nullptr;
  std::vector<ats_level *> levels;
  ats_solve_opts opts{};
  bool fp64 = true, paper = false;
  int n = 0, n_items = 0, grid = 1;
  int grids[3] = {1, 1, 1};  // tick kernels: k_op, k_ref, k_upd
  SolveDev *d_solves = nullptr;
  SolveScalars *d_sc = nullptr;     // [2][n] double-buffered scalars
  SolveScalars *d_final = nullptr;  // [n] state of finished solves
  WorkItem *d_items = nullptr;
  double *d_partials = nullptr;     // [n_items][4] op partials, then [2][n_items][4] update partials
  TickArgs targs{};
  int *d_active = nullptr;
  unsigned long long *d_cells = nullptr;
  int32_t *d_lists = nullptr;      // [2 parities][2 phases][n_items] active work lists
  int32_t *d_ident = nullptr;      // [n_items] 0..n_items-1 (the full list)
  TickCtl *d_ctl = nullptr;
  int **d_flag_ptrs = nullptr;     // [n] the levels' error flags
  int *d_flags = nullptr;          // [n] gathered flags, then [n] negative-result flags
  const double **d_src = nullptr;  // [n] device pointers for x copy-in (or null)
  double **d_dst = nullptr;        // [n] device pointers for x copy-out by k_final (or null)
  double **d_rdst = nullptr;       // [n] ... by the FP32-bulk resident kernels at a solve's end (or null)
  double *d_xstage = nullptr;      // [sum N] host x staged on the device (host-memory solves)
  int *h_active = nullptr;         // pinned [2]: one per poll slot
  std::vector<SolveDev> h_solves;
  std::vector<SolveScalars> h_sc;
  cudaGraphExec_t exec = nullptr;          // one interval of ticks
  cudaGraphExec_t exec_prof[2] = {nullptr, nullptr};  // the same with the timing events of set 0 / 1
  // use_graph = 2: the whole tick loop as one graph (WHILE node over one
  // interval of ticks); d_loop counts the intervals run
  cudaGraphExec_t loop_exec = nullptr;
  cudaGraph_t loop_ticks = nullptr;  // the loop's body: one interval of ticks
  int *d_loop = nullptr;
  int loop_max = 0;
  // start-of-run state kept on the device (the solves' initial scalars, the
  // active count, the tick control block), and the host image last uploaded;
  // the x pointers last uploaded to d_src / d_dst.  A run whose start state
  // and pointers are already resident copies them device to device only
  unsigned char *d_init = nullptr;
  std::vector<unsigned char> h_init;
  std::vector<const double *> h_src;
  std::vector<double *> h_dst, h_rdst;
  // host-memory solves: the last host x pointers seen, whether the device
  // can write each directly (pinned), and the pointers copy_runs copies back
  // (null where the resident kernel wrote the host array itself)
  std::vector<double *> h_xhost, h_xdev;
  std::vector<char> h_xdirect;
  std::vector<double *> h_copyback;
  bool profiling = false;
  // two sets (by poll slot) of: chunk start, then kTickEvents per tick of a
  // chunk, so that one interval runs while the other's events are read
  std::vector<cudaEvent_t> evs;
  cudaEvent_t poll_ev[2] = {nullptr, nullptr};
  TickStreams fj{nullptr, nullptr, nullptr};  // k_ref's stream, fork / join events
  cudaStream_t side = nullptr;                // timing events (profiling)
  cudaEvent_t mark = nullptr;
  int slot = 0;
  double op_ms = 0.0, ref_ms = 0.0, upd_ms = 0.0, op_bytes = 0.0, ref_bytes = 0.0, upd_bytes = 0.0;
  int launches = 0;
  int ticks = 0;
  // resident solver (whole solves in one launch): per solve 0 = tick path,
  // 1 = a cluster of res_cluster CTAs, 2 = one CTA, 3 = a cluster of
  // res_cluster_big CTAs; the queues hold the big-cluster solves, the
  // cluster solves, then the CTA solves, each by estimated work, largest first
  std::vector<int8_t> mode;
  int n_bq = 0, n_cq = 0, n_tq = 0, n_tick = 0, n_tick_items = 0;
  int n_mq = 0;  // mode 5: the middle clusters (res_cluster_mid CTAs)
  // mode 4: the whole-GPU form (one cooperative launch of res_grid_all CTAs
  // takes these solves one after another); its barrier, partial sums and
  // give-up flag
  int n_gq = 0, res_grid_all = 0;
  // the split of the device's CTA slots between the three resident launches:
  // clusters of each size that fit at once, the slots, and whether the split
  // follows measured per-class SM-time (after a completed run) or the
  // estimates
  int res_clA = 0, res_clB = 0, res_clM = 0, res_slots = 0;
  bool res_split_measured = false;
  // measured duration (ns) of each resident solve in the last completed run;
  // the queues are ordered by it (largest first) once every solve of a queue
  // has one, uploaded again at the next start (queue_dirty)
  std::vector<double> res_meas;
  bool queue_dirty = false;
  std::vector<int32_t> h_queue;  // the queue order last uploaded
  unsigned *d_gbar = nullptr;
  float *d_gpart = nullptr;
  int *d_gerr = nullptr;
  int res_threads = 512, res_cluster = 8, res_cluster_big = 16, res_grid = 0, res_grid_big = 0;
  int res_cluster_mid = 8, res_grid_mid = 0;
  bool res_smem = false;  // K, z, p of each CTA's octs in shared memory (FP32 bulk)
  int res_cap = 0;        // octs per CTA kept in shared memory
  int res_fill = 0;       // single CTAs launched beside the clusters on the SMs they leave
  int32_t *d_queue = nullptr;   // [n_bq + n_mq + n_cq + n_tq + n_gq]
  int *d_heads = nullptr;       // [4] next position of each queue: big, cluster, CTA, middle
  cudaStream_t aux2 = nullptr, aux3 = nullptr;  // the third and fourth concurrent resident launches
  cudaEvent_t join2 = nullptr, join3 = nullptr;
  cudaEvent_t res_ev[2] = {nullptr, nullptr};
  double res_ms = 0.0, res_bytes = 0.0;
  int res_launches = 0;
  unsigned long long *d_tsolve = nullptr;  // [n][2] per-solve start / end of the resident solves
  double res_span_ms = 0.0, res_longest_ms = 0.0, res_occupancy = 0.0, res_end_ms[3] = {0.0, 0.0, 0.0};
  int res_longest = -1;
};

struct ats_batch {
  Plan *plan = nullptr;
  // host inputs of the batched build, staged in one device buffer per kind
  // (cell arrays K, E_old, s, src; face arrays K, E, F) so that runs of levels
  // whose host arrays are contiguous cost one copy; two sets, used in turn,
  // so that the next step's inputs can be copied while a solve runs
  double *stage_cell[2][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
  double *stage_face[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int cur_set = 0;  // the set the operators were last built from
  // ats_batch_prefetch_operators: copies on their own stream into the other set
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copied = nullptr, released = nullptr;
  bool prefetched = false;
  std::vector<const double *> pf_ptrs;  // the prefetched host arrays, 7 per level
  // batched operator build
  CoefArgs *d_args = nullptr;
  int32_t *d_blk_level = nullptr;  // batched build: level of each block
  int32_t *d_blk_first = nullptr;  // [n + 1] first block of each level
  int n_blocks = 0;
  std::vector<CoefArgs> h_args;  // last uploaded arguments
};

namespace {

void fill_defaults(ats_solve_opts *o) {
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->stop_rule = ATS_STOP_RESIDUAL;
  o->precision = ATS_PREC_FP64;
  o->max_iter = 20000;
  o->max_refine = 40;
  o->inner_rtol = 1e-6;
  o->tile_octs = 0;
  o->check_every = 16;
  o->use_graph = 0;
  o->mem = ATS_MEM_HOST;
  o->sched = ATS_SCHED_AUTO;
  o->res_threads = 0;
  o->res_cluster = 0;
  o->res_cta_octs = 0;
  o->res_max_octs = 0;
  o->cg_scalars = 0;
  o->res_state = 0;
}

ats_solve_opts normalize(const ats_solve_opts *in) {
  ats_solve_opts o;
  fill_defaults(&o);
  if (!in) return o;
  o = *in;
  if (!(o.tol > 0.0)) o.tol = 1e-10;
  if (o.max_iter <= 0) o.max_iter = 20000;
  if (o.max_refine <= 0) o.max_refine = 40;
  if (!(o.inner_rtol > 0.0)) o.inner_rtol = 1e-6;
  if (o.check_every <= 0) o.check_every = 16;
  // 3 (a hierarchy step as one graph) is 2 for a solve on its own
  if (o.use_graph > 2) o.use_graph = 2;
  return o;
}

// Octs per work item (one CTA of kThreads threads, one oct per thread and
// pass).  A level gets about one item per CTA of the stencil kernel's
// resident grid `grid` -- a large solve keeps every SM busy with as few
// per-item reductions as possible -- rounded up to a multiple of 128 octs and
// kept within 256..1024: smaller levels take 256, and their items spread over
// the CTAs beside the other solves of a batch.
int choose_tile(int64_t n_oct, int requested, int grid) {
  if (requested > 0) return std::max(32, (requested + 31) / 32 * 32);
  const int64_t g = std::max(1, grid);
  const int64_t per_cta = (n_oct + g - 1) / g;
  const int64_t t = (per_cta + 127) / 128 * 128;
  return (int)std::min<int64_t>(8 * kThreads, std::max<int64_t>(2 * kThreads, t));
}

// Copy per-level host arrays into (h2d) or out of one device buffer at the
// levels' offsets off[k]: levels whose host arrays follow each other in
// memory form one run and cost one copy.  Levels with a null host pointer are
// skipped.
ats_status copy_runs(cudaStream_t st, bool h2d, double *dev, const int64_t *off, int n, double *const *host) {
  int k = 0;
  while (k < n) {
    if (!host[k]) {
      ++k;
      continue;
    }
    int e = k + 1;
    while (e < n && host[e] && host[e] == host[e - 1] + (off[e] - off[e - 1])) ++e;
    const size_t bytes = sizeof(double) * (size_t)(off[e] - off[k]);
    if (bytes) {
      CUDA_TRY(h2d ? cudaMemcpyAsync(dev + off[k], host[k], bytes, cudaMemcpyHostToDevice, st)
                   : cudaMemcpyAsync(host[k], dev + off[k], bytes, cudaMemcpyDeviceToHost, st));
    }
    k = e;
  }
  return ATS_OK;
}

ats_status ensure_vectors(ats_level *L, bool fp64) {
  const int k = fp64 ? 0 : 1;
  ats_context *ctx = L->ctx;
  const size_t es = fp64 ? sizeof(double) : sizeof(float);
  ats_status s;
  if (!L->x64 && (s = dev_alloc_t(ctx, L->N, &L->x64)) != ATS_OK) return s;
  if (!L->e[k] && (s = dev_alloc(ctx, es * L->N, &L->e[k])) != ATS_OK) return s;
  if (!L->z[k] && (s = dev_alloc(ctx, es * L->N, &L->z[k])) != ATS_OK) return s;
  if (!L->p0[k] && (s = dev_alloc(ctx, es * L->N, &L->p0[k])) != ATS_OK) return s;
  if (!L->p1[k] && (s = dev_alloc(ctx, es * L->N, &L->p1[k])) != ATS_OK) return s;
  if (!L->q[k] && (s = dev_alloc(ctx, es * L->N, &L->q[k])) != ATS_OK) return s;
  if (!L->dg[k] && (s = dev_alloc(ctx, es * L->N, &L->dg[k])) != ATS_OK) return s;
  return ATS_OK;
}

void plan_free(Plan *P) {
  if (!P) return;
  ats_context *ctx = P->ctx;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  for (auto g : P->exec_prof)
    if (g) cudaGraphExecDestroy(g);
  if (P->loop_exec) cudaGraphExecDestroy(P->loop_exec);
  dev_free(ctx, P->d_loop);
  for (auto e : P->evs) cudaEventDestroy(e);
  for (auto e : P->poll_ev)
    if (e) cudaEventDestroy(e);
  if (P->fj.fork) cudaEventDestroy(P->fj.fork);
  if (P->fj.join) cudaEventDestroy(P->fj.join);
  if (P->fj.aux) cudaStreamDestroy(P->fj.aux);
  if (P->mark) cudaEventDestroy(P->mark);
  if (P->side) cudaStreamDestroy(P->side);
  dev_free(ctx, P->d_solves);
  dev_free(ctx, P->d_sc);
  dev_free(ctx, P->d_final);
  dev_free(ctx, P->d_items);
  dev_free(ctx, P->d_partials);
  dev_free(ctx, P->d_active);
  dev_free(ctx, P->d_cells);
  dev_free(ctx, P->d_lists);
  dev_free(ctx, P->d_ident);
  dev_free(ctx, P->d_ctl);
  dev_free(ctx, P->d_flag_ptrs);
  dev_free(ctx, P->d_flags);
  dev_free(ctx, P->d_src);
  dev_free(ctx, P->d_dst);
  dev_free(ctx, P->d_rdst);
  dev_free(ctx, P->d_xstage);
  dev_free(ctx, P->d_queue);
  dev_free(ctx, P->d_heads);
  dev_free(ctx, P->d_gbar);
  dev_free(ctx, P->d_gpart);
  dev_free(ctx, P->d_gerr);
  dev_free(ctx, P->d_tsolve);
  dev_free(ctx, P->d_init);
  if (P->loop_ticks) cudaGraphDestroy(P->loop_ticks);
  if (P->join2) cudaEventDestroy(P->join2);
  if (P->aux2) cudaStreamDestroy(P->aux2);
  if (P->join3) cudaEventDestroy(P->join3);
  if (P->aux3) cudaStreamDestroy(P->aux3);
  for (auto e : P->res_ev)
    if (e) cudaEventDestroy(e);
  if (P->h_active) cudaFreeHost(P->h_active);
  delete P;
}

// Estimated work of a level solve, to order the resident queues (largest
// first): octs times an iteration estimate, the square root of the stiffness
// 1 + 8 h (h = dt / (2 dx^2), K ~ 1) capped by four times the oct count's
// cube root (about twice the level's width in cells).
double est_work(const ats_level *L) {
  const double h = 0.5 * L->dt / (L->dx * L->dx);
  const double o = (double)L->n_oct;
  return o * std::min(std::sqrt(1.0 + 8.0 * h), 4.0 * std::cbrt(o));
}

// Upload the resident queues of P in work order: big-cluster solves, cluster
// solves, CTA solves.
ats_status plan_upload_queues(Plan *P) {
  std::vector<int32_t> bq, mq, cq, tq, gq;
  for (int k = 0; k < P->n; ++k) {
    if (P->mode[k] == 3) bq.push_back(k);
    if (P->mode[k] == 5) mq.push_back(k);
    if (P->mode[k] == 1) cq.push_back(k);
    if (P->mode[k] == 2) tq.push_back(k);
    if (P->mode[k] == 4) gq.push_back(k);
  }
  auto by_work = [&](std::vector<int32_t> &q) {
    std::vector<double> w(P->n, 0.0);
    bool meas = !P->res_meas.empty();
    for (int32_t k : q) meas = meas && P->res_meas[k] > 0.0;
    for (int32_t k : q) w[k] = meas ? P->res_meas[k] : est_work(P->levels[k]);
    std::stable_sort(q.begin(), q.end(), [&](int32_t a, int32_t b) { return w[a] > w[b]; });
  };
  by_work(bq);
  by_work(mq);
  by_work(cq);
  by_work(tq);
  bq.insert(bq.end(), mq.begin(), mq.end());
  bq.insert(bq.end(), cq.begin(), cq.end());
  bq.insert(bq.end(), tq.begin(), tq.end());
  bq.insert(bq.end(), gq.begin(), gq.end());
  if (bq == P->h_queue) return ATS_OK;  // already on the device
  P->h_queue = bq;
  if (!bq.empty())
    CUDA_TRY(cudaMemcpyAsync(P->d_queue, P->h_queue.data(), sizeof(int32_t) * bq.size(), cudaMemcpyHostToDevice,
                             P->ctx->stream));
  ++P->ctx->epoch;
  return ATS_OK;
}

// The CTA slots of the device, shared by the resident launches in proportion
// to their queues' work w[0] (big clusters), w[1] (middle clusters), w[2]
// (clusters), w[3] (single CTAs): the single CTAs get at least their share
// (so the largest of them start at once), the big and middle clusters theirs
// in whole clusters, and the smallest cluster class present every remaining
// whole cluster; what is left runs single CTAs beside them.  A cluster that
// has emptied its queue goes on with single-CTA solves.
void plan_split(Plan *P, const double (&w)[4]) {
  const int slots = P->res_slots;
  const int size[3] = {P->res_cluster_big, P->res_cluster_mid, P->res_cluster};
  const int lim[3] = {P->res_clA, P->res_clM, P->res_clB};
  const int cnt[3] = {P->n_bq, P->n_mq, P->n_cq};
  const double wsum = std::max(1e-300, w[0] + w[1] + w[2] + w[3]);
  const int c_min = P->n_tq > 0 ? std::max(1, (int)std::ceil(slots * w[3] / wsum)) : 0;
  int k[3] = {0, 0, 0};
  int last = -1;  // the smallest cluster class present takes the remainder
  for (int q = 0; q < 3; ++q)
    if (cnt[q] > 0) last = q;
  int used = c_min;
  for (int q = 0; q < 3; ++q) {
    if (cnt[q] <= 0 || q == last) continue;
    k[q] = std::max(1, std::min(lim[q], (int)std::lround(slots * w[q] / wsum / size[q])));
    used += k[q] * size[q];
  }
  if (last >= 0) k[last] = std::max(1, std::min(lim[last], (slots - used) / size[last]));
  auto total = [&] { return k[0] * size[0] + k[1] * size[1] + k[2] * size[2] + c_min; };
  while (total() > slots) {
    int q_max = -1;
    for (int q = 0; q < 3; ++q)
      if (k[q] > 1 && (q_max < 0 || k[q] * size[q] > k[q_max] * size[q_max])) q_max = q;
    if (q_max < 0) break;
    --k[q_max];
  }
  P->res_grid_big = k[0] * size[0];
  P->res_grid_mid = k[1] * size[1];
  const bool clusters = P->n_bq + P->n_mq + P->n_cq > 0;
  P->res_grid = clusters ? k[2] * size[2] : slots;
  P->res_fill = (P->n_tq > 0 && clusters)
                    ? std::max(0, slots - P->res_grid - P->res_grid_big - P->res_grid_mid)
                    : 0;
}

// CTAs of each solve's group, by mode
int group_ctas(const Plan *P, int mode) {
  switch (mode) {
    case 1: return P->res_cluster;
    case 3: return P->res_cluster_big;
    case 4: return P->res_grid_all;
    case 5: return P->res_cluster_mid;
    default: return 1;
  }
}

// After a completed run: the SM-time each class of resident solves took
// (each solve's duration times its group's CTAs), from the solves' start and
// end stamps; the next run splits the slots by it and orders each queue by
// the measured durations.  Which group and layout a solve takes does not
// change, so neither do its results.
void plan_adapt_split(Plan *P, const std::vector<unsigned long long> &ts) {
  double w[4] = {0.0, 0.0, 0.0, 0.0};
  int present = 0, measured = 0;
  const int cls[4] = {P->n_bq, P->n_mq, P->n_cq, P->n_tq};
  for (int q = 0; q < 4; ++q) present += cls[q] > 0;
  if (present < 1 || P->n < 2) return;
  auto class_of = [](int m) { return m == 3 ? 0 : m == 5 ? 1 : m == 1 ? 2 : m == 2 ? 3 : -1; };
  for (int k = 0; k < P->n; ++k) {
    const int q = class_of(P->mode[k]);
    if (q < 0 || ts[2 * k + 1] <= ts[2 * k]) continue;
    w[q] += (double)(ts[2 * k + 1] - ts[2 * k]) * group_ctas(P, P->mode[k]);
  }
  for (int q = 0; q < 4; ++q) measured += (cls[q] > 0 && w[q] > 0.0);
  // each queue in the order of the measured durations (largest first)
  P->res_meas.assign(P->n, 0.0);
  for (int k = 0; k < P->n; ++k)
    if (class_of(P->mode[k]) >= 0 && ts[2 * k + 1] > ts[2 * k]) P->res_meas[k] = (double)(ts[2 * k + 1] - ts[2 * k]);
  P->queue_dirty = true;
  if (measured != present) return;
  plan_split(P, w);
  P->res_split_measured = true;
}

ats_status plan_create(ats_context *ctx, ats_level *const *levels, int n, const ats_solve_opts *opts_in,
                       Plan **out) {
  *out = nullptr;
  if (!ctx || !levels || n <= 0) {
    set_error("plan: bad arguments");
    return ATS_ERR_INVALID_ARG;
  }
  ats_solve_opts o = normalize(opts_in);
  if (o.precision != ATS_PREC_FP64 && o.precision != ATS_PREC_MIXED) {
    set_error("bad precision");
    return ATS_ERR_INVALID_ARG;
  }
  if (o.stop_rule < 0 || o.stop_rule > 2) {
    set_error("bad stop_rule");
    return ATS_ERR_INVALID_ARG;
  }
  if (o.x0 != ATS_X0_GIVEN && o.x0 != ATS_X0_E_OLD) {
    set_error("bad x0");
    return ATS_ERR_INVALID_ARG;
  }
  if (o.sched < ATS_SCHED_AUTO || o.sched > ATS_SCHED_GRID || (o.res_threads != 0 && o.res_threads != 256 &&
      o.res_threads != 512) || o.res_cluster < 0 || o.res_cluster > 16 || o.res_max_octs < 0 || o.res_state < 0 ||
      o.res_state > 1 || o.res_cluster_big > 16 || o.res_big_work < 0 || o.res_cluster_mid > 16 || o.cg_form < 0 ||
      o.cg_form > 2) {
    set_error("bad resident-solver options (sched 0..3, res_threads 0/256/512, res_cluster, res_cluster_mid and "
              "res_cluster_big up to 16, res_state 0/1, cg_form 0..2)");
    return ATS_ERR_INVALID_ARG;
  }
  CUDA_TRY(cudaSetDevice(ctx->device));
  Plan *P = new (std::nothrow) Plan();
  if (!P) return ATS_ERR_OOM;
  P->ctx = ctx;
  P->opts = o;
  P->fp64 = (o.precision == ATS_PREC_FP64);
  P->paper = (o.stop_rule == ATS_STOP_PAPER);
  P->n = n;
  std::vector<WorkItem> items;
  tick_grids(P->fp64, P->paper, ctx->device, P->grids);  // the item size follows the stencil kernel's grid
  P->h_solves.resize(n);
  P->h_sc.resize(n);
  ats_status s;
  for (int k = 0; k < n; ++k) {
    ats_level *L = levels[k];
    if (!L || L->ctx != ctx) {
      plan_free(P);
      set_error("plan: level is null or from another context");
      return ATS_ERR_INVALID_ARG;
    }
    if (!L->built) {
      plan_free(P);
      set_error("plan: level operator not built");
      return ATS_ERR_INVALID_ARG;
    }
    if ((s = ensure_vectors(L, P->fp64)) != ATS_OK) {
      plan_free(P);
      return s;
    }
    P->levels.push_back(L);
    SolveDev &sd = P->h_solves[k];
    std::memset(&sd, 0, sizeof(sd));
    sd.nbr = L->nbr;
    sd.xrec = L->dense_xd ? L->xrec_dense : L->frec;
    sd.n_xd = (int32_t)(L->dense_xd ? L->n_oct : L->n_rec);
    sd.K64 = L->K64;
    sd.C64 = L->C64;
    sd.KT = P->fp64 ? (const void *)L->K64 : (const void *)L->K32;
    sd.xd64 = L->xd64;
    sd.xdT = P->fp64 ? (const void *)L->xd64 : (const void *)L->xd32;
    sd.b64 = L->b64;
    sd.x64 = L->x64;
    sd.cn_base = L->cn_base;
    const int vk = P->fp64 ? 0 : 1;
    sd.e = L->e[vk];
    sd.z = L->z[vk];
    sd.p0 = L->p0[vk];
    sd.p1 = L->p1[vk];
    sd.q = L->q[vk];
    sd.dg = L->dg[vk];
    sd.h = 0.5 * L->dt / (L->dx * L->dx);
    sd.tol = o.tol;
    sd.inner_rtol = P->fp64 ? 0.0 : o.inner_rtol;
    sd.final_safety = P->fp64 ? 1.0 : 0.5;
    sd.n_oct = (int32_t)L->n_oct;
    sd.stop_rule = o.stop_rule;
    sd.max_iter = o.max_iter;
    sd.max_refine = o.max_refine;
    sd.inner_max = P->fp64 ? o.max_iter : 4000;
    const int tile = choose_tile(L->n_oct, o.tile_octs, P->grids[0]);
    sd.item_begin = (int32_t)items.size();
    for (int64_t b = 0; b < L->n_oct; b += tile) {
      WorkItem w;
      w.solve = k;
      w.oct_begin = (int32_t)b;
      w.n_oct = (int32_t)std::min<int64_t>(tile, L->n_oct - b);
      w.pad = 0;
      items.push_back(w);
    }
    sd.n_items = (int32_t)items.size() - sd.item_begin;
    SolveScalars &sc = P->h_sc[k];
    std::memset(&sc, 0, sizeof(sc));
    sc.phase = kRefine;
    sc.status = ATS_OK;
  }
  P->n_items = (int)items.size();
  // resident or tick path per solve, by a rule on the level and the options
  // alone (a level then runs the same arithmetic alone and in any batch)
  P->res_threads = o.res_threads > 0 ? o.res_threads : (P->fp64 ? 256 : 512);
  P->res_cluster = o.res_cluster > 0 ? o.res_cluster : 4;
  P->res_cluster_big = o.res_cluster_big == 0 ? 16 : (o.res_cluster_big < 0 ? 0 : o.res_cluster_big);
  P->res_cluster_mid = o.res_cluster_mid == 0 ? 8 : (o.res_cluster_mid < 0 ? 0 : o.res_cluster_mid);
  // a middle size only between the two others
  if (P->res_cluster_mid <= P->res_cluster || (P->res_cluster_big > 0 && P->res_cluster_mid >= P->res_cluster_big))
    P->res_cluster_mid = 0;
  {
    const bool res_ok = o.sched != ATS_SCHED_TICK && o.stop_rule != ATS_STOP_PAPER;
    const int64_t cta_octs = o.res_cta_octs == 0 ? 2048 : o.res_cta_octs;
    // default limit: mixed precision 16384 octs (the shared-memory form
    // beats a whole-GPU tick loop up to about there for one solve alone);
    // FP64 (the global-memory form) 2048
    const int64_t max_octs = o.sched == ATS_SCHED_RESIDENT
                                 ? INT64_MAX
                                 : (o.res_max_octs > 0 ? o.res_max_octs : (P->fp64 ? 2048 : 16384));
    const double big_work = o.res_big_work > 0 ? (double)o.res_big_work : HUGE_VAL;  // 0: no work rule
    // FP32 bulk: the shared-memory kernel, its CG state in shared memory
    // (res_state 0, where the device has room) or in global memory (cap 0);
    // FP64: the global-memory kernel
    P->res_smem = !P->fp64;
    if (P->res_smem) {
      P->res_cap = o.res_state == 0 ? resident_smem_cap(P->res_threads, ctx->device) : 0;
      if (P->res_cap < 0) P->res_cap = 0;
    }
    auto max_clusters = [&](int cl) {
      if (cl <= 0) return 0;
      return P->res_smem ? resident_smem_clusters(P->res_threads, cl, P->res_cap)
                         : resident_max_clusters(P->fp64, P->res_threads, cl);
    };
    // levels above the limit: the whole-GPU form (FP32 bulk, each CTA's run
    // in shared memory) when asked for, and with ATS_SCHED_AUTO when the runs
    // on its CTAs keep all six arrays in shared memory; else the tick path
    const bool grid_ok = (o.sched == ATS_SCHED_GRID || o.sched == ATS_SCHED_AUTO) && P->res_smem && P->res_cap > 0;
    const int grid_all = grid_ok ? resident_grid_ctas(P->res_threads, ctx->device) : 0;
    const int64_t grid_auto_octs = (int64_t)grid_all * std::min(P->res_cap, resident_six_cap());
    P->mode.assign(n, 0);
    for (int k = 0; k < n; ++k) {
      const int64_t no = P->levels[k]->n_oct;
      if (!res_ok) continue;
      if (no > max_octs) {
        if (grid_all > 0 && (o.sched == ATS_SCHED_GRID || no <= grid_auto_octs)) P->mode[k] = 4;
        continue;
      }
      // a level whose runs on res_cluster CTAs would not fit their shared
      // memory takes the smallest larger cluster whose runs fit (the middle
      // size, else the big one); the work rule sends it to the big clusters
      const auto fits = [&](int cl) { return P->res_cap <= 0 || no <= (int64_t)cl * P->res_cap; };
      if (no <= cta_octs) P->mode[k] = 2;
      else if (P->res_cluster_big > 0 && est_work(P->levels[k]) > big_work) P->mode[k] = 3;
      else if (fits(P->res_cluster)) P->mode[k] = 1;
      else if (P->res_cluster_mid > 0 && fits(P->res_cluster_mid)) P->mode[k] = 5;
      else P->mode[k] = P->res_cluster_big > 0 ? 3 : 1;
    }
    int clA = 0, clM = 0, clB = 0;  // clusters of each size that fit the device at once
    bool anyA = false, anyM = false, anyB = false;
    for (int k = 0; k < n; ++k) {
      anyA = anyA || P->mode[k] == 3;
      anyM = anyM || P->mode[k] == 5;
      anyB = anyB || P->mode[k] == 1;
    }
    if (anyA) clA = max_clusters(P->res_cluster_big);
    if (anyM || (anyA && clA <= 0)) clM = max_clusters(P->res_cluster_mid);
    if (anyB || anyM || anyA) clB = max_clusters(P->res_cluster);
    // a cluster shape that does not fit this device: its levels take the
    // smaller clusters, or the tick path
    for (int k = 0; k < n; ++k) {
      if (P->mode[k] == 3 && clA <= 0) P->mode[k] = P->res_cluster_mid > 0 ? 5 : 1;
      if (P->mode[k] == 5 && clM <= 0) P->mode[k] = 1;
      if (P->mode[k] == 1 && clB <= 0) P->mode[k] = 0;
    }
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < n; ++k) {
      P->n_bq += P->mode[k] == 3;
      P->n_mq += P->mode[k] == 5;
      P->n_cq += P->mode[k] == 1;
      P->n_tq += P->mode[k] == 2;
      P->n_tick += P->mode[k] == 0;
      P->n_gq += P->mode[k] == 4;
      if (P->mode[k] == 0 || P->mode[k] == 4) continue;
      const int q = P->mode[k] == 3 ? 0 : P->mode[k] == 5 ? 1 : P->mode[k] == 1 ? 2 : 3;
      w[q] += est_work(P->levels[k]);
    }
    // the first split follows the estimated work; after each completed run,
    // the measured SM-time of each class (plan_adapt_split)
    const int cta_per_sm = P->res_smem ? 1 : std::max(1, resident_cta_blocks(P->fp64, P->res_threads));
    P->res_slots = cta_per_sm * ctx->num_sms;
    P->res_clA = clA;
    P->res_clM = clM;
    P->res_clB = clB;
    plan_split(P, w);
    if (P->n_gq > 0) P->res_grid_all = grid_all;
  }
  const int bps = tick_blocks_per_sm(P->fp64, P->paper);
  P->grid = std::max(1, std::min(P->n_items, bps * ctx->num_sms));
  for (int k = 0; k < 3; ++k) P->grids[k] = std::max(1, std::min(P->n_items, P->grids[k]));
  if ((s = dev_alloc_t(ctx, n, &P->d_solves)) != ATS_OK ||
      (s = dev_alloc_t(ctx, 2 * (size_t)n, &P->d_sc)) != ATS_OK ||
      (s = dev_alloc_t(ctx, n, &P->d_final)) != ATS_OK ||
      (s = dev_alloc_t(ctx, P->n_items, &P->d_items)) != ATS_OK ||
      (s = dev_alloc_t(ctx, 3 * (size_t)P->n_items * kNumPartials, &P->d_partials)) != ATS_OK ||
      (s = dev_alloc_t(ctx, 1, &P->d_active)) != ATS_OK ||
      (s = dev_alloc_t(ctx, 2 * kCellCounters, &P->d_cells)) != ATS_OK ||
      (s = dev_alloc_t(ctx, std::max(1, P->n_bq + P->n_mq + P->n_cq + P->n_tq + P->n_gq), &P->d_queue)) != ATS_OK ||
      (P->n_bq + P->n_mq + P->n_cq + P->n_tq + P->n_gq > 0 &&
       (s = dev_alloc_t(ctx, 2 * (size_t)n, &P->d_tsolve)) != ATS_OK) ||
      (P->n_gq > 0 && (s = dev_alloc_t(ctx, 2, &P->d_gbar)) != ATS_OK) ||
      (P->n_gq > 0 && (s = dev_alloc_t(ctx, 12 * ((size_t)P->res_grid_all + 1), &P->d_gpart)) != ATS_OK) ||
      (P->n_gq > 0 && (s = dev_alloc_t(ctx, 1, &P->d_gerr)) != ATS_OK) ||
      (s = dev_alloc_t(ctx, 4, &P->d_heads)) != ATS_OK ||
      (s = dev_alloc_t(ctx, 4 * (size_t)P->n_items, &P->d_lists)) != ATS_OK ||
      (s = dev_alloc_t(ctx, (size_t)P->n_items, &P->d_ident)) != ATS_OK ||
      (s = dev_alloc_t(ctx, 1, &P->d_ctl)) != ATS_OK ||
      (s = dev_alloc_t(ctx, n, &P->d_flag_ptrs)) != ATS_OK ||
      (s = dev_alloc_t(ctx, 2 * (size_t)n, &P->d_flags)) != ATS_OK ||
      (s = dev_alloc_t(ctx, n, &P->d_src)) != ATS_OK ||
      (s = dev_alloc_t(ctx, n, &P->d_dst)) != ATS_OK || (s = dev_alloc_t(ctx, n, &P->d_rdst)) != ATS_OK) {
    plan_free(P);
    return s;
  }
  if (cudaMallocHost(&P->h_active, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    plan_free(P);
    set_error("cudaMallocHost failed");
    return ATS_ERR_OOM;
  }
  cudaStream_t st = ctx->stream;
  CUDA_TRY(cudaMemcpyAsync(P->d_solves, P->h_solves.data(), sizeof(SolveDev) * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(P->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, st));
  {
    // the tick path's first list: the work items of the tick-path solves
    std::vector<int32_t> ident;
    for (int i = 0; i < P->n_items; ++i)
      if (P->mode[items[i].solve] == 0) ident.push_back(i);
    P->n_tick_items = (int)ident.size();
    if (!ident.empty())
      CUDA_TRY(cudaMemcpyAsync(P->d_ident, ident.data(), sizeof(int32_t) * ident.size(), cudaMemcpyHostToDevice, st));
    if ((s = plan_upload_queues(P)) != ATS_OK) {
      plan_free(P);
      return s;
    }
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  {
    std::vector<int *> fp(n);
    for (int k = 0; k < n; ++k) fp[k] = P->levels[k]->err_flag;
    CUDA_TRY(cudaMemcpyAsync(P->d_flag_ptrs, fp.data(), sizeof(int *) * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  {
    TickArgs &t = P->targs;
    t.solves = P->d_solves;
    t.sbuf = P->d_sc;
    t.final_sc = P->d_final;
    t.items = P->d_items;
    t.lists = P->d_lists;
    t.n_items = P->n_items;
    t.n_solves = n;
    t.ctl = P->d_ctl;
    t.p_op = P->d_partials;
    t.p_upd = P->d_partials + (size_t)P->n_items * kNumPartials;
    t.n_active = P->d_active;
    t.cells = P->d_cells;
  }
  CUDA_TRY(cudaEventCreateWithFlags(&P->poll_ev[0], cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&P->poll_ev[1], cudaEventDisableTiming));
  CUDA_TRY(cudaStreamCreateWithFlags(&P->fj.aux, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&P->fj.fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&P->fj.join, cudaEventDisableTiming));
  CUDA_TRY(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&P->mark, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreate(&P->res_ev[0]));
  CUDA_TRY(cudaEventCreate(&P->res_ev[1]));
  CUDA_TRY(cudaStreamCreateWithFlags(&P->aux2, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&P->join2, cudaEventDisableTiming));
  CUDA_TRY(cudaStreamCreateWithFlags(&P->aux3, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&P->join3, cudaEventDisableTiming));
  CUDA_TRY(cudaStreamSynchronize(st));
  *out = P;
  return ATS_OK;
}

// Enqueue the resident launches of P's solves (after plan_begin): the big
// clusters on the context stream, the clusters and the single CTAs on the
// plan's two side streams, all three forked from and joined back into the
// context stream (profiling: between the two timing events).
ats_status plan_launch_resident(Plan *P, bool prof, int *neg) {
  if (P->n_bq + P->n_mq + P->n_cq + P->n_tq + P->n_gq == 0) return ATS_OK;
  cudaStream_t st = P->ctx->stream;
  ResArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  ra.solves = P->d_solves;
  ra.final_sc = P->d_final;
  ra.tq = P->d_queue + P->n_bq + P->n_mq + P->n_cq;
  ra.n_tq = P->n_tq;
  ra.tq_head = P->d_heads + 2;
  ra.n_solves = P->n;
  ra.cg_scalars = P->opts.cg_scalars ? 1 : 0;
  ra.x_out = P->res_smem ? P->d_rdst : nullptr;
  ra.neg = neg;
  ra.q_recur = P->opts.cg_form == 1 ? 0 : 1;
  ra.cells = prof ? P->d_cells + kCellCounters : nullptr;
  // every resident solve stamps its start and end (the split of the next run
  // follows them; profiling reads the timeline)
  if (P->d_tsolve) CUDA_TRY(cudaMemsetAsync(P->d_tsolve, 0, 2 * sizeof(unsigned long long) * P->n, st));
  ra.t_solve = P->d_tsolve;
  ra.cap = P->res_cap;
  CUDA_TRY(cudaMemsetAsync(P->d_heads, 0, 4 * sizeof(int), st));
  if (prof) CUDA_TRY(cudaEventRecord(P->res_ev[0], st));
  // the larger clusters first: they need that many free SMs of one GPC at
  // once, so their CTAs are scheduled ahead of the smaller groups' (launch
  // priorities from the device's greatest down, single CTAs at the default)
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
    cudaGetLastError();
    prio_least = prio_greatest = 0;
  }
  auto launch = [&](int cluster, int grid, const ResArgs &a, cudaStream_t s2, bool cta_only) -> cudaError_t {
    const int rank = cta_only                                                   ? 3
                     : (P->res_cluster_big > 0 && cluster >= P->res_cluster_big) ? 0
                     : (P->res_cluster_mid > 0 && cluster >= P->res_cluster_mid) ? 1
                                                                                 : 2;
    const int prio = cta_only ? 0 : std::min(prio_least, prio_greatest + rank);
    return P->res_smem ? launch_resident_smem(P->res_threads, cluster, grid, a, s2, cta_only, prio)
                       : launch_resident(P->fp64, P->res_threads, cluster, grid, a, s2, cta_only);
  };
  // the launches in order: big clusters, clusters, single CTAs (the first
  // one on st, the others on the side streams, forked before the first)
  struct L {
    int cluster, grid;
    ResArgs a;
    bool cta_only;
  };
  std::vector<L> ls;
  const bool part = P->n_bq + P->n_mq + P->n_cq + P->n_tq > 0;  // any solve for the cluster / CTA launches
  if (P->n_bq > 0) {
    ResArgs a = ra;
    a.cq = P->d_queue;
    a.n_cq = P->n_bq;
    a.cq_head = P->d_heads;
    ls.push_back({P->res_cluster_big, P->res_grid_big, a, false});
  }
  if (P->n_mq > 0) {
    ResArgs a = ra;
    a.cq = P->d_queue + P->n_bq;
    a.n_cq = P->n_mq;
    a.cq_head = P->d_heads + 3;
    ls.push_back({P->res_cluster_mid, P->res_grid_mid, a, false});
  }
  if (P->n_cq > 0) {
    ResArgs a = ra;
    a.cq = P->d_queue + P->n_bq + P->n_mq;
    a.n_cq = P->n_cq;
    a.cq_head = P->d_heads + 1;
    ls.push_back({P->res_cluster, P->res_grid, a, false});
  }
  if (ls.empty() && part) {
    ResArgs a = ra;
    a.cq = P->d_queue;
    a.n_cq = 0;
    a.cq_head = P->d_heads;
    ls.push_back({1, P->res_grid, a, true});
  } else if (P->res_fill > 0) {
    ResArgs a = ra;
    a.cq = P->d_queue;
    a.n_cq = 0;
    a.cq_head = P->d_heads;
    ls.push_back({1, P->res_fill, a, true});
  }
  cudaStream_t side[3] = {P->fj.aux, P->aux2, P->aux3};
  cudaEvent_t joins[3] = {P->fj.join, P->join2, P->join3};
  if (ls.size() > 1) CUDA_TRY(cudaEventRecord(P->fj.fork, st));
  for (size_t i = 0; i < ls.size(); ++i) {
    cudaStream_t s2 = i == 0 ? st : side[i - 1];
    if (i > 0) CUDA_TRY(cudaStreamWaitEvent(s2, P->fj.fork, 0));
    // the launches after the first start a little later: a cluster needs that
    // many free SMs of one GPC, and the largest clusters (the first launch)
    // are placed before smaller groups can take SMs in their GPCs
    if (i > 0) CUDA_TRY(launch_hold(20000ull * i, s2));
    CUDA_TRY(launch(ls[i].cluster, ls[i].grid, ls[i].a, s2, ls[i].cta_only));
    if (i > 0) CUDA_TRY(cudaEventRecord(joins[i - 1], s2));
  }
  for (size_t i = 1; i < ls.size(); ++i) CUDA_TRY(cudaStreamWaitEvent(st, joins[i - 1], 0));
  // the whole-GPU solves after the others (the cooperative launch needs every SM)
  if (P->n_gq > 0) {
    ResArgs a = ra;
    a.gq = P->d_queue + P->n_bq + P->n_mq + P->n_cq + P->n_tq;
    a.n_gq = P->n_gq;
    a.gbar = P->d_gbar;
    a.gpart = P->d_gpart;
    a.gerr = P->d_gerr;
    CUDA_TRY(cudaMemsetAsync(P->d_gbar, 0, 2 * sizeof(unsigned), st));
    CUDA_TRY(cudaMemsetAsync(P->d_gerr, 0, sizeof(int), st));
    CUDA_TRY(launch_resident_grid(P->res_threads, P->res_grid_all, a, st));
  }
  if (prof) CUDA_TRY(cudaEventRecord(P->res_ev[1], st));
  // the resident kernels, the hold kernels before the later ones, the whole-GPU launch
  P->res_launches += (int)ls.size() + std::max(0, (int)ls.size() - 1) + (P->n_gq > 0 ? 1 : 0);
  return ATS_OK;
}

size_t events_per_set(const Plan *P) { return 1 + kTickEvents * (size_t)P->opts.check_every; }

ats_status plan_ensure_events(Plan *P) {
  const size_t need = 2 * events_per_set(P);
  while (P->evs.size() < need) {
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e));
    P->evs.push_back(e);
  }
  return ATS_OK;
}

// `k` ticks on st; when profiling, with the timing events of event set `set`
// on the side stream (chunk start, then per tick), the side stream rejoining
// st at the end.
cudaError_t timed_ticks(Plan *P, const TickArgs &ta, cudaStream_t st, int k, bool capture, int set) {
  cudaError_t err = cudaSuccess;
  if (!P->profiling) {
    for (int t = 0; t < k && err == cudaSuccess; ++t)
      err = launch_tick(P->fp64, P->paper, ta, P->grids, st, &P->fj, nullptr, capture);
    return err;
  }
  cudaEvent_t *evs = &P->evs[set * events_per_set(P)];
  TickTiming tt{P->side, P->mark, nullptr};
  if ((err = record_after(tt, evs[0], st, capture)) != cudaSuccess) return err;
  for (int t = 0; t < k && err == cudaSuccess; ++t) {
    tt.ev = &evs[1 + kTickEvents * t];
    err = launch_tick(P->fp64, P->paper, ta, P->grids, st, &P->fj, &tt, capture);
  }
  if (err != cudaSuccess) return err;
  if ((err = cudaEventRecord(P->mark, P->side)) != cudaSuccess) return err;
  return cudaStreamWaitEvent(st, P->mark, 0);
}

// The device-driven loop of use_graph = 2: a graph holding one WHILE node
// whose body is one interval of ticks followed by the condition kernel.  The
// handle's default value 1 runs the body once per launch before the first
// test.  The interval graph is captured once per plan; the loop graph is
// built once per interval bound (fixed by the options).
ats_status plan_ensure_loop(Plan *P, int max_chunks) {
  if (P->loop_exec && P->loop_max == max_chunks) return ATS_OK;
  if (P->loop_exec) {
    cudaGraphExecDestroy(P->loop_exec);
    P->loop_exec = nullptr;
  }
  ats_context *ctx = P->ctx;
  cudaStream_t st = ctx->stream;
  if (!P->d_loop) {
    ats_status s = dev_alloc_t(ctx, 1, &P->d_loop);
    if (s != ATS_OK) return s;
    CUDA_TRY(cudaMemsetAsync(P->d_loop, 0, sizeof(int), st));
  }
  cudaError_t err = cudaSuccess;
  if (!P->loop_ticks) {
    err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
      TickArgs ta = P->targs;
      ta.cells = nullptr;
      for (int t = 0; t < P->opts.check_every && err == cudaSuccess; ++t)
        err = launch_tick(P->fp64, P->paper, ta, P->grids, st, &P->fj, nullptr, true);
      cudaGraph_t out = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(st, &out);
      if (err == cudaSuccess) err = e2;
      if (err == cudaSuccess) P->loop_ticks = out;
      else if (out) cudaGraphDestroy(out);
    }
  }
  cudaGraph_t g = nullptr;
  if (err == cudaSuccess) err = cudaGraphCreate(&g, 0);
  cudaGraphNode_t node;
  if (err == cudaSuccess) err = add_while_loop(g, nullptr, 0, P->loop_ticks, P->d_active, P->d_loop, max_chunks, &node);
  if (err == cudaSuccess) err = cudaGraphInstantiate(&P->loop_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (err != cudaSuccess) {
    cudaGetLastError();
    P->loop_exec = nullptr;
    set_error(std::string("device loop graph: ") + cudaGetErrorString(err));
    return ATS_ERR_CUDA;
  }
  P->loop_max = max_chunks;
  return ATS_OK;
}

// Enqueue the device loop of P (built by plan_ensure_loop) on st: a launch of
// its graph, or, while st is under capture, the same WHILE node added to the
// graph being captured (a graph launch cannot sit inside another graph when
// it holds a conditional node).
ats_status plan_enqueue_loop(Plan *P, cudaStream_t st, bool capture) {
  if (!capture) {
    CUDA_TRY(cudaGraphLaunch(P->loop_exec, st));
    return ATS_OK;
  }
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t n_deps = 0;
  CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &n_deps));
  if (cs != cudaStreamCaptureStatusActive) {
    set_error("device loop: the stream is not under capture");
    return ATS_ERR_CUDA;
  }
  cudaGraphNode_t node;
  CUDA_TRY(add_while_loop(g, deps, n_deps, P->loop_ticks, P->d_active, P->d_loop, P->loop_max, &node));
  CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return ATS_OK;
}

// Enqueue one poll interval (check_every ticks) on the stream; when
// profiling, its timing events are the set of this poll slot.
ats_status plan_enqueue_chunk(Plan *P) {
  cudaStream_t st = P->ctx->stream;
  const int k = P->opts.check_every;
  const bool prof = P->profiling;
  const int set = P->slot;
  if (P->opts.use_graph) {
    cudaGraphExec_t &exec = prof ? P->exec_prof[set] : P->exec;
    if (!exec) {
      if (prof) {
        ats_status s = plan_ensure_events(P);
        if (s != ATS_OK) return s;
      }
      cudaGraph_t g = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      cudaError_t err = cudaSuccess;
      TickArgs ta = P->targs;
      if (!prof) ta.cells = nullptr;
      err = timed_ticks(P, ta, st, k, true, set);
      cudaError_t err2 = cudaStreamEndCapture(st, &g);
      if (err != cudaSuccess || err2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        set_error(std::string("graph capture failed: ") + cudaGetErrorString(err != cudaSuccess ? err : err2));
        return ATS_ERR_CUDA;
      }
      err = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (err != cudaSuccess) {
        exec = nullptr;
        set_error(std::string("graph instantiate failed: ") + cudaGetErrorString(err));
        return ATS_ERR_CUDA;
      }
    }
    CUDA_TRY(cudaGraphLaunch(exec, st));
  } else {
    if (prof) {
      ats_status s = plan_ensure_events(P);
      if (s != ATS_OK) return s;
    }
    TickArgs ta = P->targs;
    if (!prof) ta.cells = nullptr;
    CUDA_TRY(timed_ticks(P, ta, st, k, false, set));
  }
  P->ticks += k;
  P->launches += 3 * k;
  CUDA_TRY(cudaMemcpyAsync(P->h_active + P->slot, P->d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaEventRecord(P->poll_ev[P->slot], st));
  P->slot ^= 1;
  return ATS_OK;
}

// Per tick: k_op and k_ref both start when the previous k_upd (or the chunk)
// ends; k_upd starts when the later of the two ends.  `set`: the event set of
// the interval (its poll slot).
ats_status plan_collect_events(Plan *P, int set) {
  const int k = P->opts.check_every;
  cudaEvent_t *evs = &P->evs[set * events_per_set(P)];
  cudaEvent_t prev = evs[0];
  for (int t = 0; t < k; ++t) {
    float a = 0.f, b = 0.f, c = 0.f, order = 0.f;
    cudaEvent_t *e = &evs[1 + kTickEvents * t];
    CUDA_TRY(cudaEventElapsedTime(&a, prev, e[0]));
    CUDA_TRY(cudaEventElapsedTime(&b, prev, e[1]));
    CUDA_TRY(cudaEventElapsedTime(&order, e[0], e[1]));
    CUDA_TRY(cudaEventElapsedTime(&c, order >= 0.f ? e[1] : e[0], e[2]));
    P->op_ms += a;
    P->ref_ms += b;
    P->upd_ms += c;
    prev = e[2];
  }
  return ATS_OK;
}

// Algorithmic bytes per cell of each kernel and phase: the compulsory traffic
// of the vectors and coefficients (neighbour tables and records not counted).
//   k_op, CG:        read z, p_old, K_T, D; write p_new, q            (6 words;
//                    5 in the first iteration of an inner solve: p = z)
//   k_ref:           read x64, b64, the three FP64 face coefficients, K_T;
//                    write z, D                                        (40 B + 3 words)
//   k_upd, CG:       read p, q, D, z, e; write z, e                   (7 words)
//   k_upd, x += e:   read/write x (FP64) and e (end of an inner solve) (16 B + 2 words)
void plan_bytes(const Plan *P, const unsigned long long cells[kCellCounters], double *op_b, double *ref_b,
                double *upd_b) {
  const double w = P->fp64 ? 8.0 : 4.0;
  *op_b = 6 * w * cells[0] + 5 * w * cells[4];  // first iteration of an inner solve: no p_old
  *ref_b = (40 + 3 * w) * cells[1];
  *upd_b = 7 * w * cells[2] + (16 + 2 * w) * cells[3];
}

// Enqueue the start of a run: refresh the solve descriptors of levels
// rebuilt since the plan was made, copy x in (device x is read in place,
// host x goes through one staging buffer, one copy per run of levels whose
// host arrays are contiguous), reset every solve's state and the work lists.
// off: [n + 1] offsets of the levels in the staging buffer.  The start state
// and the x pointers are uploaded only when they differ from what the device
// holds; the reset itself is device to device.  capture: st is under stream
// capture, so nothing may come from the host (device x only, and every
// upload already resident, else ATS_ERR_INVALID_ARG).
ats_status plan_begin(Plan *P, double *const *x_inout, std::vector<int64_t> &off, bool capture = false) {
  ats_context *ctx = P->ctx;
  cudaStream_t st = ctx->stream;
  const int n = P->n;
  const bool dev = (P->opts.mem == ATS_MEM_DEVICE);
  CUDA_TRY(cudaSetDevice(ctx->device));
  // a level rebuilt with another dt (or another diagonal-extra layout) since
  // the plan was made: refresh the solve descriptors
  bool stale = false;
  for (int k = 0; k < n; ++k) {
    ats_level *L = P->levels[k];
    SolveDev &sd = P->h_solves[k];
    const double h = 0.5 * L->dt / (L->dx * L->dx);
    const int32_t *xrec = L->dense_xd ? L->xrec_dense : L->frec;
    const void *xdT = P->fp64 ? (const void *)L->xd64 : (const void *)L->xd32;
    if (sd.h != h || sd.xrec != xrec || sd.xd64 != L->xd64 || sd.xdT != xdT || sd.cn_base != L->cn_base) {
      sd.h = h;
      sd.cn_base = L->cn_base;
      sd.xrec = xrec;
      sd.n_xd = (int32_t)(L->dense_xd ? L->n_oct : L->n_rec);
      sd.xd64 = L->xd64;
      sd.xdT = xdT;
      stale = true;
    }
  }
  if (stale && capture) {
    set_error("graph capture: a level was rebuilt with another time step since its last solve");
    return ATS_ERR_INVALID_ARG;
  }
  if (!dev && capture) {
    set_error("graph capture: host-memory solves cannot be captured");
    return ATS_ERR_INVALID_ARG;
  }
  if (stale) {
    ++ctx->epoch;
    CUDA_TRY(cudaMemcpyAsync(P->d_solves, P->h_solves.data(), sizeof(SolveDev) * n, cudaMemcpyHostToDevice, st));
    P->res_meas.clear();  // the work estimates follow dt
    P->queue_dirty = true;
  }
  if (P->queue_dirty && !capture) {
    ats_status sq = plan_upload_queues(P);
    if (sq != ATS_OK) return sq;
    P->queue_dirty = false;
  }
  // copy-in of x: device x is read in place; host x goes through one staging
  // buffer, one copy per run of levels whose host arrays are contiguous
  std::vector<const double *> src(n, nullptr);
  std::vector<double *> dst(n, nullptr);
  off.assign(n + 1, 0);
  const bool x0_e = P->opts.x0 == ATS_X0_E_OLD;
  for (int k = 0; k < n; ++k) {
    if (!x_inout || !x_inout[k]) {
      set_error("x_inout[k] is NULL");
      return ATS_ERR_INVALID_ARG;
    }
    if (x0_e && !P->levels[k]->E_dev) {
      set_error("x0 = E_old: the level has no operator build");
      return ATS_ERR_INVALID_ARG;
    }
    off[k + 1] = off[k] + P->levels[k]->N;
  }
  if (!dev) {
    if (!P->d_xstage) {
      ats_status s2 = dev_alloc_t(ctx, std::max<int64_t>(1, off[n]), &P->d_xstage);
      if (s2 != ATS_OK) return s2;
    }
    if (!x0_e) {
      ats_status s2 = copy_runs(st, true, P->d_xstage, off.data(), n, x_inout);
      if (s2 != ATS_OK) return s2;
    }
  }
  // where each result goes: the FP32-bulk resident kernels write their
  // solves' results themselves as each solve ends -- into device x, into host
  // x directly when the device can write it (pinned), else into the staging
  // buffer -- and k_final writes the others; copy_runs brings back the staged
  // host results
  if (!dev) {
    std::vector<double *> hx(x_inout, x_inout + n);
    if (hx != P->h_xhost) {
      P->h_xhost = hx;
      P->h_xdev.assign(n, nullptr);
      P->h_xdirect.assign(n, 0);
      for (int k = 0; k < n; ++k) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, hx[k]) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer) {
          P->h_xdev[k] = (double *)pa.devicePointer;
          P->h_xdirect[k] = 1;
        }
        cudaGetLastError();
      }
    }
  }
  std::vector<double *> rdst(n, nullptr);
  P->h_copyback.assign(n, nullptr);
  for (int k = 0; k < n; ++k) {
    double *stage = dev ? x_inout[k] : P->d_xstage + off[k];
    src[k] = x0_e ? P->levels[k]->E_dev : stage;
    const int m = P->mode[k];
    const bool res_out = P->res_smem && (m == 1 || m == 2 || m == 3 || m == 5);
    const bool direct = !dev && res_out && P->h_xdirect[k];
    dst[k] = res_out ? nullptr : stage;
    rdst[k] = res_out ? (direct ? P->h_xdev[k] : stage) : nullptr;
    if (!dev && !direct) P->h_copyback[k] = x_inout[k];
  }
  if (src != P->h_src || dst != P->h_dst || rdst != P->h_rdst) {
    if (capture) {
      set_error("graph capture: the solve's x is not the one of its last run");
      return ATS_ERR_INVALID_ARG;
    }
    ++ctx->epoch;
    P->h_src = src;
    P->h_dst = dst;
    P->h_rdst = rdst;
    CUDA_TRY(cudaMemcpyAsync(P->d_src, P->h_src.data(), sizeof(double *) * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(P->d_dst, P->h_dst.data(), sizeof(double *) * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(P->d_rdst, P->h_rdst.data(), sizeof(double *) * n, cudaMemcpyHostToDevice, st));
  }
  CUDA_TRY(launch_init(P->fp64, P->d_solves, P->d_items, P->n_items, P->d_src, P->grid, st));
  // the start state: every solve's scalars (live and final copies), the
  // active count (only the tick-path solves count for the tick loop) and the
  // tick control block (every item of every tick-path solve starts in the
  // refinement phase, r0 = b - A x0)
  const size_t sc_b = sizeof(SolveScalars) * n;
  const size_t ctl_at = (sc_b + sizeof(int) + 15) / 16 * 16;
  std::vector<unsigned char> img(ctl_at + sizeof(TickCtl), 0);
  std::memcpy(img.data(), P->h_sc.data(), sc_b);
  std::memcpy(img.data() + sc_b, &P->n_tick, sizeof(int));
  {
    TickCtl c0;
    std::memset(&c0, 0, sizeof(c0));
    c0.count[0][kRefine] = P->n_tick_items;
    std::memcpy(img.data() + ctl_at, &c0, sizeof(c0));
  }
  if (img != P->h_init) {
    if (capture) {
      set_error("graph capture: the solves' start state is not resident");
      return ATS_ERR_INVALID_ARG;
    }
    if (!P->d_init) {
      ats_status s2 = dev_alloc_t(ctx, img.size(), &P->d_init);
      if (s2 != ATS_OK) return s2;
    }
    ++ctx->epoch;
    P->h_init = img;
    CUDA_TRY(cudaMemcpyAsync(P->d_init, P->h_init.data(), img.size(), cudaMemcpyHostToDevice, st));
  }
  CUDA_TRY(cudaMemcpyAsync(P->d_sc, P->d_init, sc_b, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(P->d_final, P->d_init, sc_b, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemsetAsync(P->d_cells, 0, 2 * kCellCounters * sizeof(unsigned long long), st));
  CUDA_TRY(cudaMemcpyAsync(P->d_active, P->d_init + sc_b, sizeof(int), cudaMemcpyDeviceToDevice, st));
  if (P->n_tick_items > 0)
    CUDA_TRY(cudaMemcpyAsync(P->d_lists + (size_t)kRefine * P->n_items, P->d_ident,
                             sizeof(int32_t) * P->n_tick_items, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(P->d_ctl, P->d_init + ctl_at, sizeof(TickCtl), cudaMemcpyDeviceToDevice, st));
  P->op_ms = P->ref_ms = P->upd_ms = 0.0;
  P->res_ms = P->res_bytes = 0.0;
  P->launches = 0;
  P->res_launches = 0;
  P->ticks = 0;
  return ATS_OK;
}

// The tick bound of a run: every solve ends within it (an inner pass's
// convergence is seen one tick late: two ticks per pass boundary).
int64_t plan_max_ticks(const Plan *P) {
  return 2 * ((int64_t)P->opts.max_iter + 2 * ((int64_t)P->opts.max_refine + 2)) + 2 * P->opts.check_every;
}

// After a plan's launches, an error return first waits for the work already
// queued on the stream: the resident kernels write each solve's result into
// the caller's array (pinned host memory included) when the solve ends, and
// must not do so after the call has returned.
struct DrainOnReturn {
  cudaStream_t st;
  bool armed;
  ~DrainOnReturn() {
    if (armed) {
      cudaStreamSynchronize(st);
      cudaGetLastError();
    }
  }
};

// Run a plan to completion: x_inout[k] (host or device per opts.mem) is the
// initial guess and receives the result.  A right-hand-side override is the
// caller's: ats_solve writes it into the level's b before and restores b after.
ats_status plan_run(Plan *P, double *const *x_inout, ats_solve_stats *stats) {
  ats_context *ctx = P->ctx;
  cudaStream_t st = ctx->stream;
  const int n = P->n;
  const bool dev = (P->opts.mem == ATS_MEM_DEVICE);
  std::vector<int64_t> off;
  {
    ats_status s0 = plan_begin(P, x_inout, off);
    if (s0 != ATS_OK) return s0;
  }

  // host guard: every solve ends within a bounded number of ticks
  const int64_t max_ticks = plan_max_ticks(P);
  int64_t ticks = 0;
  ats_status s;
  bool timed_out = false;
  // the resident solves: one launch runs every one of them to its end (and
  // writes their results; the negative-result flags are zeroed first)
  CUDA_TRY(cudaMemsetAsync(P->d_flags + n, 0, sizeof(int) * n, st));
  // the host copies of the solves' scalars and flags outlive the drain
  std::vector<SolveScalars> sc(n);
  std::vector<int> flags(2 * n, 0);
  DrainOnReturn drain{st, true};
  if ((s = plan_launch_resident(P, P->profiling, P->d_flags + n)) != ATS_OK) return s;
  // use_graph = 2 (not while profiling: the timing events cannot sit in a
  // conditional body): the whole loop is one graph launch, ended on the device
  const bool device_loop = P->opts.use_graph == 2 && !P->profiling && P->n_tick > 0;
  int chunks_run = 0;
  int drain_slot = 0, drain_n = 0;  // intervals still queued when the host loop ended
  if (P->n_tick == 0) {
    // no tick-path solve: no tick loop
  } else if (device_loop) {
    const int max_chunks = (int)std::min<int64_t>((max_ticks + P->opts.check_every - 1) / P->opts.check_every, 1 << 30);
    if ((s = plan_ensure_loop(P, max_chunks)) != ATS_OK) return s;
    CUDA_TRY(cudaMemsetAsync(P->d_loop, 0, sizeof(int), st));
    CUDA_TRY(cudaGraphLaunch(P->loop_exec, st));
    CUDA_TRY(cudaMemcpyAsync(P->h_active, P->d_loop, sizeof(int), cudaMemcpyDeviceToHost, st));  // pinned
  } else {
  // Keep one poll interval queued ahead of the one being polled, so the GPU
  // never idles on the host's check.  Extra intervals after convergence are
  // no-ops: every work item of a finished solve is skipped.  When profiling,
  // the two queued intervals record into the two event sets (one per poll
  // slot), and an interval's events are read before its slot is reused; the
  // interval still queued at the end is read too, so the kernel times cover
  // every tick that ran.
  P->slot = 0;
  int pending = 0;  // intervals enqueued but not yet polled
  int poll_slot = 0;
  for (int k = 0; k < 2; ++k) {
    if ((s = plan_enqueue_chunk(P)) != ATS_OK) return s;
    ++pending;
    ticks += P->opts.check_every;
  }
  for (;;) {
    CUDA_TRY(cudaEventSynchronize(P->poll_ev[poll_slot]));
    const int active = P->h_active[poll_slot];
    if (P->profiling) {
      if ((s = plan_collect_events(P, poll_slot)) != ATS_OK) return s;
    }
    poll_slot ^= 1;
    --pending;
    if (active <= 0) break;
    if (ticks >= max_ticks) {
      timed_out = true;
      break;
    }
    if ((s = plan_enqueue_chunk(P)) != ATS_OK) return s;
    ++pending;
    ticks += P->opts.check_every;
  }
  drain_slot = poll_slot;
  drain_n = pending;
  }
  // copy-out (k_final: the results the resident kernels did not write)
  CUDA_TRY(launch_final(P->d_solves, P->d_items, P->n_items, P->d_dst, P->d_flags + n, P->grid, st));
  if (!dev) {
    ats_status s2 = copy_runs(st, false, P->d_xstage, off.data(), n, P->h_copyback.data());
    if (s2 != ATS_OK) return s2;
  }
  CUDA_TRY(cudaMemcpyAsync(sc.data(), P->d_final, sizeof(SolveScalars) * n, cudaMemcpyDeviceToHost, st));
  unsigned long long cells[2 * kCellCounters] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // tick kernels, resident launch
  if (P->profiling) CUDA_TRY(cudaMemcpyAsync(cells, P->d_cells, sizeof(cells), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(launch_gather_flags(P->d_flag_ptrs, n, P->d_flags, st));
  CUDA_TRY(cudaMemcpyAsync(flags.data(), P->d_flags, sizeof(int) * 2 * n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  drain.armed = false;
  if (P->profiling) {
    for (int k = 0; k < drain_n; ++k, drain_slot ^= 1) {
      ats_status s3 = plan_collect_events(P, drain_slot);
      if (s3 != ATS_OK) return s3;
    }
  }
  if (device_loop) {
    chunks_run = P->h_active[0];
    P->ticks = chunks_run * P->opts.check_every;
    P->launches = 3 * P->ticks + chunks_run;
    if ((int64_t)chunks_run * P->opts.check_every >= max_ticks) timed_out = true;
  }
  if (P->profiling) {
    plan_bytes(P, cells, &P->op_bytes, &P->ref_bytes, &P->upd_bytes);
    if (P->n_bq + P->n_mq + P->n_cq + P->n_tq + P->n_gq > 0) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, P->res_ev[0], P->res_ev[1]));
      P->res_ms = ms;
      // the minimal traffic of the method, as if every vector were streamed
      // from memory: 10 words per cell and CG iteration (read p, K, x, r, q,
      // D^-1; write q, x, r, p) and 5 FP64 words per cell and refinement pass
      // (read x, b, K; write r, D) -- the resident solver keeps most of it
      // on chip, so its DRAM traffic is far lower
      const unsigned long long *rc = cells + kCellCounters;
      const double w = P->fp64 ? 8.0 : 4.0;
      P->res_bytes = 10.0 * w * (double)(rc[0] + rc[4]) + 40.0 * (double)rc[1];
      // the launch's timeline: span from the first solve's start to the last
      // one's end, the longest solve, and the fraction of the launch's
      // CTA-time spent inside solves
      std::vector<unsigned long long> ts(2 * (size_t)n);
      CUDA_TRY(cudaMemcpy(ts.data(), P->d_tsolve, sizeof(unsigned long long) * ts.size(), cudaMemcpyDeviceToHost));
      unsigned long long t0 = ~0ull, t1 = 0;
      double busy = 0.0, longest = 0.0;
      P->res_longest = -1;
      for (int k = 0; k < n; ++k) {
        if (P->mode[k] == 0 || ts[2 * k + 1] < ts[2 * k]) continue;
        t0 = std::min(t0, ts[2 * k]);
        t1 = std::max(t1, ts[2 * k + 1]);
        const double d = (double)(ts[2 * k + 1] - ts[2 * k]) * 1e-6;
        busy += d * group_ctas(P, P->mode[k]);
        if (d > longest) {
          longest = d;
          P->res_longest = k;
        }
      }
      P->res_span_ms = t1 > t0 ? (double)(t1 - t0) * 1e-6 : 0.0;
      // when the last solve of each kind ended (big clusters, clusters, one CTA)
      for (int q = 0; q < 3; ++q) P->res_end_ms[q] = 0.0;
      for (int k = 0; k < n; ++k) {
        if (P->mode[k] == 0 || ts[2 * k + 1] < ts[2 * k] || t1 <= t0) continue;
        const int q = (P->mode[k] == 3 || P->mode[k] == 4 || P->mode[k] == 5) ? 0 : P->mode[k] == 1 ? 1 : 2;
        P->res_end_ms[q] = std::max(P->res_end_ms[q], (double)(ts[2 * k + 1] - t0) * 1e-6);
      }
      P->res_longest_ms = longest;
      P->res_occupancy =
          P->res_span_ms > 0
              ? busy / (P->res_span_ms * (P->res_grid + P->res_grid_big + P->res_grid_mid + P->res_fill))
              : 0.0;
    }
  }
  // the next run's split of the slots between the resident launches
  if (P->n_bq + P->n_mq + P->n_cq + P->n_tq > 0 && P->d_tsolve) {
    std::vector<unsigned long long> ts(2 * (size_t)n);
    CUDA_TRY(cudaMemcpy(ts.data(), P->d_tsolve, sizeof(unsigned long long) * ts.size(), cudaMemcpyDeviceToHost));
    plan_adapt_split(P, ts);
  }
  ats_status first_err = ATS_OK, first_warn = ATS_OK;
  for (int k = 0; k < n; ++k) {
    int status = sc[k].status;
    if (flags[k]) status = ATS_ERR_BAD_INPUT;
    if (timed_out && sc[k].phase != kDone) status = ATS_ERR_TIMEOUT;
    if (P->mode[k] != 0 && sc[k].phase != kDone && status == ATS_OK) status = ATS_ERR_TIMEOUT;  // never ran
    if (status == ATS_OK && flags[n + k]) status = ATS_WARN_NEGATIVE;
    if (stats) {
      ats_solve_stats &o = stats[k];
      o.status = status;
      o.iterations = sc[k].iters;
      o.refinements = sc[k].refines;
      o.ticks = sc[k].ticks;
      o.r0_norm = sc[k].r0;
      o.res_norm = sc[k].rnorm;
      o.x_norm = sc[k].xnorm;
      o.err_bound = sc[k].xnorm > 0.0 ? sc[k].rnorm / sc[k].xnorm : 0.0;
    }
    if (status < 0 && first_err == ATS_OK) first_err = status;
    if (status > 0 && first_warn == ATS_OK) first_warn = status;
  }
  if (first_err != ATS_OK) {
    set_error(std::string("solve failed: ") + ats_status_string(first_err));
    return first_err;
  }
  return first_warn;
}

}  // namespace

namespace ats {
int tile_for(int64_t n_oct, int requested, int grid) { return choose_tile(n_oct, requested, grid); }
ats_solve_opts normalized_opts(const ats_solve_opts *in) { return normalize(in); }
ats_status solve_dev_for(ats_level *L, const ats_solve_opts &o, bool fp64, int item_begin, int n_items,
                         SolveDev *out) {
  ats_status s = ensure_vectors(L, fp64);
  if (s != ATS_OK) return s;
  SolveDev &sd = *out;
  std::memset(&sd, 0, sizeof(sd));
  sd.nbr = L->nbr;
  sd.xrec = L->dense_xd ? L->xrec_dense : L->frec;
  sd.n_xd = (int32_t)(L->dense_xd ? L->n_oct : L->n_rec);
  sd.K64 = L->K64;
  sd.C64 = L->C64;
  sd.KT = fp64 ? (const void *)L->K64 : (const void *)L->K32;
  sd.xd64 = L->xd64;
  sd.xdT = fp64 ? (const void *)L->xd64 : (const void *)L->xd32;
  sd.b64 = L->b64;
  sd.x64 = L->x64;
  sd.cn_base = L->cn_base;
  const int vk = fp64 ? 0 : 1;
  sd.e = L->e[vk];
  sd.z = L->z[vk];
  sd.p0 = L->p0[vk];
  sd.p1 = L->p1[vk];
  sd.q = L->q[vk];
  sd.dg = L->dg[vk];
  sd.h = 0.5 * L->dt / (L->dx * L->dx);
  sd.tol = o.tol;
  sd.inner_rtol = fp64 ? 0.0 : o.inner_rtol;
  sd.final_safety = fp64 ? 1.0 : 0.5;
  sd.n_oct = (int32_t)L->n_oct;
  sd.item_begin = item_begin;
  sd.n_items = n_items;
  sd.stop_rule = o.stop_rule;
  sd.max_iter = o.max_iter;
  sd.max_refine = o.max_refine;
  sd.inner_max = fp64 ? o.max_iter : 4000;
  return ATS_OK;
}
}  // namespace ats

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

void ats_default_opts(ats_solve_opts *opts) {
  if (opts) fill_defaults(opts);
}

const char *ats_status_string(ats_status s) {
  switch (s) {
    case ATS_OK: return "ok";
    case ATS_ERR_INVALID_ARG: return "invalid argument";
    case ATS_ERR_OOM: return "out of device memory";
    case ATS_ERR_OVER_BUDGET: return "device memory budget exceeded";
    case ATS_ERR_NOT_CONVERGED: return "not converged";
    case ATS_ERR_BREAKDOWN: return "CG breakdown";
    case ATS_ERR_TIMEOUT: return "timeout";
    case ATS_ERR_CUDA: return "CUDA error";
    case ATS_ERR_NO_DEVICE: return "no CUDA device";
    case ATS_ERR_BAD_INPUT: return "bad input (non-finite value or K <= 0)";
    case ATS_WARN_NEGATIVE: return "warning: negative energy in solution";
    default: return "unknown status";
  }
}

const char *ats_last_error(void) { return g_last_error.c_str(); }

ats_status ats_layout_neighbors(const ats_level_desc *desc, int32_t *nbr) {
  try {  // no C++ exception leaves the library
    if (!desc || !nbr) {
      set_error("null argument");
      return ATS_ERR_INVALID_ARG;
    }
    Layout lay;
    std::string msg = build_layout(*desc, lay);
    if (!msg.empty()) {
      set_error(msg);
      return ATS_ERR_INVALID_ARG;
    }
    std::memcpy(nbr, lay.nbr.data(), sizeof(int32_t) * lay.nbr.size());
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_context_create(int device, size_t budget, ats_context **out) {
  try {  // no C++ exception leaves the library
    if (!out) return ATS_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
      cudaGetLastError();
      set_error("no CUDA device");
      return ATS_ERR_NO_DEVICE;
    }
    if (device < 0 || device >= count) {
      set_error("device index out of range");
      return ATS_ERR_INVALID_ARG;
    }
    CUDA_TRY(cudaSetDevice(device));
    ats_context *ctx = new (std::nothrow) ats_context();
    if (!ctx) return ATS_ERR_OOM;
    ctx->device = device;
    ctx->budget = budget;
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete ctx;
      set_error(cudaGetErrorString(e));
      return ATS_ERR_CUDA;
    }
    ctx->stream = ctx->own_stream;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (ctx->num_sms <= 0) ctx->num_sms = 1;
    *out = ctx;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_context_destroy(ats_context *ctx) {
  try {  // no C++ exception leaves the library
    if (!ctx) return ATS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->allocs) cudaFree(kv.first);
    ctx->allocs.clear();
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_context_set_stream(ats_context *ctx, void *stream) {
  try {  // no C++ exception leaves the library
    if (!ctx) return ATS_ERR_INVALID_ARG;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_context_memory(const ats_context *ctx, size_t *used, size_t *budget) {
  try {  // no C++ exception leaves the library
    if (!ctx) return ATS_ERR_INVALID_ARG;
    if (used) *used = ctx->used;
    if (budget) *budget = ctx->budget;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_level_create(ats_context *ctx, const ats_level_desc *desc, ats_level **out) {
  try {  // no C++ exception leaves the library
    if (!ctx || !desc || !out) {
      set_error("null argument");
      return ATS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    Layout lay;
    std::string msg = build_layout(*desc, lay);
    if (!msg.empty()) {
      set_error(msg);
      return ATS_ERR_INVALID_ARG;
    }
    return ats::level_create_with_layout(ctx, desc, lay, out);
  } catch (...) {
    return ats::abi_exception();
  }
}

}  // extern "C"

ats_status ats::level_create_with_layout(ats_context *ctx, const ats_level_desc *desc, const Layout &lay,
                                         ats_level **out) {
  *out = nullptr;
  CUDA_TRY(cudaSetDevice(ctx->device));
  ats_level *L = new (std::nothrow) ats_level();
  if (!L) return ATS_ERR_OOM;
  L->ctx = ctx;
  L->n_oct = desc->n_oct;
  L->N = 8 * desc->n_oct;
  L->n_face = desc->n_face;
  L->n_rec = lay.n_rec;
  L->dx = desc->dx;
  cudaStream_t st = ctx->stream;
  ats_status s;
  auto fail = [&](ats_status code) {
    ats_level_destroy(L);
    return code;
  };
  if ((s = dev_alloc_t(ctx, 6 * L->n_oct, &L->nbr)) != ATS_OK) return fail(s);
  if ((s = dev_alloc_t(ctx, L->n_oct, &L->frec)) != ATS_OK) return fail(s);
  if ((s = dev_alloc_t(ctx, std::max<int64_t>(1, 48 * L->n_rec), &L->rec_face)) != ATS_OK) return fail(s);
  if ((s = dev_alloc_t(ctx, L->n_oct, &L->leaf)) != ATS_OK) return fail(s);
  if ((s = dev_alloc_t(ctx, 1, &L->err_flag)) != ATS_OK) return fail(s);
  std::vector<uint8_t> leaf(L->n_oct, 0xFF);
  if (desc->leaf_mask) std::memcpy(leaf.data(), desc->leaf_mask, L->n_oct);
  if (cudaMemcpyAsync(L->nbr, lay.nbr.data(), sizeof(int32_t) * lay.nbr.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(L->frec, lay.frec.data(), sizeof(int32_t) * lay.frec.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (L->n_rec > 0 && cudaMemcpyAsync(L->rec_face, lay.rec_face.data(), sizeof(int32_t) * lay.rec_face.size(),
                                       cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      cudaMemcpyAsync(L->leaf, leaf.data(), L->n_oct, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(L->err_flag, 0, sizeof(int), st) != cudaSuccess) {
    set_error("level upload failed");
    return fail(ATS_ERR_CUDA);
  }
  if (L->n_face > 0) {
    if ((s = dev_alloc_t(ctx, L->n_face, &L->fkind)) != ATS_OK) return fail(s);
    if ((s = dev_alloc_t(ctx, L->n_face, &L->frel)) != ATS_OK) return fail(s);
    if ((s = dev_alloc_t(ctx, L->n_face, &L->falpha)) != ATS_OK) return fail(s);
    std::vector<double> alpha(L->n_face, 1.0);
    if (desc->face_alpha) std::memcpy(alpha.data(), desc->face_alpha, sizeof(double) * L->n_face);
    if (cudaMemcpyAsync(L->fkind, desc->face_kind, L->n_face, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(L->frel, desc->face_rel, L->n_face, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(L->falpha, alpha.data(), sizeof(double) * L->n_face, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      set_error("face upload failed");
      return fail(ATS_ERR_CUDA);
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("level upload sync failed");
    return fail(ATS_ERR_CUDA);
  }
  *out = L;
  return ATS_OK;
}

extern "C" {

ats_status ats_level_destroy(ats_level *L) {
  try {  // no C++ exception leaves the library
    if (!L) return ATS_ERR_INVALID_ARG;
    ats_context *ctx = L->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (L->solo) plan_free(L->solo);
    void *ptrs[] = {L->nbr, L->frec, L->rec_face, L->xrec_dense, L->leaf, L->fkind, L->frel,
                    L->falpha, L->K64, L->xd64, L->b64, L->C64, L->K32, L->xd32, L->err_flag,
                    L->stage_cell, L->stage_face, L->x64, L->rhs_save,
                    L->e[0], L->z[0], L->p0[0], L->p1[0], L->e[1], L->z[1], L->p0[1], L->p1[1],
                    L->q[0], L->dg[0], L->q[1], L->dg[1]};
    for (void *p : ptrs) dev_free(ctx, p);
    delete L;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_level_size(const ats_level *L, int64_t *n_oct, int64_t *n_cell, int64_t *n_face) {
  try {  // no C++ exception leaves the library
    if (!L) return ATS_ERR_INVALID_ARG;
    if (n_oct) *n_oct = L->n_oct;
    if (n_cell) *n_cell = L->N;
    if (n_face) *n_face = L->n_face;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

}  // extern "C"

namespace {

// Validate a coefficient description, allocate the level's operator arrays,
// stage host arrays on the device, and fill the kernel arguments.  Enqueues
// copies on the context stream; does not launch the kernel.
ats_status prepare_operator(ats_level *L, const ats_coef_desc *c, CoefArgs *out) {
  if (!L || !c) {
    set_error("null argument");
    return ATS_ERR_INVALID_ARG;
  }
  if (!(c->dt > 0.0) || !std::isfinite(c->dt)) {
    set_error("dt must be finite and > 0");
    return ATS_ERR_INVALID_ARG;
  }
  if (!c->K || !c->E_old) {
    set_error("K and E_old are required");
    return ATS_ERR_INVALID_ARG;
  }
  if (c->mem != ATS_MEM_HOST && c->mem != ATS_MEM_DEVICE) {
    set_error("bad mem");
    return ATS_ERR_INVALID_ARG;
  }
  const bool cn = (c->integrator == ATS_INTEGRATOR_CRANK_NICOLSON);
  if (!cn && c->integrator != ATS_INTEGRATOR_BACKWARD_EULER) {
    set_error("unknown integrator");
    return ATS_ERR_INVALID_ARG;
  }
  if (cn && c->s) {
    set_error("the Crank-Nicolson integrator takes no shift s");
    return ATS_ERR_INVALID_ARG;
  }
  // Crank-Nicolson: the backward-Euler system of the half step (sources at
  // half weight); the solve extrapolates E^{n+1} = 2 x - E^n from its root
  const double dt_op = cn ? 0.5 * c->dt : c->dt;
  ats_context *ctx = L->ctx;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  ats_status s;
  const int64_t N = L->N;
  if (!L->K64) {
    if ((s = dev_alloc_t(ctx, N, &L->K64)) != ATS_OK) return s;
    if ((s = dev_alloc_t(ctx, N, &L->K32)) != ATS_OK) return s;
    if ((s = dev_alloc_t(ctx, N, &L->b64)) != ATS_OK) return s;
    if ((s = dev_alloc_t(ctx, 3 * N, &L->C64)) != ATS_OK) return s;
  }
  // diagonal extras: sparse records, or dense when a shift s is given
  const bool dense = (c->s != nullptr);
  const int64_t need = dense ? L->n_oct : L->n_rec;
  if (need > L->xd_cap) {
    dev_free(ctx, L->xd64);
    dev_free(ctx, L->xd32);
    L->xd64 = nullptr;
    L->xd32 = nullptr;
    L->xd_cap = 0;
    if ((s = dev_alloc_t(ctx, std::max<int64_t>(1, 8 * need), &L->xd64)) != ATS_OK) return s;
    if ((s = dev_alloc_t(ctx, std::max<int64_t>(1, 8 * need), &L->xd32)) != ATS_OK) return s;
    L->xd_cap = need;
  }
  if (dense && !L->xrec_dense) {
    if ((s = dev_alloc_t(ctx, L->n_oct, &L->xrec_dense)) != ATS_OK) return s;
    std::vector<int32_t> id(L->n_oct);
    for (int64_t o = 0; o < L->n_oct; ++o) id[o] = (int32_t)o;
    CUDA_TRY(cudaMemcpyAsync(L->xrec_dense, id.data(), sizeof(int32_t) * L->n_oct, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  L->dense_xd = dense;

  const double *K = c->K, *E = c->E_old, *sh = c->s, *src = c->src;
  const double *fK = c->face_K, *fE = c->face_E, *fF = c->face_F;
  if (c->mem == ATS_MEM_HOST) {
    if (!L->stage_cell) {
      if ((s = dev_alloc_t(ctx, 4 * N, &L->stage_cell)) != ATS_OK) return s;
      if ((s = dev_alloc_t(ctx, std::max<int64_t>(1, 3 * L->n_face), &L->stage_face)) != ATS_OK) return s;
    }
    double *dK = L->stage_cell, *dE = dK + N, *dS = dE + N, *dSrc = dS + N;
    double *dfK = L->stage_face, *dfE = dfK + L->n_face, *dfF = dfE + L->n_face;
    CUDA_TRY(cudaMemcpyAsync(dK, K, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(dE, E, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    K = dK;
    E = dE;
    if (sh) {
      CUDA_TRY(cudaMemcpyAsync(dS, sh, sizeof(double) * N, cudaMemcpyHostToDevice, st));
      sh = dS;
    }
    if (src) {
      CUDA_TRY(cudaMemcpyAsync(dSrc, src, sizeof(double) * N, cudaMemcpyHostToDevice, st));
      src = dSrc;
    }
    if (L->n_face > 0) {
      if (fK) {
        CUDA_TRY(cudaMemcpyAsync(dfK, fK, sizeof(double) * L->n_face, cudaMemcpyHostToDevice, st));
        fK = dfK;
      }
      if (fE) {
        CUDA_TRY(cudaMemcpyAsync(dfE, fE, sizeof(double) * L->n_face, cudaMemcpyHostToDevice, st));
        fE = dfE;
      }
      if (fF) {
        CUDA_TRY(cudaMemcpyAsync(dfF, fF, sizeof(double) * L->n_face, cudaMemcpyHostToDevice, st));
        fF = dfF;
      }
    }
  }
  CoefArgs &a = *out;
  std::memset(&a, 0, sizeof(a));
  a.n_oct = L->n_oct;
  a.leaf = L->leaf;
  a.frec = L->frec;
  a.rec_face = L->rec_face;
  a.xrec = dense ? L->xrec_dense : L->frec;
  a.face_kind = L->fkind;
  a.face_rel = L->frel;
  a.face_alpha = L->falpha;
  a.face_K = L->n_face ? fK : nullptr;
  a.face_E = L->n_face ? fE : nullptr;
  a.face_F = L->n_face ? fF : nullptr;
  a.K = K;
  a.E_old = E;
  a.s = sh;
  a.src = src;
  a.h = 0.5 * dt_op / (L->dx * L->dx);
  a.src_scale = cn ? 0.5 : 1.0;
  a.K64 = L->K64;
  a.K32 = L->K32;
  a.xd64 = L->xd64;
  a.xd32 = L->xd32;
  a.b64 = L->b64;
  a.err_flag = L->err_flag;
  a.nbr = L->nbr;
  a.C64 = L->C64;
  a.n_rec = L->n_rec;
  a.n_xd = dense ? L->n_oct : L->n_rec;
  a.n_face = L->n_face;
  L->E_dev = E;
  L->cn_base = cn ? E : nullptr;
  L->dt = dt_op;
  L->built = true;
  return ATS_OK;
}

}  // namespace

extern "C" {

ats_status ats_level_build_operator(ats_level *L, const ats_coef_desc *c) {
  try {  // no C++ exception leaves the library
    CoefArgs a;
    ats_status s = prepare_operator(L, c, &a);
    if (s != ATS_OK) return s;
    cudaStream_t st = L->ctx->stream;
    CUDA_TRY(cudaMemsetAsync(L->err_flag, 0, sizeof(int), st));
    CUDA_TRY(launch_coef_build(a, st));
    // host arrays: the caller may reuse them once the call returns
    if (c->mem == ATS_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(st));
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_level_get_rhs(ats_level *L, double *b, int mem) {
  try {  // no C++ exception leaves the library
    if (!L || !b || !L->built) return ATS_ERR_INVALID_ARG;
    CUDA_TRY(cudaSetDevice(L->ctx->device));
    CUDA_TRY(cudaMemcpyAsync(b, L->b64, sizeof(double) * L->N, kind_of(mem, false), L->ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(L->ctx->stream));
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_level_apply(ats_level *L, const double *x, double *y, int mem) {
  try {  // no C++ exception leaves the library
    if (!L || !x || !y || !L->built) return ATS_ERR_INVALID_ARG;
    ats_context *ctx = L->ctx;
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    double *dx = nullptr, *dy = nullptr;
    ats_status s;
    if (mem == ATS_MEM_HOST) {
      if ((s = dev_alloc_t(ctx, L->N, &dx)) != ATS_OK) return s;
      if ((s = dev_alloc_t(ctx, L->N, &dy)) != ATS_OK) {
        dev_free(ctx, dx);
        return s;
      }
      cudaMemcpyAsync(dx, x, sizeof(double) * L->N, cudaMemcpyHostToDevice, st);
    }
    SolveDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.nbr = L->nbr;
    sd.xrec = L->dense_xd ? L->xrec_dense : L->frec;
    sd.n_xd = (int32_t)(L->dense_xd ? L->n_oct : L->n_rec);
    sd.K64 = L->K64;
    sd.xd64 = L->xd64;
    sd.h = 0.5 * L->dt / (L->dx * L->dx);
    sd.n_oct = (int32_t)L->n_oct;
    cudaError_t e = launch_apply64(&sd, mem == ATS_MEM_HOST ? dx : x, mem == ATS_MEM_HOST ? dy : y, st);
    if (e == cudaSuccess && mem == ATS_MEM_HOST)
      e = cudaMemcpyAsync(y, dy, sizeof(double) * L->N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(ctx, dx);
    dev_free(ctx, dy);
    if (e != cudaSuccess) {
      set_error(cudaGetErrorString(e));
      return ATS_ERR_CUDA;
    }
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_solve(ats_level *L, const double *rhs, double *x_inout, const ats_solve_opts *opts,
                     ats_solve_stats *stats);
}  // extern "C"

namespace ats {

ats_status level_solve_deferred(ats_level *L, double *x_dev, const ats_solve_opts *opts, DeferredRec *d_rec,
                                int *check_every, int64_t *max_ticks, bool capture) {
  if (!L || !x_dev || !d_rec || !L->built) {
    set_error("deferred solve: bad argument or level operator not built");
    return ATS_ERR_INVALID_ARG;
  }
  ats_solve_opts o = normalize(opts);
  o.use_graph = 2;
  o.mem = ATS_MEM_DEVICE;
  ats_context *ctx = L->ctx;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  ats_status s;
  const bool stale_plan = L->solo && (std::memcmp(&L->solo->opts, &o, sizeof(o)) != 0 ||
                                      L->solo->fp64 != (o.precision == ATS_PREC_FP64));
  if (capture && (!L->solo || stale_plan)) {
    set_error("graph capture: the level has no plan for these options");
    return ATS_ERR_INVALID_ARG;
  }
  if (stale_plan) {
    plan_free(L->solo);
    L->solo = nullptr;
  }
  if (!L->solo) {
    ats_level *arr[1] = {L};
    if ((s = plan_create(ctx, arr, 1, &o, &L->solo)) != ATS_OK) return s;
  }
  Plan *P = L->solo;
  const bool prof = P->profiling;
  P->profiling = false;
  std::vector<int64_t> off;
  double *xs[1] = {x_dev};
  s = plan_begin(P, xs, off, capture);
  const int64_t mt = plan_max_ticks(P);
  const int max_chunks = (int)std::min<int64_t>((mt + o.check_every - 1) / o.check_every, 1 << 30);
  if (capture && s == ATS_OK && (!P->d_loop || (P->n_tick > 0 && (!P->loop_exec || P->loop_max != max_chunks)))) {
    set_error("graph capture: the level's device loop is not built");
    s = ATS_ERR_INVALID_ARG;
  }
  if (s == ATS_OK && P->n_tick > 0) s = plan_ensure_loop(P, max_chunks);
  if (s == ATS_OK && !P->d_loop) s = dev_alloc_t(ctx, 1, &P->d_loop);
  if (s == ATS_OK) {
    const cudaError_t e = cudaMemsetAsync(&d_rec->neg, 0, sizeof(int), st);
    if (e != cudaSuccess) {
      set_error(std::string("CUDA error: ") + cudaGetErrorString(e) + " zeroing the negative-result flag");
      s = ATS_ERR_CUDA;
    } else {
      s = plan_launch_resident(P, false, &d_rec->neg);
    }
  }
  P->profiling = prof;
  if (s != ATS_OK) return s;
  CUDA_TRY(cudaMemsetAsync(P->d_loop, 0, sizeof(int), st));
  if (P->n_tick > 0 && (s = plan_enqueue_loop(P, st, capture)) != ATS_OK) return s;
  CUDA_TRY(launch_final(P->d_solves, P->d_items, P->n_items, P->d_dst, &d_rec->neg, P->grid, st));
  CUDA_TRY(cudaMemcpyAsync(&d_rec->sc, P->d_final, sizeof(SolveScalars), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(launch_gather_flags(P->d_flag_ptrs, 1, &d_rec->flag, st));
  CUDA_TRY(cudaMemcpyAsync(&d_rec->chunks, P->d_loop, sizeof(int), cudaMemcpyDeviceToDevice, st));
  *check_every = o.check_every;
  *max_ticks = mt;
  return ATS_OK;
}

ats_status deferred_result(const DeferredRec &r, int check_every, int64_t max_ticks, ats_solve_stats *out) {
  int status = r.sc.status;
  if (r.flag) status = ATS_ERR_BAD_INPUT;
  else if ((int64_t)r.chunks * check_every >= max_ticks && r.sc.phase != kDone) status = ATS_ERR_TIMEOUT;
  if (status == ATS_OK && r.neg) status = ATS_WARN_NEGATIVE;
  if (out) {
    out->status = status;
    out->iterations = r.sc.iters;
    out->refinements = r.sc.refines;
    out->ticks = r.sc.ticks;
    out->r0_norm = r.sc.r0;
    out->res_norm = r.sc.rnorm;
    out->x_norm = r.sc.xnorm;
    out->err_bound = r.sc.xnorm > 0.0 ? r.sc.rnorm / r.sc.xnorm : 0.0;
  }
  return status;
}

}  // namespace ats

extern "C" {

ats_status ats_solve(ats_level *L, const double *rhs, double *x_inout, const ats_solve_opts *opts,
                     ats_solve_stats *stats) {
  try {  // no C++ exception leaves the library
    if (!L || !x_inout) {
      set_error("null argument");
      return ATS_ERR_INVALID_ARG;
    }
    if (!L->built) {
      set_error("level operator not built");
      return ATS_ERR_INVALID_ARG;
    }
    ats_solve_opts o = normalize(opts);
    ats_context *ctx = L->ctx;
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    ats_status s;
    // (re)use the cached single-solve plan when its options match
    if (L->solo && (std::memcmp(&L->solo->opts, &o, sizeof(o)) != 0 ||
                    L->solo->fp64 != (o.precision == ATS_PREC_FP64))) {
      plan_free(L->solo);
      L->solo = nullptr;
    }
    if (!L->solo) {
      ats_level *arr[1] = {L};
      if ((s = plan_create(ctx, arr, 1, &o, &L->solo)) != ATS_OK) return s;
    }
    if (rhs) {
      if (!L->rhs_save && (s = dev_alloc_t(ctx, L->N, &L->rhs_save)) != ATS_OK) return s;
      CUDA_TRY(cudaMemcpyAsync(L->rhs_save, L->b64, sizeof(double) * L->N, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(cudaMemcpyAsync(L->b64, rhs, sizeof(double) * L->N, kind_of(o.mem, true), st));
    }
    double *xs[1] = {x_inout};
    s = plan_run(L->solo, xs, stats);
    if (rhs) {
      cudaMemcpyAsync(L->b64, L->rhs_save, sizeof(double) * L->N, cudaMemcpyDeviceToDevice, st);
      cudaStreamSynchronize(st);
    }
    return s;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_batch_create(ats_context *ctx, ats_level *const *levels, int n, const ats_solve_opts *opts,
                            ats_batch **out) {
  try {  // no C++ exception leaves the library
    if (!out) return ATS_ERR_INVALID_ARG;
    *out = nullptr;
    Plan *P = nullptr;
    ats_status s = plan_create(ctx, levels, n, opts, &P);
    if (s != ATS_OK) return s;
    ats_batch *B = new (std::nothrow) ats_batch();
    if (!B) {
      plan_free(P);
      return ATS_ERR_OOM;
    }
    B->plan = P;
    *out = B;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_batch_solve(ats_batch *B, double *const *x_inout, ats_solve_stats *stats) {
  try {  // no C++ exception leaves the library
    if (!B || !B->plan) return ATS_ERR_INVALID_ARG;
    for (ats_level *L : B->plan->levels) {
      if (!L->built) {
        set_error("level operator not built");
        return ATS_ERR_INVALID_ARG;
      }
    }
    return plan_run(B->plan, x_inout, stats);
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_batch_destroy(ats_batch *B) {
  try {  // no C++ exception leaves the library
    if (!B) return ATS_ERR_INVALID_ARG;
    if (B->plan) {
      ats_context *ctx = B->plan->ctx;
      cudaSetDevice(ctx->device);
      cudaStreamSynchronize(ctx->stream);
      dev_free(ctx, B->d_args);
      dev_free(ctx, B->d_blk_level);
      dev_free(ctx, B->d_blk_first);
      if (B->copy_st) cudaStreamSynchronize(B->copy_st);
      for (auto &set : B->stage_cell)
        for (double *p : set) dev_free(ctx, p);
      for (auto &set : B->stage_face)
        for (double *p : set) dev_free(ctx, p);
      if (B->copied) cudaEventDestroy(B->copied);
      if (B->released) cudaEventDestroy(B->released);
      if (B->copy_st) cudaStreamDestroy(B->copy_st);
      plan_free(B->plan);
    }
    delete B;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_batch_run(ats_context *ctx, ats_level *const *levels, int n, double *const *x_inout,
                         const ats_solve_opts *opts, ats_solve_stats *stats) {
  try {  // no C++ exception leaves the library
    ats_batch *B = nullptr;
    ats_status s = ats_batch_create(ctx, levels, n, opts, &B);
    if (s != ATS_OK) return s;
    s = ats_batch_solve(B, x_inout, stats);
    ats_batch_destroy(B);
    return s;
  } catch (...) {
    return ats::abi_exception();
  }
}

}  // extern "C"

namespace {

// The host arrays of a batch's coefficient descriptors (7 per level; null for
// device arrays or absent ones), to recognise the arrays of a prefetch.
std::vector<const double *> batch_host_ptrs(const ats_coef_desc *coefs, int n) {
  std::vector<const double *> out;
  out.reserve(7 * (size_t)n);
  for (int k = 0; k < n; ++k) {
    const ats_coef_desc &c = coefs[k];
    const bool h = c.mem == ATS_MEM_HOST;
    for (const double *p : {c.K, c.E_old, c.s, c.src, c.face_K, c.face_E, c.face_F}) out.push_back(h ? p : nullptr);
  }
  return out;
}

// Stage the host arrays of coefs in staging set `set` (allocated on first
// use), one copy per run of levels whose host arrays are contiguous, on
// stream st (copy = false: the arrays are already there); dc[k] gets the
// device pointers.
ats_status batch_stage(ats_batch *B, const ats_coef_desc *coefs, int set, cudaStream_t st, bool copy,
                       ats_coef_desc *dc) {
  Plan *P = B->plan;
  ats_context *ctx = P->ctx;
  const int n = P->n;
  ats_status s;
  std::vector<int64_t> oc(n + 1, 0), of(n + 1, 0);
  for (int k = 0; k < n; ++k) {
    oc[k + 1] = oc[k] + P->levels[k]->N;
    of[k + 1] = of[k] + P->levels[k]->n_face;
  }
  const double *ats_coef_desc::*cell_kind[4] = {&ats_coef_desc::K, &ats_coef_desc::E_old, &ats_coef_desc::s,
                                                &ats_coef_desc::src};
  const double *ats_coef_desc::*face_kind[3] = {&ats_coef_desc::face_K, &ats_coef_desc::face_E,
                                                &ats_coef_desc::face_F};
  std::vector<double *> hp(n);
  for (int q = 0; q < 7; ++q) {
    const bool cell = q < 4;
    const double *ats_coef_desc::*m = cell ? cell_kind[q] : face_kind[q - 4];
    const std::vector<int64_t> &o = cell ? oc : of;
    bool any = false;
    for (int k = 0; k < n; ++k) {
      const bool h = coefs[k].mem == ATS_MEM_HOST && coefs[k].*m && o[k + 1] > o[k];
      hp[k] = h ? const_cast<double *>(coefs[k].*m) : nullptr;
      any = any || h;
    }
    if (!any) continue;
    double *&stage = cell ? B->stage_cell[set][q] : B->stage_face[set][q - 4];
    if (!stage && (s = dev_alloc_t(ctx, std::max<int64_t>(1, o[n]), &stage)) != ATS_OK) return s;
    if (copy && (s = copy_runs(st, true, stage, o.data(), n, hp.data())) != ATS_OK) return s;
    for (int k = 0; k < n; ++k)
      if (hp[k]) dc[k].*m = stage + o[k];
  }
  for (int k = 0; k < n; ++k) dc[k].mem = ATS_MEM_DEVICE;
  return ATS_OK;
}

}  // namespace

extern "C" {

ats_status ats_batch_build_operators(ats_batch *B, const ats_coef_desc *coefs) {
  try {  // no C++ exception leaves the library
    if (!B || !B->plan || !coefs) {
      set_error("null argument");
      return ATS_ERR_INVALID_ARG;
    }
    Plan *P = B->plan;
    ats_context *ctx = P->ctx;
    const int n = P->n;
    cudaStream_t st = ctx->stream;
    ats_status s;
    std::vector<CoefArgs> args(n);
    std::vector<ats_coef_desc> dc(coefs, coefs + n);
    bool any_host = false;
    for (int k = 0; k < n; ++k) any_host = any_host || coefs[k].mem == ATS_MEM_HOST;
    bool from_prefetch = false;
    if (any_host) {
      // host inputs go to the set not used by the last build (the last solve may
      // still read that one's E_old); a matching prefetch has copied them already
      CUDA_TRY(cudaSetDevice(ctx->device));
      const int set = B->cur_set ^ 1;
      from_prefetch = B->prefetched && batch_host_ptrs(coefs, n) == B->pf_ptrs;
      if (from_prefetch) CUDA_TRY(cudaStreamWaitEvent(st, B->copied, 0));
      else if (B->prefetched && B->copy_st) CUDA_TRY(cudaStreamSynchronize(B->copy_st));  // a stale prefetch
      if ((s = batch_stage(B, coefs, set, st, !from_prefetch, dc.data())) != ATS_OK) return s;
      B->cur_set = set;
    }
    B->prefetched = false;
    for (int k = 0; k < n; ++k) {
      s = prepare_operator(P->levels[k], &dc[k], &args[k]);
      if (s != ATS_OK) return s;
    }
    if (!B->d_args) {
      if ((s = dev_alloc_t(ctx, n, &B->d_args)) != ATS_OK) return s;
      std::vector<int32_t> first(n + 1, 0), level;
      for (int k = 0; k < n; ++k) {
        const int64_t nb = (P->levels[k]->N + kCoefThreads - 1) / kCoefThreads;
        first[k + 1] = first[k] + (int32_t)nb;
        for (int64_t b = 0; b < nb; ++b) level.push_back(k);
      }
      B->n_blocks = first[n];
      if ((s = dev_alloc_t(ctx, n + 1, &B->d_blk_first)) != ATS_OK) return s;
      if ((s = dev_alloc_t(ctx, std::max<int64_t>(1, B->n_blocks), &B->d_blk_level)) != ATS_OK) return s;
      CUDA_TRY(cudaMemcpyAsync(B->d_blk_first, first.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
      if (B->n_blocks)
        CUDA_TRY(cudaMemcpyAsync(B->d_blk_level, level.data(), sizeof(int32_t) * B->n_blocks, cudaMemcpyHostToDevice, st));
      CUDA_TRY(cudaStreamSynchronize(st));  // the host tables go out of scope
    }
    // upload the per-level arguments only when they changed (same buffers and
    // dt from step to step is the common case)
    if (B->h_args.size() != (size_t)n || std::memcmp(B->h_args.data(), args.data(), sizeof(CoefArgs) * n) != 0) {
      B->h_args = args;
      CUDA_TRY(cudaMemcpyAsync(B->d_args, B->h_args.data(), sizeof(CoefArgs) * n, cudaMemcpyHostToDevice, st));
    }
    CUDA_TRY(launch_coef_build_batch(B->d_args, B->d_blk_level, B->d_blk_first, B->n_blocks, n, P->d_flag_ptrs, st));
    // host arrays: the caller may reuse them once the call returns
    if (from_prefetch) CUDA_TRY(cudaEventSynchronize(B->copied));
    else if (any_host) CUDA_TRY(cudaStreamSynchronize(st));
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_batch_prefetch_operators(ats_batch *B, const ats_coef_desc *coefs) {
  try {  // no C++ exception leaves the library
    if (!B || !B->plan || !coefs) {
      set_error("null argument");
      return ATS_ERR_INVALID_ARG;
    }
    Plan *P = B->plan;
    ats_context *ctx = P->ctx;
    const int n = P->n;
    bool any_host = false;
    for (int k = 0; k < n; ++k) any_host = any_host || coefs[k].mem == ATS_MEM_HOST;
    B->prefetched = false;
    if (!any_host) return ATS_OK;  // nothing to copy
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (!B->copy_st) {
      CUDA_TRY(cudaStreamCreateWithFlags(&B->copy_st, cudaStreamNonBlocking));
      CUDA_TRY(cudaEventCreateWithFlags(&B->copied, cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&B->released, cudaEventDisableTiming));
    }
    // the other set is free once the work queued so far on the context stream
    // (which read it two builds ago) has run
    CUDA_TRY(cudaEventRecord(B->released, ctx->stream));
    CUDA_TRY(cudaStreamWaitEvent(B->copy_st, B->released, 0));
    std::vector<ats_coef_desc> dc(coefs, coefs + n);
    ats_status s = batch_stage(B, coefs, B->cur_set ^ 1, B->copy_st, true, dc.data());
    if (s != ATS_OK) return s;
    CUDA_TRY(cudaEventRecord(B->copied, B->copy_st));
    B->pf_ptrs = batch_host_ptrs(coefs, n);
    B->prefetched = true;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_batch_set_profiling(ats_batch *B, int on) {
  try {  // no C++ exception leaves the library
    if (!B || !B->plan) return ATS_ERR_INVALID_ARG;
    B->plan->profiling = on != 0;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_batch_autotune(ats_batch *B, double *const *x_inout, const int *tiles, int n_tiles,
                              const int *checks, int n_checks, int reps, ats_tune_result *out) {
  try {  // no C++ exception leaves the library
    if (!B || !B->plan || !x_inout || n_tiles < 0 || n_checks < 0 || (n_tiles > 0 && !tiles) ||
        (n_checks > 0 && !checks)) {
      set_error("ats_batch_autotune: bad arguments");
      return ATS_ERR_INVALID_ARG;
    }
    Plan *P = B->plan;
    ats_context *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    const int n = P->n;
    const ats_solve_opts base = P->opts;
    const bool dev = base.mem == ATS_MEM_DEVICE;
    const bool restore = base.x0 == ATS_X0_GIVEN;  // every trial starts from the caller's x
    reps = std::max(1, reps);
    for (int k = 0; k < n; ++k) {
      if (!x_inout[k]) {
        set_error("x_inout[k] is NULL");
        return ATS_ERR_INVALID_ARG;
      }
      if (!P->levels[k]->built) {
        set_error("level operator not built");
        return ATS_ERR_INVALID_ARG;
      }
    }
    static const int kTiles[] = {0, 128, 256, 384, 512};
    static const int kChecks[] = {8, 16, 32};
    if (n_tiles == 0) {
      tiles = kTiles;
      n_tiles = (int)(sizeof(kTiles) / sizeof(kTiles[0]));
    }
    if (n_checks == 0) {
      checks = kChecks;
      n_checks = (int)(sizeof(kChecks) / sizeof(kChecks[0]));
    }
    for (int i = 0; i < n_tiles; ++i)
      if (tiles[i] < 0) {
        set_error("ats_batch_autotune: negative tile");
        return ATS_ERR_INVALID_ARG;
      }
    // the caller's x, kept for the trials to start from
    std::vector<int64_t> off(n + 1, 0);
    for (int k = 0; k < n; ++k) off[k + 1] = off[k] + P->levels[k]->N;
    double *dsave = nullptr;
    std::vector<double> hsave;
    ats_status s;
    if (restore) {
      if (dev) {
        if ((s = dev_alloc_t(ctx, std::max<int64_t>(1, off[n]), &dsave)) != ATS_OK) return s;
        for (int k = 0; k < n; ++k)
          CUDA_TRY(cudaMemcpyAsync(dsave + off[k], x_inout[k], sizeof(double) * (off[k + 1] - off[k]),
                                   cudaMemcpyDeviceToDevice, st));
      } else {
        hsave.resize((size_t)off[n]);
        for (int k = 0; k < n; ++k) std::memcpy(hsave.data() + off[k], x_inout[k], sizeof(double) * (off[k + 1] - off[k]));
      }
    }
    auto put_back = [&]() -> ats_status {
      if (!restore) return ATS_OK;
      for (int k = 0; k < n; ++k) {
        const size_t bytes = sizeof(double) * (off[k + 1] - off[k]);
        if (dev) CUDA_TRY(cudaMemcpyAsync(x_inout[k], dsave + off[k], bytes, cudaMemcpyDeviceToDevice, st));
        else std::memcpy(x_inout[k], hsave.data() + off[k], bytes);
      }
      return ATS_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // one plan per candidate: a warm-up solve (graph capture), then the fastest of reps solves
    auto time_plan = [&](Plan *Q, double *ms) -> ats_status {
      ats_status r;
      if ((r = put_back()) != ATS_OK) return r;
      if ((r = plan_run(Q, x_inout, nullptr)) != ATS_OK) return r;
      *ms = 1e300;
      for (int i = 0; i < reps; ++i) {
        if ((r = put_back()) != ATS_OK) return r;
        CUDA_TRY(cudaEventRecord(e0, st));
        if ((r = plan_run(Q, x_inout, nullptr)) != ATS_OK) return r;
        CUDA_TRY(cudaEventRecord(e1, st));
        CUDA_TRY(cudaEventSynchronize(e1));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        *ms = std::min(*ms, (double)t);
      }
      return ATS_OK;
    };
    ats_tune_result res;
    std::memset(&res, 0, sizeof(res));
    res.chosen = base;
    s = ATS_OK;
    const bool was_profiling = P->profiling;
    P->profiling = false;
    if ((s = time_plan(P, &res.ms_default)) == ATS_OK) {
      res.tile_octs = base.tile_octs;
      res.check_every = base.check_every;
      res.ms = res.ms_default;
      res.candidates = 1;
      res.res_threads = P->res_threads;
      res.res_cluster = P->res_cluster;
      res.res_cta_octs = base.res_cta_octs;
      // the candidates: work-item size x poll interval for the tick-path
      // solves, CTA threads x cluster size x one-CTA limit for the resident
      // ones, each with the batch's other options
      std::vector<ats_solve_opts> cands;
      if (P->n_tick > 0) {
        for (int i = 0; i < n_tiles; ++i)
          for (int j = 0; j < n_checks; ++j) {
            ats_solve_opts o = base;
            o.tile_octs = tiles[i];
            o.check_every = checks[j];
            if (o.tile_octs == base.tile_octs && normalize(&o).check_every == base.check_every) continue;
            cands.push_back(o);
          }
      }
      if (P->n_bq + P->n_mq + P->n_cq + P->n_tq > 0) {
        // (threads per CTA, cluster size, one-CTA limit, big-cluster size; -1 = none)
        static const int kShapes[][4] = {{512, 4, 2048, 16}, {512, 8, 2048, 16}, {512, 8, 2048, -1},
                                         {256, 4, 2048, 16}, {512, 4, 1024, 16}, {512, 2, 2048, 16},
                                         {512, 4, 2048, 8}, {512, 16, 2048, -1}};
        const int base_cta = base.res_cta_octs ? base.res_cta_octs : 2048;
        const int base_big = P->res_cluster_big > 0 ? P->res_cluster_big : -1;
        for (const auto &sh : kShapes) {
          if (sh[0] == P->res_threads && sh[1] == P->res_cluster && sh[2] == base_cta && sh[3] == base_big) continue;
          ats_solve_opts o = base;
          o.res_threads = sh[0];
          o.res_cluster = sh[1];
          o.res_cta_octs = sh[2];
          o.res_cluster_big = sh[3];
          cands.push_back(o);
        }
      }
      ats_solve_opts best = base;
      for (size_t i = 0; i < cands.size() && s == ATS_OK; ++i) {
        const ats_solve_opts &o = cands[i];
        Plan *Q = nullptr;
        if ((s = plan_create(ctx, P->levels.data(), n, &o, &Q)) != ATS_OK) break;
        double ms = 0.0;
        s = time_plan(Q, &ms);
        const int qth = Q->res_threads, qcl = Q->res_cluster;
        plan_free(Q);
        if (s != ATS_OK) break;
        ++res.candidates;
        if (ms < res.ms) {
          res.ms = ms;
          best = o;
          res.tile_octs = o.tile_octs;
          res.check_every = normalize(&o).check_every;
          res.res_threads = qth;
          res.res_cluster = qcl;
          res.res_cta_octs = o.res_cta_octs;
        }
      }
      res.chosen = best;
    }
    // the batch keeps the fastest configuration, and x_inout holds its solution
    if (s == ATS_OK && std::memcmp(&res.chosen, &base, sizeof(base)) != 0) {
      ats_solve_opts o = res.chosen;
      Plan *Q = nullptr;
      if ((s = plan_create(ctx, P->levels.data(), n, &o, &Q)) == ATS_OK) {
        plan_free(P);
        B->plan = P = Q;
      }
    }
    P->profiling = was_profiling;
    if (s == ATS_OK && (s = put_back()) == ATS_OK) s = plan_run(P, x_inout, nullptr);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (dsave) {
      cudaStreamSynchronize(st);
      dev_free(ctx, dsave);
    }
    if (s == ATS_OK && out) *out = res;
    return s;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_batch_kernel_stats(const ats_batch *B, ats_kernel_stats *out) {
  try {  // no C++ exception leaves the library
    if (!B || !B->plan || !out) return ATS_ERR_INVALID_ARG;
    const Plan *P = B->plan;
    out->op_ms = P->op_ms;
    out->op_bytes = P->op_bytes;
    out->ref_ms = P->ref_ms;
    out->ref_bytes = P->ref_bytes;
    out->upd_ms = P->upd_ms;
    out->upd_bytes = P->upd_bytes;
    out->launches = P->launches;
    out->ticks = P->ticks;
    out->res_ms = P->res_ms;
    out->res_bytes = P->res_bytes;
    out->res_launches = P->res_launches;
    out->res_solves = P->n_bq + P->n_mq + P->n_cq + P->n_tq + P->n_gq;
    out->res_span_ms = P->res_span_ms;
    out->res_longest_ms = P->res_longest_ms;
    out->res_occupancy = P->res_occupancy;
    out->res_longest = P->res_longest;
    out->res_grid = P->res_grid + P->res_grid_big + P->res_grid_mid + P->res_fill;
    for (int q = 0; q < 3; ++q) out->res_end_ms[q] = P->res_end_ms[q];
    out->res_grids[0] = P->res_grid_big + P->res_grid_mid;
    out->res_grids[1] = P->res_grid;
    out->res_grids[2] = P->res_fill;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

}  // extern "C"
