// Serving loop: continuous batching of level solves.
//
// Requests (one level solve each: topology, per-step values, tolerance) are
// queued by any thread.  A scheduler thread owns one private context and a
// fixed-capacity device plan (solve slots, a pool of work items, partials,
// active lists).  Between ticks it admits queued requests while slots, work
// items and the device-memory budget allow: the level is built, its solve
// descriptor and scalars are written into a free slot and its items are
// appended to the running tick's work list on the device (k_admit), so new
// solves join solves already in flight.  Every tick advances all resident
// solves by one step (the same k_op / k_ref / k_upd kernels, one CUDA graph
// of `check_every` ticks captured once).  Finished solves are found by
// polling their final state, copied back, and their memory released.  The
// arithmetic of a solve never involves another solve, so its result is the
// same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ats_internal.h"

using namespace ats;

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  uint64_t ticket = 0;
  // host copies of the request
  std::vector<int32_t> oct_xyz;
  std::vector<uint8_t> leaf;
  bool has_leaf = false;
  double dx = 0.0, dt = 0.0;
  std::vector<int32_t> face_cell;
  std::vector<int8_t> face_dir, face_kind, face_rel;
  std::vector<double> face_alpha, K, E, s, src, face_K, face_E, face_F, x0;
  int integrator = ATS_INTEGRATOR_BACKWARD_EULER;
  double tol = 1e-10;
  int stop_rule = ATS_STOP_RESIDUAL;
  Clock::time_point submitted;
  size_t bytes = 0;  // device-memory estimate
  Layout layout;     // built by the submitting thread, off the device loop
};

struct Slot {
  bool used = false;
  uint64_t ticket = 0;
  ats_level *lvl = nullptr;
  int item_begin = 0, n_items = 0;
  size_t bytes = 0;
  Clock::time_point submitted, admitted;
};

struct Done {
  ats_status status = ATS_OK;
  ats_solve_stats stats{};
  std::vector<double> x;
  double latency_us = 0.0, queue_us = 0.0;
};

// first-fit allocator of contiguous work-item ranges
struct ItemPool {
  std::map<int, int> free_;  // begin -> length
  explicit ItemPool(int cap) { free_[0] = cap; }
  int alloc(int n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const int b = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[b + n] = len - n;
        return b;
      }
    }
    return -1;
  }
  void release(int b, int n) {
    auto it = free_.emplace(b, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

size_t estimate_bytes(const Pending &p, bool fp64) {
  const size_t n_oct = p.oct_xyz.size() / 3;
  const size_t N = 8 * n_oct;
  const size_t w = fp64 ? 8 : 4;
  // topology, operator (K64, K32, b64, xd), staging (4 N + faces), x64,
  // four CG vectors, faces
  return n_oct * (24 + 4 + 1) + N * (8 + 4 + 8 + 12) + N * 8 * 4 + N * 8 + 4 * N * w + p.face_cell.size() * 60 +
         ((size_t)1 << 16);
}

}  // namespace

struct ats_server {
  ats_context *ctx = nullptr;
  ats_solve_opts opts{};
  bool fp64 = false;
  int max_slots = 0, max_items = 0;
  int grids[3] = {1, 1, 1};  // tick kernels: k_op, k_ref, k_upd
  size_t budget = 0, resident = 0;
  // device plan
  SolveDev *d_solves = nullptr;
  SolveScalars *d_sc = nullptr, *d_final = nullptr;
  WorkItem *d_items = nullptr;
  int32_t *d_lists = nullptr, *d_admit = nullptr;
  double *d_part = nullptr;
  TickCtl *d_ctl = nullptr;
  int *d_active = nullptr;
  TickArgs targs{};
  cudaGraphExec_t exec = nullptr;
  SolveScalars *h_final = nullptr;  // pinned
  int *h_active = nullptr;          // pinned
  cudaStream_t st = nullptr;
  TickStreams fj{nullptr, nullptr, nullptr};  // k_ref's stream, fork / join events
  // host state
  std::vector<Slot> slots;
  std::unique_ptr<ItemPool> pool;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Pending>> queue;
  std::map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  std::string fatal;
  // statistics
  uint64_t completed = 0;
  int64_t ticks = 0;
  int peak_resident = 0;
};

namespace {

#define S_TRY(expr)                                                                   \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      set_error(std::string("CUDA error: ") + cudaGetErrorString(_e) + " at " #expr); \
      return ATS_ERR_CUDA;                                                            \
    }                                                                                 \
  } while (0)

// Build the level of a request and place it in a free slot (scheduler thread).
ats_status admit_one_impl(ats_server *S, Pending &p, int slot, std::vector<int32_t> &new_slots);

// Admit one request into a free slot; on failure everything it took is
// released again.  ATS_ERR_OVER_BUDGET: no contiguous run of work items now.
ats_status admit_one(ats_server *S, Pending &p, int slot, std::vector<int32_t> &new_slots) {
  Slot &sl = S->slots[slot];
  sl.lvl = nullptr;
  sl.n_items = 0;
  sl.item_begin = -1;
  ats_status s = admit_one_impl(S, p, slot, new_slots);
  if (s != ATS_OK) {
    if (sl.lvl) ats_level_destroy(sl.lvl);
    sl.lvl = nullptr;
    if (sl.item_begin >= 0 && sl.n_items > 0) S->pool->release(sl.item_begin, sl.n_items);
    sl.n_items = 0;
    sl.item_begin = -1;
    sl.used = false;
  }
  return s;
}

ats_status admit_one_impl(ats_server *S, Pending &p, int slot, std::vector<int32_t> &new_slots) {
  Slot &sl = S->slots[slot];
  ats_level_desc d;
  std::memset(&d, 0, sizeof(d));
  d.n_oct = (int64_t)p.oct_xyz.size() / 3;
  d.oct_xyz = p.oct_xyz.data();
  d.leaf_mask = p.has_leaf ? p.leaf.data() : nullptr;
  d.dx = p.dx;
  d.n_face = (int64_t)p.face_cell.size();
  d.face_cell = p.face_cell.data();
  d.face_dir = p.face_dir.data();
  d.face_kind = p.face_kind.data();
  d.face_rel = p.face_rel.data();
  d.face_alpha = p.face_alpha.empty() ? nullptr : p.face_alpha.data();
  ats_status s = level_create_with_layout(S->ctx, &d, p.layout, &sl.lvl);
  if (s != ATS_OK) return s;
  ats_coef_desc c;
  std::memset(&c, 0, sizeof(c));
  c.dt = p.dt;
  c.integrator = p.integrator;
  c.mem = ATS_MEM_HOST;
  c.K = p.K.data();
  c.E_old = p.E.data();
  c.s = p.s.empty() ? nullptr : p.s.data();
  c.src = p.src.empty() ? nullptr : p.src.data();
  c.face_K = p.face_K.empty() ? nullptr : p.face_K.data();
  c.face_E = p.face_E.empty() ? nullptr : p.face_E.data();
  c.face_F = p.face_F.empty() ? nullptr : p.face_F.data();
  if ((s = ats_level_build_operator(sl.lvl, &c)) != ATS_OK) return s;
  const int tile = tile_for(d.n_oct, S->opts.tile_octs, S->grids[0]);
  const int n_items = (int)((d.n_oct + tile - 1) / tile);
  if (n_items > S->max_items) {
    set_error("request needs more work items than the server holds");
    return ATS_ERR_INVALID_ARG;
  }
  const int ib = S->pool->alloc(n_items);
  if (ib < 0) return ATS_ERR_OVER_BUDGET;
  sl.item_begin = ib;
  sl.n_items = n_items;
  ats_solve_opts o = S->opts;
  o.tol = p.tol;
  o.stop_rule = p.stop_rule;
  SolveDev sd;
  if ((s = solve_dev_for(sl.lvl, o, S->fp64, ib, n_items, &sd)) != ATS_OK) return s;
  std::vector<WorkItem> items(n_items);
  for (int k = 0; k < n_items; ++k) {
    items[k].solve = slot;
    items[k].oct_begin = k * tile;
    items[k].n_oct = (int32_t)std::min<int64_t>(tile, d.n_oct - (int64_t)k * tile);
    items[k].pad = 0;
  }
  SolveScalars sc;
  std::memset(&sc, 0, sizeof(sc));
  sc.phase = kRefine;
  sc.status = ATS_OK;
  cudaStream_t st = S->st;
  const int64_t N = 8 * d.n_oct;
  const double *x0 = p.x0.empty() ? p.E.data() : p.x0.data();
  S_TRY(cudaMemcpyAsync(level_x64(sl.lvl), x0, sizeof(double) * N, cudaMemcpyHostToDevice, st));
  S_TRY(cudaMemsetAsync((void *)sd.e, 0, (S->fp64 ? 8 : 4) * N, st));
  S_TRY(cudaMemcpyAsync(S->d_solves + slot, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
  S_TRY(cudaMemcpyAsync(S->d_sc + slot, &sc, sizeof(sc), cudaMemcpyHostToDevice, st));
  S_TRY(cudaMemcpyAsync(S->d_sc + S->max_slots + slot, &sc, sizeof(sc), cudaMemcpyHostToDevice, st));
  S_TRY(cudaMemcpyAsync(S->d_final + slot, &sc, sizeof(sc), cudaMemcpyHostToDevice, st));
  S_TRY(cudaMemcpyAsync(S->d_items + ib, items.data(), sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice, st));
  S_TRY(cudaStreamSynchronize(st));  // host buffers of this request are about to go away
  sl.used = true;
  sl.ticket = p.ticket;
  sl.bytes = p.bytes;
  sl.submitted = p.submitted;
  sl.admitted = Clock::now();
  new_slots.push_back(slot);
  return ATS_OK;
}

void retire(ats_server *S, int slot, const SolveScalars &fin) {
  Slot &sl = S->slots[slot];
  Done dn;
  const int64_t N = level_cells(sl.lvl);
  dn.x.resize(N);
  if (const double *base = level_cn_base(sl.lvl))  // Crank-Nicolson: E^{n+1} = 2 x - E^n
    launch_cn_extrapolate(N, level_x64(sl.lvl), base, level_x64(sl.lvl), S->st);
  cudaMemcpyAsync(dn.x.data(), level_x64(sl.lvl), sizeof(double) * N, cudaMemcpyDeviceToHost, S->st);
  cudaStreamSynchronize(S->st);
  dn.status = fin.status;  // the negative-energy warning is found by the waiting thread
  dn.stats.status = fin.status;
  dn.stats.iterations = fin.iters;
  dn.stats.refinements = fin.refines;
  dn.stats.ticks = fin.ticks;
  dn.stats.r0_norm = fin.r0;
  dn.stats.res_norm = fin.rnorm;
  dn.stats.x_norm = fin.xnorm;
  dn.stats.err_bound = fin.xnorm > 0.0 ? fin.rnorm / fin.xnorm : 0.0;
  const auto now = Clock::now();
  dn.latency_us = std::chrono::duration<double, std::micro>(now - sl.submitted).count();
  dn.queue_us = std::chrono::duration<double, std::micro>(sl.admitted - sl.submitted).count();
  ats_level_destroy(sl.lvl);
  sl.lvl = nullptr;
  S->pool->release(sl.item_begin, sl.n_items);
  sl.used = false;
  std::lock_guard<std::mutex> lk(S->mu);
  S->resident -= sl.bytes;
  S->done[sl.ticket] = std::move(dn);
  S->completed += 1;
  S->cv_done.notify_all();
}

ats_status capture_graph(ats_server *S) {
  cudaGraph_t g = nullptr;
  S_TRY(cudaStreamBeginCapture(S->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int t = 0; t < S->opts.check_every && err == cudaSuccess; ++t)
    err = launch_tick(S->fp64, false, S->targs, S->grids, S->st, &S->fj, nullptr, true);
  cudaError_t err2 = cudaStreamEndCapture(S->st, &g);
  if (err != cudaSuccess || err2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    set_error("server graph capture failed");
    return ATS_ERR_CUDA;
  }
  err = cudaGraphInstantiate(&S->exec, g, 0);
  cudaGraphDestroy(g);
  if (err != cudaSuccess) {
    S->exec = nullptr;
    set_error("server graph instantiate failed");
    return ATS_ERR_CUDA;
  }
  return ATS_OK;
}

void fail_all(ats_server *S, ats_status code, const std::string &msg) {
  std::lock_guard<std::mutex> lk(S->mu);
  S->fatal = msg;
  for (auto &p : S->queue) {
    Done dn;
    dn.status = code;
    S->done[p->ticket] = std::move(dn);
  }
  S->queue.clear();
  for (auto &sl : S->slots) {
    if (!sl.used) continue;
    Done dn;
    dn.status = code;
    S->done[sl.ticket] = std::move(dn);
    sl.used = false;
  }
  S->cv_done.notify_all();
}

void worker_loop(ats_server *S) {
  cudaSetDevice(ctx_device(S->ctx));
  ats_status s = capture_graph(S);
  if (s != ATS_OK) {
    fail_all(S, s, "graph capture failed");
    return;
  }
  int n_res = 0;  // resident solves
  for (;;) {
    // ---- admission (continuous batching) ----
    std::vector<int32_t> new_slots;
    for (;;) {
      std::unique_ptr<Pending> p;
      {
        std::unique_lock<std::mutex> lk(S->mu);
        if (n_res == 0 && S->queue.empty() && !S->stop) S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
        if (S->stop && S->queue.empty() && n_res == 0) return;
        if (S->queue.empty()) break;
        Pending &front = *S->queue.front();
        if (front.bytes > S->budget) {
          // can never fit: reject
          Done dn;
          dn.status = ATS_ERR_OVER_BUDGET;
          S->done[front.ticket] = std::move(dn);
          S->queue.pop_front();
          S->cv_done.notify_all();
          continue;
        }
        if (S->resident + front.bytes > S->budget) break;  // wait for memory to free up
        int slot = -1;
        for (int k = 0; k < S->max_slots; ++k)
          if (!S->slots[k].used) {
            slot = k;
            break;
          }
        if (slot < 0) break;
        p = std::move(S->queue.front());
        S->queue.pop_front();
        S->resident += p->bytes;
        lk.unlock();
        ats_status a = admit_one(S, *p, slot, new_slots);
        if (a != ATS_OK) {
          std::lock_guard<std::mutex> lk2(S->mu);
          S->resident -= p->bytes;
          const bool transient = (a == ATS_ERR_OVER_BUDGET || a == ATS_ERR_OOM) && n_res > 0;
          if (transient) {
            // no room right now (work items or device memory): retry after
            // resident solves finish
            S->queue.push_front(std::move(p));
            break;
          }
          Done dn;
          dn.status = a;
          S->done[p->ticket] = std::move(dn);
          S->cv_done.notify_all();
          continue;
        }
        ++n_res;
      }
    }
    if (!new_slots.empty()) {
      cudaMemcpyAsync(S->d_admit, new_slots.data(), sizeof(int32_t) * new_slots.size(), cudaMemcpyHostToDevice,
                      S->st);
      if (launch_admit(S->targs, S->d_admit, (int)new_slots.size(), S->st) != cudaSuccess) {
        fail_all(S, ATS_ERR_CUDA, "admit kernel failed");
        return;
      }
      std::lock_guard<std::mutex> lk(S->mu);
      S->peak_resident = std::max(S->peak_resident, n_res);
    }
    if (n_res == 0) continue;
    // ---- one poll interval of ticks ----
    if (cudaGraphLaunch(S->exec, S->st) != cudaSuccess) {
      fail_all(S, ATS_ERR_CUDA, "graph launch failed");
      return;
    }
    S->ticks += S->opts.check_every;
    cudaMemcpyAsync(S->h_final, S->d_final, sizeof(SolveScalars) * S->max_slots, cudaMemcpyDeviceToHost, S->st);
    if (cudaStreamSynchronize(S->st) != cudaSuccess) {
      fail_all(S, ATS_ERR_CUDA, "tick failed");
      return;
    }
    for (int k = 0; k < S->max_slots; ++k) {
      if (S->slots[k].used && S->h_final[k].phase == kDone) {
        retire(S, k, S->h_final[k]);
        --n_res;
      }
    }
  }
}

}  // namespace

extern "C" {

ats_status ats_server_create(int device, size_t mem_budget_bytes, const ats_server_opts *so, ats_server **out) {
  try {  // no C++ exception leaves the library
    if (!out) return ATS_ERR_INVALID_ARG;
    *out = nullptr;
    ats_server_opts defaults;
    std::memset(&defaults, 0, sizeof(defaults));
    const ats_server_opts &o = so ? *so : defaults;
    ats_server *S = new (std::nothrow) ats_server();
    if (!S) return ATS_ERR_OOM;
    ats_status s = ats_context_create(device, 0, &S->ctx);
    if (s != ATS_OK) {
      delete S;
      return s;
    }
    S->opts = normalized_opts(&o.solve);
    S->fp64 = S->opts.precision == ATS_PREC_FP64;
    S->max_slots = o.max_slots > 0 ? o.max_slots : 1024;
    S->max_items = o.max_items > 0 ? o.max_items : 1 << 16;
    S->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)1 << 40;
    S->slots.resize(S->max_slots);
    S->pool.reset(new ItemPool(S->max_items));
    S->st = ctx_stream(S->ctx);
    auto fail = [&](ats_status code) {
      ats_server_destroy(S);
      return code;
    };
    if (cudaStreamCreateWithFlags(&S->fj.aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->fj.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->fj.join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      set_error("server: stream or event creation failed");
      return fail(ATS_ERR_CUDA);
    }
    void *p;
    const size_t ms = S->max_slots, mi = S->max_items;
    if ((s = ctx_alloc(S->ctx, sizeof(SolveDev) * ms, &p)) != ATS_OK) return fail(s);
    S->d_solves = (SolveDev *)p;
    if ((s = ctx_alloc(S->ctx, sizeof(SolveScalars) * 2 * ms, &p)) != ATS_OK) return fail(s);
    S->d_sc = (SolveScalars *)p;
    if ((s = ctx_alloc(S->ctx, sizeof(SolveScalars) * ms, &p)) != ATS_OK) return fail(s);
    S->d_final = (SolveScalars *)p;
    if ((s = ctx_alloc(S->ctx, sizeof(WorkItem) * mi, &p)) != ATS_OK) return fail(s);
    S->d_items = (WorkItem *)p;
    if ((s = ctx_alloc(S->ctx, sizeof(int32_t) * 4 * mi, &p)) != ATS_OK) return fail(s);
    S->d_lists = (int32_t *)p;
    if ((s = ctx_alloc(S->ctx, sizeof(int32_t) * ms, &p)) != ATS_OK) return fail(s);
    S->d_admit = (int32_t *)p;
    if ((s = ctx_alloc(S->ctx, sizeof(double) * kNumPartials * 3 * mi, &p)) != ATS_OK) return fail(s);
    S->d_part = (double *)p;
    if ((s = ctx_alloc(S->ctx, sizeof(TickCtl), &p)) != ATS_OK) return fail(s);
    S->d_ctl = (TickCtl *)p;
    if ((s = ctx_alloc(S->ctx, sizeof(int), &p)) != ATS_OK) return fail(s);
    S->d_active = (int *)p;
    if (cudaMallocHost(&S->h_final, sizeof(SolveScalars) * ms) != cudaSuccess) return fail(ATS_ERR_OOM);
    TickCtl c0;
    std::memset(&c0, 0, sizeof(c0));
    std::vector<SolveScalars> done_init(ms);
    for (auto &x : done_init) {
      std::memset(&x, 0, sizeof(x));
      x.phase = kDone;
    }
    const int zero = 0;
    if (cudaMemcpyAsync(S->d_ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, S->st) != cudaSuccess ||
        cudaMemcpyAsync(S->d_active, &zero, sizeof(int), cudaMemcpyHostToDevice, S->st) != cudaSuccess ||
        cudaMemcpyAsync(S->d_final, done_init.data(), sizeof(SolveScalars) * ms, cudaMemcpyHostToDevice, S->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(S->st) != cudaSuccess)
      return fail(ATS_ERR_CUDA);
    TickArgs &t = S->targs;
    t.solves = S->d_solves;
    t.sbuf = S->d_sc;
    t.final_sc = S->d_final;
    t.items = S->d_items;
    t.lists = S->d_lists;
    t.n_items = S->max_items;
    t.n_solves = S->max_slots;
    t.ctl = S->d_ctl;
    t.p_op = S->d_part;
    t.p_upd = S->d_part + (size_t)kNumPartials * mi;
    t.n_active = S->d_active;
    t.cells = nullptr;
    tick_grids(S->fp64, false, device, S->grids);
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_server_submit(ats_server *S, const ats_request *r, uint64_t *ticket) {
  try {  // no C++ exception leaves the library
    if (!S || !r || !r->level || !r->coef || !ticket) {
      set_error("ats_server_submit: null argument");
      return ATS_ERR_INVALID_ARG;
    }
    const ats_level_desc &d = *r->level;
    const ats_coef_desc &c = *r->coef;
    if (c.mem != ATS_MEM_HOST || d.n_oct <= 0 || !d.oct_xyz || !c.K || !c.E_old || !(c.dt > 0.0)) {
      set_error("ats_server_submit: request arrays must be host arrays with n_oct > 0, K, E_old and dt > 0");
      return ATS_ERR_INVALID_ARG;
    }
    if ((c.integrator != ATS_INTEGRATOR_BACKWARD_EULER && c.integrator != ATS_INTEGRATOR_CRANK_NICOLSON) ||
        (c.integrator == ATS_INTEGRATOR_CRANK_NICOLSON && c.s)) {
      set_error("ats_server_submit: unknown integrator, or a shift s with Crank-Nicolson");
      return ATS_ERR_INVALID_ARG;
    }
    std::unique_ptr<Pending> p(new (std::nothrow) Pending());
    if (!p) return ATS_ERR_OOM;
    const size_t n = (size_t)d.n_oct, N = 8 * n, nf = (size_t)d.n_face;
    p->oct_xyz.assign(d.oct_xyz, d.oct_xyz + 3 * n);
    if (d.leaf_mask) {
      p->leaf.assign(d.leaf_mask, d.leaf_mask + n);
      p->has_leaf = true;
    }
    p->dx = d.dx;
    p->dt = c.dt;
    if (nf) {
      p->face_cell.assign(d.face_cell, d.face_cell + nf);
      p->face_dir.assign(d.face_dir, d.face_dir + nf);
      p->face_kind.assign(d.face_kind, d.face_kind + nf);
      p->face_rel.assign(d.face_rel, d.face_rel + nf);
      if (d.face_alpha) p->face_alpha.assign(d.face_alpha, d.face_alpha + nf);
      if (c.face_K) p->face_K.assign(c.face_K, c.face_K + nf);
      if (c.face_E) p->face_E.assign(c.face_E, c.face_E + nf);
      if (c.face_F) p->face_F.assign(c.face_F, c.face_F + nf);
    }
    p->K.assign(c.K, c.K + N);
    p->E.assign(c.E_old, c.E_old + N);
    if (c.s) p->s.assign(c.s, c.s + N);
    if (c.src) p->src.assign(c.src, c.src + N);
    if (r->x0) p->x0.assign(r->x0, r->x0 + N);
    p->integrator = c.integrator;
    if (r->x0 && p->integrator == ATS_INTEGRATOR_CRANK_NICOLSON)
      for (size_t i = 0; i < N; ++i) p->x0[i] = 0.5 * (p->x0[i] + p->E[i]);  // guess of the half-step root
    p->tol = r->tol > 0.0 ? r->tol : 1e-10;
    p->stop_rule = r->stop_rule;
    p->submitted = Clock::now();
    p->bytes = estimate_bytes(*p, S->fp64);
    {
      // the host part of level creation (neighbour table, interface records) runs
      // in the submitting thread, so the scheduler only uploads
      ats_level_desc dd = d;
      dd.oct_xyz = p->oct_xyz.data();
      dd.leaf_mask = p->has_leaf ? p->leaf.data() : nullptr;
      dd.face_cell = p->face_cell.data();
      dd.face_dir = p->face_dir.data();
      dd.face_kind = p->face_kind.data();
      dd.face_rel = p->face_rel.data();
      dd.face_alpha = p->face_alpha.empty() ? nullptr : p->face_alpha.data();
      std::string msg = build_layout(dd, p->layout);
      if (!msg.empty()) {
        set_error("ats_server_submit: " + msg);
        return ATS_ERR_INVALID_ARG;
      }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->fatal.empty()) {
      set_error("server failed: " + S->fatal);
      return ATS_ERR_CUDA;
    }
    p->ticket = S->next_ticket++;
    *ticket = p->ticket;
    S->queue.push_back(std::move(p));
    S->cv_work.notify_one();
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_server_wait(ats_server *S, uint64_t ticket, int64_t timeout_us, double *x_out, ats_result *res) {
  try {  // no C++ exception leaves the library
    if (!S) return ATS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return S->done.count(ticket) > 0; };
    if (timeout_us < 0) {
      S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
      set_error("ats_server_wait: timed out");
      return ATS_ERR_TIMEOUT;
    }
    Done dn = std::move(S->done[ticket]);
    S->done.erase(ticket);
    lk.unlock();
    if (dn.status == ATS_OK)  // a negative energy in the result: the warning of the solve (here, off the scheduler)
      for (double v : dn.x)
        if (v < 0.0) {
          dn.status = ATS_WARN_NEGATIVE;
          dn.stats.status = ATS_WARN_NEGATIVE;
          break;
        }
    if (x_out && !dn.x.empty()) std::memcpy(x_out, dn.x.data(), sizeof(double) * dn.x.size());
    if (res) {
      res->status = dn.status;
      res->stats = dn.stats;
      res->latency_us = dn.latency_us;
      res->queue_us = dn.queue_us;
    }
    return dn.status;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_server_stats(ats_server *S, ats_server_counters *out) {
  try {  // no C++ exception leaves the library
    if (!S || !out) return ATS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out->completed = S->completed;
    out->queued = (uint64_t)S->queue.size();
    out->ticks = S->ticks;
    out->peak_resident = S->peak_resident;
    out->resident_bytes = S->resident;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_server_destroy(ats_server *S) {
  try {  // no C++ exception leaves the library
    if (!S) return ATS_ERR_INVALID_ARG;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
      S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    if (S->ctx) {
      cudaStreamSynchronize(S->st);
      for (auto &sl : S->slots)
        if (sl.lvl) ats_level_destroy(sl.lvl);
      if (S->exec) cudaGraphExecDestroy(S->exec);
      if (S->h_final) cudaFreeHost(S->h_final);
      if (S->fj.fork) cudaEventDestroy(S->fj.fork);
      if (S->fj.join) cudaEventDestroy(S->fj.join);
      if (S->fj.aux) cudaStreamDestroy(S->fj.aux);
      ats_context_destroy(S->ctx);  // frees every device buffer of the server
    }
    delete S;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

}  // extern "C"
