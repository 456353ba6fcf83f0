// AMR hierarchy and the level substep driver (adaptive time stepping).
//
// Sect. 2.2: a level l advances with its own time step, dt^l = dt^{l+1}_1 +
// dt^{l+1}_2, finer levels first.  Sect. 3.3.1 (fine-to-coarse): a cell of
// level l next to a coarser leaf sees a Dirichlet value, the coarse energy
// held at E^n over both fine substeps, at distance 3 dx / 2 (factor 2/3).
// Sect. 3.3.2 (coarse-to-fine): a cell next to a refined cell sees the
// restriction of the refined cell (mean of its oct of children after the fine
// update), factor 1, Dirichlet.  Each level is solved on its own (Sect. 3.1).
//
// Two orders are provided: ATS_ORDER_FINE_FIRST (the paper's) and
// ATS_ORDER_COARSE_FIRST, where the coarse step is taken first and the fine
// substeps see the coarse value linear in time across the coarse step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "ats_internal.h"

using namespace ats;

namespace {

uint64_t key3(int64_t x, int64_t y, int64_t z) {
  const int64_t off = int64_t(1) << 20;
  return (uint64_t(x + off) << 42) | (uint64_t(y + off) << 21) | uint64_t(z + off);
}

int64_t floor_div2(int64_t v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }

struct LevelIndex {
  std::unordered_map<uint64_t, int32_t> oct;
  const ats_level_desc *d = nullptr;
  explicit LevelIndex(const ats_level_desc *desc) : d(desc) {
    oct.reserve((size_t)desc->n_oct * 2);
    for (int64_t o = 0; o < desc->n_oct; ++o)
      oct.emplace(key3(desc->oct_xyz[3 * o], desc->oct_xyz[3 * o + 1], desc->oct_xyz[3 * o + 2]), (int32_t)o);
  }
  // cell index at this level of level cell coordinates (x, y, z), or -1
  int64_t cell(int64_t x, int64_t y, int64_t z) const {
    auto it = oct.find(key3(floor_div2(x), floor_div2(y), floor_div2(z)));
    if (it == oct.end()) return -1;
    const int c = (int)((x - 2 * floor_div2(x)) + 2 * (y - 2 * floor_div2(y)) + 4 * (z - 2 * floor_div2(z)));
    return 8 * (int64_t)it->second + c;
  }
  bool leaf(int64_t cell) const { return !d->leaf_mask || ((d->leaf_mask[cell >> 3] >> (cell & 7)) & 1); }
};

constexpr int kAx[6] = {0, 0, 1, 1, 2, 2};
constexpr int kSg[6] = {-1, 1, -1, 1, -1, 1};

}  // namespace

namespace ats {

std::string plan_level_faces(const ats_level_desc *levels, int n_levels, int l, LevelFaces &out,
                             const int8_t *wall_kind) {
  if (l < 0 || l >= n_levels) return "level out of range";
  if (wall_kind)
    for (int k = 0; k < 6; ++k)
      if (wall_kind[k] != -1 && wall_kind[k] != ATS_FACE_DIRICHLET) return "wall_kind: -1 or ATS_FACE_DIRICHLET";
  // a face on the domain boundary: a Dirichlet side gets a face with the
  // side's ghost (src_cell = side), a zero-flux side nothing
  auto wall = [&](int64_t cell, int dir) {
    if (!wall_kind || wall_kind[dir] != ATS_FACE_DIRICHLET) return;
    out.cell.push_back((int32_t)cell);
    out.dir.push_back((int8_t)dir);
    out.rel.push_back((int8_t)ATS_REL_SAME);
    out.src_cell.push_back((int32_t)dir);
  };
  std::vector<LevelIndex> idx;
  idx.reserve(n_levels);
  for (int k = 0; k < n_levels; ++k) {
    if (!levels[k].oct_xyz || levels[k].n_oct <= 0) return "level without octs";
    idx.emplace_back(&levels[k]);
  }
  const ats_level_desc &d = levels[l];
  out = LevelFaces();
  for (int64_t o = 0; o < d.n_oct; ++o) {
    for (int c = 0; c < 8; ++c) {
      const int64_t cell = 8 * o + c;
      if (!idx[l].leaf(cell)) continue;
      const int64_t p[3] = {2 * (int64_t)d.oct_xyz[3 * o] + (c & 1), 2 * (int64_t)d.oct_xyz[3 * o + 1] + ((c >> 1) & 1),
                            2 * (int64_t)d.oct_xyz[3 * o + 2] + ((c >> 2) & 1)};
      for (int dir = 0; dir < 6; ++dir) {
        int64_t q[3] = {p[0], p[1], p[2]};
        q[kAx[dir]] += kSg[dir];
        const int64_t j = idx[l].cell(q[0], q[1], q[2]);
        if (j >= 0) {
          if (idx[l].leaf(j)) continue;  // interior face
          out.cell.push_back((int32_t)cell);
          out.dir.push_back((int8_t)dir);
          out.rel.push_back((int8_t)ATS_REL_FINER);
          out.src_cell.push_back((int32_t)j);
          continue;
        }
        if (l == 0) {  // outside the base level: the domain boundary
          wall(cell, dir);
          continue;
        }
        const int64_t m[3] = {floor_div2(q[0]), floor_div2(q[1]), floor_div2(q[2])};
        const int64_t jc = idx[l - 1].cell(m[0], m[1], m[2]);
        if (jc >= 0) {
          if (!idx[l - 1].leaf(jc)) return "level " + std::to_string(l) + ": a refined coarse cell has no oct at this level";
          out.cell.push_back((int32_t)cell);
          out.dir.push_back((int8_t)dir);
          out.rel.push_back((int8_t)ATS_REL_COARSER);
          out.src_cell.push_back((int32_t)jc);
          continue;
        }
        // no coarser cell either: 2:1 balance violated, or the domain wall
        int64_t r[3] = {m[0], m[1], m[2]};
        for (int k = l - 2; k >= 0; --k) {
          for (int a = 0; a < 3; ++a) r[a] = floor_div2(r[a]);
          if (idx[k].cell(r[0], r[1], r[2]) >= 0)
            return "level " + std::to_string(l) + ": 2:1 balance violated (neighbour found at level " +
                   std::to_string(k) + ")";
        }
        wall(cell, dir);
      }
    }
  }
  // refined cells of this level and their child octs
  if (l + 1 < n_levels) {
    const ats_level_desc &f = levels[l + 1];
    for (int64_t o = 0; o < f.n_oct; ++o) {
      const int64_t x = f.oct_xyz[3 * o], y = f.oct_xyz[3 * o + 1], z = f.oct_xyz[3 * o + 2];
      const int64_t R = idx[l].cell(x, y, z);
      if (R < 0) return "level " + std::to_string(l + 1) + ": oct without a parent cell";
      if (idx[l].leaf(R)) return "level " + std::to_string(l) + ": a cell with children is marked as leaf";
      out.restrict_cell.push_back((int32_t)R);
      out.restrict_child.push_back((int32_t)o);
    }
  }
  return std::string();
}

}  // namespace ats

struct HLevel {
  ats_level *lvl = nullptr;
  double dx = 0.0;
  double *rho = nullptr, *T = nullptr, *s = nullptr, *src = nullptr;  // flux-limited diffusion state
  int64_t N = 0, n_face = 0, n_restrict = 0;
  double *E = nullptr, *E_prev = nullptr, *K = nullptr, *fE = nullptr, *fK = nullptr;
  int8_t *src_rel = nullptr;  // 0 same level (FINER), 1 coarser
  int32_t *src_cell = nullptr, *r_cell = nullptr, *r_child = nullptr;
  // stored interface energy (Sect. 3.3.2): per face of this level, and for
  // each coarse-to-fine face the (up to 4) fine-to-coarse faces of the next
  // level that feed it
  int32_t *fcell = nullptr, *gather4 = nullptr;
  double *fstore = nullptr;
  std::vector<int8_t> rel;  // host copy of the face relations
};

struct ats_hierarchy {
  ats_context *ctx = nullptr;
  int order = ATS_ORDER_FINE_FIRST;
  bool fld = false;  // K, s and src from the gas state before every level solve
  double k0 = 0.0;
  int iface_kind = ATS_FACE_DIRICHLET;  // row of the coarse-to-fine faces
  double iface_alpha = 1.0;
  double *d_wall = nullptr;  // [12] ghost E and K of the six domain sides
  bool power_law = false;    // K = pl_K0 E^pl_a on the leaves before every solve
  double pl_K0 = 1.0, pl_a = 0.0;
  std::vector<HLevel> lv;
  // use_graph = 2: the level solves of one ats_level_advance are enqueued
  // without host waits; their result records are read once at the end
  DeferredRec *d_recs = nullptr;
  DeferredRec *h_recs = nullptr;  // pinned
  int rec_cap = 0, n_recs = 0;
  std::vector<std::pair<int, int64_t>> rec_meta;  // interval, tick bound per record
  bool deferred = false;
  // use_graph = 3: the whole step as one graph.  It is captured right after a
  // deferred run of the same step (which leaves every plan, device loop and
  // start state resident) and replayed while the step's arguments, the
  // hierarchy's configuration (gen) and the context's epoch are unchanged
  bool capturing = false;
  uint64_t gen = 0;  // bumped by every change of the hierarchy's configuration
  cudaGraphExec_t step_exec = nullptr;
  int step_level = -1;
  double step_dt = 0.0;
  ats_solve_opts step_opts{};
  uint64_t step_gen = 0, step_epoch = 0;
  int64_t n_captures = 0, n_replays = 0;
  std::vector<std::pair<int, int64_t>> step_meta;  // rec_meta of the captured step
};

namespace {

#define H_TRY(expr)                                                                   \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      set_error(std::string("CUDA error: ") + cudaGetErrorString(_e) + " at " #expr); \
      return ATS_ERR_CUDA;                                                            \
    }                                                                                 \
  } while (0)

void hierarchy_free(ats_hierarchy *H) {
  if (H->step_exec) cudaGraphExecDestroy(H->step_exec);
  ctx_free(H->ctx, H->d_wall);
  ctx_free(H->ctx, H->d_recs);
  if (H->h_recs) cudaFreeHost(H->h_recs);
  for (HLevel &h : H->lv) {
    void *ptrs[] = {h.E,  h.E_prev, h.K,   h.fE, h.fK, h.src_rel, h.src_cell, h.r_cell, h.r_child,
                    h.rho, h.T,     h.s,   h.src, h.fcell, h.gather4, h.fstore};
    for (void *p : ptrs) ctx_free(H->ctx, p);
    if (h.lvl) ats_level_destroy(h.lvl);
  }
  delete H;
}

// restriction of level l+1 into the refined cells of level l
ats_status restrict_into(ats_hierarchy *H, int l) {
  if (l + 1 >= (int)H->lv.size()) return ATS_OK;
  HLevel &c = H->lv[l], &f = H->lv[l + 1];
  H_TRY(launch_restrict((int)c.n_restrict, c.r_cell, c.r_child, f.E, f.K, c.E, c.K, ctx_stream(H->ctx)));
  return ATS_OK;
}

// one implicit solve of level l over dt; coarser values at theta of the
// coarser level's step
ats_status solve_level(ats_hierarchy *H, int l, double dt, double theta, const ats_solve_opts *opts,
                       ats_solve_stats *acc) {
  HLevel &h = H->lv[l];
  cudaStream_t st = ctx_stream(H->ctx);
  ats_status s = restrict_into(H, l);
  if (s != ATS_OK) return s;
  if (H->power_law)  // frozen at E^n of this level, leaf cells (refined cells keep the restriction)
    H_TRY(launch_power_law_K(h.N, level_leaf(h.lvl), h.E, H->pl_K0, H->pl_a, h.K, st));
  if (H->fld) {
    // coefficients frozen at E^n of this level (leaf cells; refined cells keep
    // the restriction of their children's K)
    H_TRY(launch_fld_coef(h.N / 8, level_nbr(h.lvl), level_leaf(h.lvl), h.E, h.rho, h.T, h.dx, dt, H->k0, h.K, h.s,
                          h.src, st));
  }
  const HLevel *coarse = l > 0 ? &H->lv[l - 1] : nullptr;
  // fine first: the coarser level has not moved, its current E is E^n;
  // coarse first: interpolate between its E^n (E_prev) and E^{n+1} (E)
  const double *ec_old = !coarse ? nullptr : (H->order == ATS_ORDER_FINE_FIRST ? coarse->E : coarse->E_prev);
  H_TRY(launch_gather_faces((int)h.n_face, h.src_rel, h.src_cell, h.E, h.K, ec_old, coarse ? coarse->E : nullptr,
                            coarse ? coarse->K : nullptr, H->order == ATS_ORDER_FINE_FIRST ? 0.0 : theta, h.fE,
                            h.fK, H->d_wall, st));
  H_TRY(cudaMemcpyAsync(h.E_prev, h.E, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, st));
  ats_coef_desc c;
  std::memset(&c, 0, sizeof(c));
  c.dt = dt;
  c.mem = ATS_MEM_DEVICE;
  c.K = h.K;
  c.E_old = h.E_prev;
  c.face_K = h.n_face ? h.fK : nullptr;
  c.face_E = h.n_face ? h.fE : nullptr;
  const bool stored = H->iface_kind != ATS_FACE_DIRICHLET;
  if (stored && h.n_face) c.face_F = h.fstore;  // the fine-side energy of the finer level's steps
  if (H->fld) {
    c.s = h.s;
    c.src = h.src;
  }
  if ((s = ats_level_build_operator(h.lvl, &c)) != ATS_OK) return s;
  ats_solve_opts o;
  if (opts) o = *opts;
  else ats_default_opts(&o);
  o.mem = ATS_MEM_DEVICE;
  ats_solve_stats st1;
  std::memset(&st1, 0, sizeof(st1));
  if (H->deferred) {
    if (H->n_recs >= H->rec_cap) {
      set_error("ats_level_advance: more solves than planned");
      return ATS_ERR_INVALID_ARG;
    }
    int ce = 0;
    int64_t mt = 0;
    s = level_solve_deferred(h.lvl, h.E, &o, H->d_recs + H->n_recs, &ce, &mt, H->capturing);
    if (s != ATS_OK) return s;
    H->rec_meta[H->n_recs++] = {ce, mt};
  } else {
    s = ats_solve(h.lvl, nullptr, h.E, &o, &st1);
  }
  // a warning (a negative energy in the result) is reported, not fatal
  const bool ok = s >= 0;
  if (ok && H->fld) H_TRY(launch_fld_temperature(h.N, level_leaf(h.lvl), h.E, h.rho, h.T, dt, H->k0, st));
  if (ok && stored) {
    if (h.n_face) H_TRY(cudaMemsetAsync(h.fstore, 0, sizeof(double) * h.n_face, st));
    if (coarse && coarse->n_face)  // this step's fine-to-coarse energy, for the coarser level's next solve
      H_TRY(launch_flux_store((int)coarse->n_face, coarse->gather4, h.fcell, h.E, h.K, h.fK, h.fE,
                              0.5 * dt / (h.dx * h.dx), H->lv[l - 1].fstore, st));
  }
  if (acc && !H->deferred) {
    acc->iterations += st1.iterations;
    acc->refinements += st1.refinements;
    acc->ticks += st1.ticks;
    acc->r0_norm = std::max(acc->r0_norm, st1.r0_norm);
    acc->res_norm = std::max(acc->res_norm, st1.res_norm);
    acc->x_norm = std::max(acc->x_norm, st1.x_norm);
    acc->err_bound = std::max(acc->err_bound, st1.err_bound);
    if (st1.status < 0 ? acc->status >= 0 : acc->status == ATS_OK) acc->status = st1.status;
  }
  return ok ? ATS_OK : s;
}

// advance level l (and, recursively, the finer ones) by dt; theta0/theta1:
// the coarser level's time fraction at the start / end of this step
ats_status advance(ats_hierarchy *H, int l, double dt, double theta1, const ats_solve_opts *opts,
                   ats_solve_stats *acc) {
  const bool has_fine = l + 1 < (int)H->lv.size();
  ats_status s;
  if (H->order == ATS_ORDER_FINE_FIRST) {
    if (has_fine) {
      if ((s = advance(H, l + 1, 0.5 * dt, 0.0, opts, acc)) != ATS_OK) return s;
      if ((s = advance(H, l + 1, 0.5 * dt, 0.0, opts, acc)) != ATS_OK) return s;
    }
    // coarser value held at E^n (the coarser level has not moved yet)
    return solve_level(H, l, dt, 0.0, opts, acc);
  }
  // coarse first: this level, then two substeps of the finer level with this
  // level's value linear in time across [t^n, t^n + dt]
  if ((s = solve_level(H, l, dt, theta1, opts, acc)) != ATS_OK) return s;
  if (has_fine) {
    if ((s = advance(H, l + 1, 0.5 * dt, 0.5, opts, acc)) != ATS_OK) return s;
    if ((s = advance(H, l + 1, 0.5 * dt, 1.0, opts, acc)) != ATS_OK) return s;
    if ((s = restrict_into(H, l)) != ATS_OK) return s;
  }
  return ATS_OK;
}

// Room for the result records of one step from `level`: at most 2^(levels
// below) + 1 solves.
ats_status ensure_records(ats_hierarchy *H, int level) {
  const int n_lv = (int)H->lv.size();
  const int need = (1 << std::min(30, n_lv - level)) + 1;
  if (need > H->rec_cap) {
    ctx_free(H->ctx, H->d_recs);
    H->d_recs = nullptr;
    if (H->h_recs) cudaFreeHost(H->h_recs);
    H->h_recs = nullptr;
    H->rec_cap = 0;
    void *p = nullptr;
    ats_status s0 = ctx_alloc(H->ctx, sizeof(DeferredRec) * need, &p);
    if (s0 != ATS_OK) return s0;
    H->d_recs = (DeferredRec *)p;
    if (cudaMallocHost(&H->h_recs, sizeof(DeferredRec) * need) != cudaSuccess) {
      cudaGetLastError();
      set_error("ats_level_advance: pinned allocation failed");
      return ATS_ERR_OOM;
    }
    H->rec_cap = need;
  }
  H->rec_meta.assign(H->rec_cap, {0, 0});
  H->n_recs = 0;
  return ATS_OK;
}

// Fold the host copies of n result records (h_recs) into acc; s: the status
// of the step so far, returned with the first failing solve's error.
ats_status fold_records(const ats_hierarchy *H, const std::vector<std::pair<int, int64_t>> &meta, int n,
                        ats_solve_stats &acc, ats_status s) {
  for (int k = 0; k < n; ++k) {
    ats_solve_stats st1;
    const ats_status r = deferred_result(H->h_recs[k], meta[k].first, meta[k].second, &st1);
    acc.iterations += st1.iterations;
    acc.refinements += st1.refinements;
    acc.ticks += st1.ticks;
    acc.r0_norm = std::max(acc.r0_norm, st1.r0_norm);
    acc.res_norm = std::max(acc.res_norm, st1.res_norm);
    acc.x_norm = std::max(acc.x_norm, st1.x_norm);
    acc.err_bound = std::max(acc.err_bound, st1.err_bound);
    if (r < 0 ? acc.status >= 0 : acc.status == ATS_OK) acc.status = r;
    if (r < 0 && s >= 0) s = r;
  }
  return s;
}

// One step from `level`: with deferred solves (use_graph >= 2) every solve is
// enqueued without a host wait and the records are read once at the end.
ats_status run_step(ats_hierarchy *H, int level, double dt, const ats_solve_opts *opts, bool deferred,
                    ats_solve_stats &acc) {
  H->deferred = deferred;
  if (deferred) {
    ats_status s0 = ensure_records(H, level);
    if (s0 != ATS_OK) {
      H->deferred = false;
      return s0;
    }
  }
  ats_status s = advance(H, level, dt, 1.0, opts, &acc);
  if (deferred) {
    H->deferred = false;
    cudaStream_t st = ctx_stream(H->ctx);
    if (H->n_recs > 0)
      H_TRY(cudaMemcpyAsync(H->h_recs, H->d_recs, sizeof(DeferredRec) * H->n_recs, cudaMemcpyDeviceToHost, st));
    H_TRY(cudaStreamSynchronize(st));
    s = fold_records(H, H->rec_meta, H->n_recs, acc, s);
  }
  return s;
}

// Record the step just taken (the same level, dt and options) as one graph:
// every enqueue of a deferred step -- restriction, ghost gather, operator
// builds, the level solves with their device loops, flux stores -- and the
// copy of the result records to the host.  Nothing runs while it is captured.
ats_status capture_step(ats_hierarchy *H, int level, double dt, const ats_solve_opts *opts) {
  cudaStream_t st = ctx_stream(H->ctx);
  if (H->step_exec) {
    cudaGraphExecDestroy(H->step_exec);
    H->step_exec = nullptr;
  }
  const uint64_t epoch0 = ctx_epoch(H->ctx);
  ats_status s = ensure_records(H, level);
  if (s != ATS_OK) return s;
  H_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  H->deferred = true;
  H->capturing = true;
  s = advance(H, level, dt, 1.0, opts, nullptr);
  H->capturing = false;
  H->deferred = false;
  cudaError_t err = cudaSuccess;
  if (s == ATS_OK && H->n_recs > 0)
    err = cudaMemcpyAsync(H->h_recs, H->d_recs, sizeof(DeferredRec) * H->n_recs, cudaMemcpyDeviceToHost, st);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (err == cudaSuccess) err = e2;
  if (s == ATS_OK && err == cudaSuccess) err = cudaGraphInstantiate(&H->step_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (s == ATS_OK && err != cudaSuccess) {
    cudaGetLastError();
    H->step_exec = nullptr;
    set_error(std::string("ats_level_advance: step graph: ") + cudaGetErrorString(err));
    s = ATS_ERR_CUDA;
  }
  if (s != ATS_OK) {
    if (H->step_exec) cudaGraphExecDestroy(H->step_exec);
    H->step_exec = nullptr;
    return s;
  }
  if (ctx_epoch(H->ctx) != epoch0) {  // the capture needed an allocation or upload
    cudaGraphExecDestroy(H->step_exec);
    H->step_exec = nullptr;
    set_error("ats_level_advance: step graph: the step changed device state while it was captured");
    return ATS_ERR_CUDA;
  }
  H->step_level = level;
  H->step_dt = dt;
  H->step_opts = *opts;
  H->step_gen = H->gen;
  H->step_epoch = epoch0;
  H->step_meta.assign(H->rec_meta.begin(), H->rec_meta.begin() + H->n_recs);
  ++H->n_captures;
  return ATS_OK;
}

}  // namespace

extern "C" {

ats_status ats_hierarchy_plan_faces(const ats_hierarchy_desc *desc, int level, int64_t *n_face, int32_t *face_cell,
                                    int8_t *face_dir, int8_t *face_rel, int32_t *src_cell) {
  try {  // no C++ exception leaves the library
    if (!desc || !n_face || desc->n_levels <= 0 || !desc->levels) {
      set_error("null argument");
      return ATS_ERR_INVALID_ARG;
    }
    LevelFaces lf;
    std::string msg = plan_level_faces(desc->levels, desc->n_levels, level, lf, desc->wall_kind);
    if (!msg.empty()) {
      set_error(msg);
      return ATS_ERR_INVALID_ARG;
    }
    *n_face = (int64_t)lf.cell.size();
    if (face_cell) std::copy(lf.cell.begin(), lf.cell.end(), face_cell);
    if (face_dir) std::copy(lf.dir.begin(), lf.dir.end(), face_dir);
    if (face_rel) std::copy(lf.rel.begin(), lf.rel.end(), face_rel);
    if (src_cell) std::copy(lf.src_cell.begin(), lf.src_cell.end(), src_cell);
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_create(ats_context *ctx, const ats_hierarchy_desc *desc, ats_hierarchy **out) {
  try {  // no C++ exception leaves the library
    if (!ctx || !desc || !out || desc->n_levels <= 0 || !desc->levels) {
      set_error("null argument");
      return ATS_ERR_INVALID_ARG;
    }
    if (desc->order != ATS_ORDER_FINE_FIRST && desc->order != ATS_ORDER_COARSE_FIRST) {
      set_error("bad order");
      return ATS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    for (int l = 1; l < desc->n_levels; ++l) {
      if (std::fabs(desc->levels[l].dx * 2.0 - desc->levels[l - 1].dx) > 1e-12 * desc->levels[l - 1].dx) {
        set_error("each level must halve dx");
        return ATS_ERR_INVALID_ARG;
      }
    }
    ats_hierarchy *H = new (std::nothrow) ats_hierarchy();
    if (!H) return ATS_ERR_OOM;
    H->ctx = ctx;
    H->order = desc->order;
    H->lv.resize(desc->n_levels);
    cudaStream_t st = ctx_stream(ctx);
    {
      // ghost values of the domain sides (used by Dirichlet sides only)
      double wall[12] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1};
      if (desc->wall_kind) {
        for (int k = 0; k < 6; ++k) {
          if (desc->wall_kind[k] != ATS_FACE_DIRICHLET) continue;
          if (!desc->wall_E || !desc->wall_K || !std::isfinite(desc->wall_E[k]) || !(desc->wall_K[k] > 0.0) ||
              !std::isfinite(desc->wall_K[k])) {
            set_error("a Dirichlet side needs a finite wall_E and a wall_K > 0");
            hierarchy_free(H);
            return ATS_ERR_INVALID_ARG;
          }
          wall[k] = desc->wall_E[k];
          wall[6 + k] = desc->wall_K[k];
        }
      }
      void *p = nullptr;
      ats_status s0 = ctx_alloc(ctx, sizeof(wall), &p);
      if (s0 != ATS_OK) {
        hierarchy_free(H);
        return s0;
      }
      H->d_wall = (double *)p;
      cudaError_t e0 = cudaMemcpyAsync(H->d_wall, wall, sizeof(wall), cudaMemcpyHostToDevice, st);
      if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(st);
      if (e0 != cudaSuccess) {
        set_error(cudaGetErrorString(e0));
        hierarchy_free(H);
        return ATS_ERR_CUDA;
      }
    }
    std::vector<LevelFaces> lfs(desc->n_levels);
    for (int l = 0; l < desc->n_levels; ++l) {
      std::string msg = plan_level_faces(desc->levels, desc->n_levels, l, lfs[l], desc->wall_kind);
      if (!msg.empty()) {
        set_error(msg);
        hierarchy_free(H);
        return ATS_ERR_INVALID_ARG;
      }
    }
    for (int l = 0; l < desc->n_levels; ++l) {
      const LevelFaces &lf = lfs[l];
      HLevel &h = H->lv[l];
      ats_level_desc d = desc->levels[l];
      const int64_t nf = (int64_t)lf.cell.size();
      std::vector<int8_t> kind(nf, ATS_FACE_DIRICHLET);
      std::vector<double> alpha(nf, 1.0);
      d.n_face = nf;
      d.face_cell = lf.cell.data();
      d.face_dir = lf.dir.data();
      d.face_kind = kind.data();
      d.face_rel = lf.rel.data();
      d.face_alpha = alpha.data();
      ats_status s = ats_level_create(ctx, &d, &h.lvl);
      if (s != ATS_OK) {
        hierarchy_free(H);
        return s;
      }
      h.N = 8 * d.n_oct;
      h.dx = d.dx;
      h.n_face = nf;
      h.n_restrict = (int64_t)lf.restrict_cell.size();
      void *p;
      auto alloc = [&](size_t bytes, void **dst) {
        ats_status r = ctx_alloc(ctx, bytes ? bytes : 16, &p);
        *dst = p;
        return r;
      };
      if ((s = alloc(sizeof(double) * h.N, (void **)&h.E)) != ATS_OK ||
          (s = alloc(sizeof(double) * h.N, (void **)&h.E_prev)) != ATS_OK ||
          (s = alloc(sizeof(double) * h.N, (void **)&h.K)) != ATS_OK ||
          (s = alloc(sizeof(double) * nf, (void **)&h.fE)) != ATS_OK ||
          (s = alloc(sizeof(double) * nf, (void **)&h.fK)) != ATS_OK ||
          (s = alloc(sizeof(int8_t) * nf, (void **)&h.src_rel)) != ATS_OK ||
          (s = alloc(sizeof(int32_t) * nf, (void **)&h.src_cell)) != ATS_OK ||
          (s = alloc(sizeof(int32_t) * h.n_restrict, (void **)&h.r_cell)) != ATS_OK ||
          (s = alloc(sizeof(int32_t) * h.n_restrict, (void **)&h.r_child)) != ATS_OK ||
          (s = alloc(sizeof(int32_t) * nf, (void **)&h.fcell)) != ATS_OK ||
          (s = alloc(sizeof(int32_t) * 4 * nf, (void **)&h.gather4)) != ATS_OK ||
          (s = alloc(sizeof(double) * nf, (void **)&h.fstore)) != ATS_OK) {
        hierarchy_free(H);
        return s;
      }
      h.rel = lf.rel;
      // coarse-to-fine face (cell, dir) of this level <- the fine-to-coarse faces
      // of the next level whose coarse cell and opposite direction match
      std::vector<int32_t> g4(4 * nf, -1);
      if (l + 1 < desc->n_levels) {
        std::unordered_map<int64_t, int64_t> at;
        for (int64_t f = 0; f < nf; ++f)
          if (lf.rel[f] == ATS_REL_FINER) at[6 * (int64_t)lf.cell[f] + lf.dir[f]] = f;
        const LevelFaces &ff = lfs[l + 1];
        for (size_t g = 0; g < ff.cell.size(); ++g) {
          if (ff.rel[g] != ATS_REL_COARSER) continue;
          auto it = at.find(6 * (int64_t)ff.src_cell[g] + (ff.dir[g] ^ 1));
          if (it == at.end()) continue;
          int32_t *slot = &g4[4 * it->second];
          for (int k = 0; k < 4; ++k)
            if (slot[k] < 0) {
              slot[k] = (int32_t)g;
              break;
            }
        }
      }
      std::vector<int8_t> srel(nf);
      for (int64_t f = 0; f < nf; ++f)
        srel[f] = lf.rel[f] == ATS_REL_COARSER ? 1 : (lf.rel[f] == ATS_REL_SAME ? 2 : 0);
      cudaError_t e = cudaSuccess;
      if (nf) {
        e = cudaMemcpyAsync(h.src_rel, srel.data(), nf, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.src_cell, lf.src_cell.data(), 4 * nf, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.fcell, lf.cell.data(), 4 * nf, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.gather4, g4.data(), 16 * nf, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(h.fstore, 0, sizeof(double) * nf, st);
      }
      if (e == cudaSuccess && h.n_restrict) {
        e = cudaMemcpyAsync(h.r_cell, lf.restrict_cell.data(), 4 * h.n_restrict, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(h.r_child, lf.restrict_child.data(), 4 * h.n_restrict, cudaMemcpyHostToDevice, st);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        set_error(cudaGetErrorString(e));
        hierarchy_free(H);
        return ATS_ERR_CUDA;
      }
    }
    *out = H;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_set_power_law(ats_hierarchy *H, double K0, double a) {
  try {  // no C++ exception leaves the library
    if (!H || !(K0 > 0.0) || !std::isfinite(K0) || !std::isfinite(a)) {
      set_error("ats_hierarchy_set_power_law: K0 > 0 and a finite a are required");
      return ATS_ERR_INVALID_ARG;
    }
    if (H->fld) {
      set_error("ats_hierarchy_set_power_law: the hierarchy is in the radiation-matter mode");
      return ATS_ERR_INVALID_ARG;
    }
    H->power_law = true;
    ++H->gen;
    H->pl_K0 = K0;
    H->pl_a = a;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_set_interface(ats_hierarchy *H, int kind, double alpha) {
  try {  // no C++ exception leaves the library
    if (!H) return ATS_ERR_INVALID_ARG;
    if (kind != ATS_FACE_DIRICHLET && kind != ATS_FACE_NEUMANN && kind != ATS_FACE_ROBIN) {
      set_error("bad interface kind");
      return ATS_ERR_INVALID_ARG;
    }
    if (kind == ATS_FACE_ROBIN && !(alpha >= 0.0 && alpha <= 1.0)) {
      set_error("Robin alpha must be in [0, 1]");
      return ATS_ERR_INVALID_ARG;
    }
    if (kind != ATS_FACE_DIRICHLET && H->order != ATS_ORDER_FINE_FIRST) {
      set_error("stored interface fluxes need the fine-first order");
      return ATS_ERR_INVALID_ARG;
    }
    const double a = kind == ATS_FACE_DIRICHLET ? 1.0 : (kind == ATS_FACE_NEUMANN ? 0.0 : alpha);
    cudaStream_t st = ctx_stream(H->ctx);
    for (HLevel &h : H->lv) {
      std::vector<int8_t> k(h.n_face, ATS_FACE_DIRICHLET);
      std::vector<double> al(h.n_face, 1.0);
      for (int64_t f = 0; f < h.n_face; ++f)
        if (h.rel[f] == ATS_REL_FINER) {
          k[f] = (int8_t)kind;
          al[f] = a;
        }
      ats_status s = level_set_face_rows(h.lvl, k.data(), al.data());
      if (s != ATS_OK) return s;
      if (h.n_face) H_TRY(cudaMemsetAsync(h.fstore, 0, sizeof(double) * h.n_face, st));
    }
    H_TRY(cudaStreamSynchronize(st));
    H->iface_kind = kind;
    ++H->gen;
    H->iface_alpha = a;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_destroy(ats_hierarchy *H) {
  try {  // no C++ exception leaves the library
    if (!H) return ATS_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx_stream(H->ctx));
    hierarchy_free(H);
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_level(ats_hierarchy *H, int level, ats_level **out) {
  try {  // no C++ exception leaves the library
    if (!H || !out || level < 0 || level >= (int)H->lv.size()) return ATS_ERR_INVALID_ARG;
    *out = H->lv[level].lvl;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_set_state(ats_hierarchy *H, int level, const double *E, const double *K, int mem) {
  try {  // no C++ exception leaves the library
    if (!H || level < 0 || level >= (int)H->lv.size() || !E || !K) return ATS_ERR_INVALID_ARG;
    HLevel &h = H->lv[level];
    cudaStream_t st = ctx_stream(H->ctx);
    const cudaMemcpyKind k = mem == ATS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    H_TRY(cudaMemcpyAsync(h.E, E, sizeof(double) * h.N, k, st));
    H_TRY(cudaMemcpyAsync(h.E_prev, E, sizeof(double) * h.N, k, st));
    H_TRY(cudaMemcpyAsync(h.K, K, sizeof(double) * h.N, k, st));
    H_TRY(cudaStreamSynchronize(st));
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_set_fld(ats_hierarchy *H, int level, const double *rho, const double *T, double k0, int mem) {
  try {  // no C++ exception leaves the library
    if (!H || level < 0 || level >= (int)H->lv.size() || !rho || !T || !(k0 > 0.0)) {
      set_error("ats_hierarchy_set_fld: bad argument");
      return ATS_ERR_INVALID_ARG;
    }
    if (H->power_law) {
      set_error("ats_hierarchy_set_fld: the hierarchy is in the power-law coefficient mode");
      return ATS_ERR_INVALID_ARG;
    }
    HLevel &h = H->lv[level];
    cudaStream_t st = ctx_stream(H->ctx);
    ats_status s;
    void *p;
    if (!h.rho) {
      const size_t b = sizeof(double) * h.N;
      if ((s = ctx_alloc(H->ctx, b, &p)) != ATS_OK) return s;
      h.rho = (double *)p;
      if ((s = ctx_alloc(H->ctx, b, &p)) != ATS_OK) return s;
      h.T = (double *)p;
      if ((s = ctx_alloc(H->ctx, b, &p)) != ATS_OK) return s;
      h.s = (double *)p;
      if ((s = ctx_alloc(H->ctx, b, &p)) != ATS_OK) return s;
      h.src = (double *)p;
    }
    const cudaMemcpyKind k = mem == ATS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    H_TRY(cudaMemcpyAsync(h.rho, rho, sizeof(double) * h.N, k, st));
    H_TRY(cudaMemcpyAsync(h.T, T, sizeof(double) * h.N, k, st));
    H->k0 = k0;
    // initial K from the current E (dt does not enter K)
    H_TRY(launch_fld_coef(h.N / 8, level_nbr(h.lvl), level_leaf(h.lvl), h.E, h.rho, h.T, h.dx, 1.0, k0, h.K, h.s,
                          h.src, st));
    H_TRY(cudaStreamSynchronize(st));
    bool all = true;
    for (const HLevel &x : H->lv) all = all && x.rho != nullptr;
    H->fld = all;
    ++H->gen;
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_get_temperature(ats_hierarchy *H, int level, double *T, int mem) {
  try {  // no C++ exception leaves the library
    if (!H || level < 0 || level >= (int)H->lv.size() || !T || !H->lv[level].T) return ATS_ERR_INVALID_ARG;
    HLevel &h = H->lv[level];
    cudaStream_t st = ctx_stream(H->ctx);
    H_TRY(cudaMemcpyAsync(T, h.T, sizeof(double) * h.N,
                          mem == ATS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    H_TRY(cudaStreamSynchronize(st));
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_get_state(ats_hierarchy *H, int level, double *E, int mem) {
  try {  // no C++ exception leaves the library
    if (!H || level < 0 || level >= (int)H->lv.size() || !E) return ATS_ERR_INVALID_ARG;
    // refined cells report the restriction of their children
    for (int l = (int)H->lv.size() - 2; l >= level; --l) {
      ats_status s = restrict_into(H, l);
      if (s != ATS_OK) return s;
    }
    HLevel &h = H->lv[level];
    cudaStream_t st = ctx_stream(H->ctx);
    H_TRY(cudaMemcpyAsync(E, h.E, sizeof(double) * h.N,
                          mem == ATS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    H_TRY(cudaStreamSynchronize(st));
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_level_advance(ats_hierarchy *H, int level, double dt, const ats_solve_opts *opts,
                             ats_solve_stats *stats) {
  try {  // no C++ exception leaves the library
    if (!H || level < 0 || level >= (int)H->lv.size() || !(dt > 0.0)) {
      set_error("ats_level_advance: bad argument");
      return ATS_ERR_INVALID_ARG;
    }
    ats_solve_stats acc;
    std::memset(&acc, 0, sizeof(acc));
    acc.status = ATS_OK;
    cudaSetDevice(ctx_device(H->ctx));
    const int ug = opts ? opts->use_graph : 0;
    ats_status s;
    if (ug == 3) {
      // use_graph = 3: replay the step's graph while it is current; else take
      // the step with deferred solves, then capture it for the next call
      const bool current = H->step_exec && H->step_level == level && H->step_dt == dt &&
                           std::memcmp(&H->step_opts, opts, sizeof(*opts)) == 0 && H->step_gen == H->gen &&
                           H->step_epoch == ctx_epoch(H->ctx);
      if (current) {
        cudaStream_t st = ctx_stream(H->ctx);
        H_TRY(cudaGraphLaunch(H->step_exec, st));
        H_TRY(cudaStreamSynchronize(st));
        ++H->n_replays;
        s = fold_records(H, H->step_meta, (int)H->step_meta.size(), acc, ATS_OK);
      } else {
        s = run_step(H, level, dt, opts, true, acc);
        if (s >= 0) {
          const ats_status sc = capture_step(H, level, dt, opts);
          if (sc != ATS_OK) s = sc;
        }
      }
    } else {
      s = run_step(H, level, dt, opts, ug == 2, acc);
    }
    // errors first; else the first warning of the step's solves
    if (s == ATS_OK && acc.status > 0) s = acc.status;
    if (stats) *stats = acc;
    return s;
  } catch (...) {
    return ats::abi_exception();
  }
}

ats_status ats_hierarchy_graph_stats(ats_hierarchy *H, int *held, int64_t *captures, int64_t *replays) {
  if (!H) {
    set_error("ats_hierarchy_graph_stats: null hierarchy");
    return ATS_ERR_INVALID_ARG;
  }
  if (held) *held = H->step_exec ? 1 : 0;
  if (captures) *captures = H->n_captures;
  if (replays) *replays = H->n_replays;
  return ATS_OK;
}

}  // extern "C"
