// sm_103a kernels of the per-level implicit diffusion solve.
//
//  k_coef_build  cell diffusion coefficients, interface diagonal extras and the
//                right-hand side b (Sect. 3.1, Eq. Er_imp1; Sect. 3.2 rows).
//  k_op / k_upd  one device "tick" of every solve in a work list: either one
//                iteration of the diagonal-preconditioned CG of Sect. 3.3.4
//                (k_op: p = z + beta p, q = (I + dt A) p, p.q; k_upd:
//                e += alpha p, r = D z - alpha q, z = D^-1 r, r.z, r.r) or one
//                FP64 true-residual pass r = b - (I + dt A)(x + e) of the
//                iterative refinement (k_op) followed by x += e (k_upd).
//
// Layout: a level is an array of octs; cell c = ix + 2 iy + 4 iz of oct o is
// element 8 o + c.  A CTA of 256 threads covers 32 octs per pass, one cell
// per thread, so the eight cells of an oct are eight consecutive lanes and
// the three in-oct neighbours of a cell are lanes c^1, c^2, c^4 (warp
// shuffles).  The three out-of-oct neighbours come from the six-entry oct
// neighbour table.  K < 0 marks a cell that is not an unknown of the level
// (refined cell); its vectors are kept at zero so it drops out of the stencil.
//
// The operator is matrix-free: an interior face contributes
// C = dt/dx^2 (K_i + K_j)/2 = h (K_i + K_j); the diagonal is
// d_i = 1 + xd_i + sum_f C_f with xd_i (coupling shift + interface w C) read
// from a sparse per-oct record.
//
// Reductions: each work item (a run of octs of one solve) writes FP64
// partial sums; the last CTA to finish a solve's items (atomic counter)
// reduces them in a fixed order and advances that solve's scalars.  No CTA
// ever waits for another.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ats_internal.h"

namespace ats {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// FP64-quality dot-product accumulation.  FP32 bulk: each product is split
// exactly (TwoProduct via FMA) and summed with TwoSum (Ogita, Rump & Oishi
// 2005, "Accurate sum and dot product", Dot2), then the (hi, lo) pair is
// carried to FP64 for the block and solve reductions.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
  __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x, float y) {
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);
    const float t = __fadd_rn(s, p);
    const float zz = __fsub_rn(t, s);
    const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, zz)), __fsub_rn(p, zz));
    s = t;
    c = __fadd_rn(c, __fadd_rn(se, pe));
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// Block reduction of kNumPartials doubles (slot 2 optionally a max), fixed
// order.  Result valid in thread 0.
template <bool kSlot2Max>
__device__ __forceinline__ void block_reduce(double (&v)[kNumPartials],
                                             double (*red)[kNumPartials]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNumPartials; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(kFull, v[k], off);
      v[k] = (kSlot2Max && k == 2) ? fmax(v[k], o) : v[k] + o;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNumPartials; ++k) red[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kNumPartials; ++k) {
      double a = red[0][k];
      for (int w = 1; w < kThreads / 32; ++w) a = (kSlot2Max && k == 2) ? fmax(a, red[w][k]) : a + red[w][k];
      v[k] = a;
    }
  }
  __syncthreads();
}

// Reduce the partials of all items of solve s (called by the last CTA).
template <bool kSlot2Max>
__device__ __forceinline__ void solve_reduce(const double *partials, int item_begin, int n_items,
                                             double (&out)[kNumPartials],
                                             double (*red)[kNumPartials]) {
  double v[kNumPartials] = {0.0, 0.0, 0.0, 0.0};
  for (int it = item_begin + (int)threadIdx.x; it < item_begin + n_items; it += kThreads) {
#pragma unroll
    for (int k = 0; k < kNumPartials; ++k) {
      const double p = __ldcg(partials + (size_t)it * kNumPartials + k);
      v[k] = (kSlot2Max && k == 2) ? fmax(v[k], p) : v[k] + p;
    }
  }
  block_reduce<kSlot2Max>(v, red);
#pragma unroll
  for (int k = 0; k < kNumPartials; ++k) out[k] = v[k];
}

// Publish an item's partials; returns true in every thread of the CTA that
// finished the last item of its solve.
__device__ __forceinline__ bool publish_item(double (&v)[kNumPartials], double *partials, int it,
                                             SolveScalars *scs, int n_items_solve, int *s_last) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kNumPartials; ++k) partials[(size_t)it * kNumPartials + k] = v[k];
    __threadfence();
    const int prev = atomicAdd(&scs->counter, 1);
    *s_last = (prev == n_items_solve - 1);
    if (*s_last) __threadfence();
  }
  __syncthreads();
  return *s_last != 0;
}

// ---------------------------------------------------------------------------
// one pass (32 octs) of each phase; the caller loops over an item's passes
// ---------------------------------------------------------------------------

struct CellCtx {
  int o;       // oct index (may be >= oct_end on a ragged tail)
  int c;       // cell in oct
  bool valid;  // o < oct_end
  int64_t i;   // 8 o + c
};

__device__ __forceinline__ CellCtx cell_ctx(int ob, int oct_end) {
  CellCtx x;
  x.o = ob + ((int)threadIdx.x >> 3);
  x.c = (int)threadIdx.x & 7;
  x.valid = x.o < oct_end;
  x.i = (int64_t)x.o * 8 + x.c;
  return x;
}

// The out-of-oct neighbour oct along each axis (the side this cell touches).
__device__ __forceinline__ void load_nbr(const int32_t *__restrict__ nbr, const CellCtx &x,
                                         int (&nb)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    nb[a] = x.valid ? __ldg(nbr + (int64_t)x.o * 6 + 2 * a + ((x.c >> a) & 1)) : -1;
}

// k_op, CG phase: p_new = z + beta p_old (first: p_new = z), q = (I + dt A) p_new,
// partial p_new . q.
template <typename T>
__device__ __forceinline__ void op_inner_pass(const SolveDev &sd, int ob, int oct_end, T h, T beta,
                                              bool first, const T *__restrict__ pold,
                                              T *__restrict__ pnew, Acc<T> &pq) {
  const T *__restrict__ KT = (const T *)sd.KT;
  const T *__restrict__ z = (const T *)sd.z;
  const CellCtx x = cell_ctx(ob, oct_end);
  int nb[3];
  load_nbr(sd.nbr, x, nb);
  T kv = T(-1), pv = T(0);
  int rec = -1;
  if (x.valid) {
    kv = KT[x.i];
    const T zv = z[x.i];
    pv = first ? zv : zv + beta * pold[x.i];
    rec = __ldg(sd.xrec + x.o);
  }
  // out-of-oct neighbours: issue all loads first
  T kj[3], pj[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    kj[a] = T(-1);
    pj[a] = T(0);
    if (nb[a] >= 0) {
      const int64_t j = (int64_t)nb[a] * 8 + (x.c ^ (1 << a));
      kj[a] = KT[j];
      const T zj = z[j];
      pj[a] = first ? zj : zj + beta * pold[j];
    }
  }
  T dsum = T(0), off = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T pn = __shfl_xor_sync(kFull, pv, 1 << a);
    const T kn = __shfl_xor_sync(kFull, kv, 1 << a);
    if (kn >= T(0)) {
      const T C = h * (kv + kn);
      dsum += C;
      off += C * pn;
    }
    if (kj[a] >= T(0)) {
      const T C = h * (kv + kj[a]);
      dsum += C;
      off += C * pj[a];
    }
  }
  if (x.valid) {
    if (kv >= T(0)) {
      const T xd = rec >= 0 ? ((const T *)sd.xdT)[(int64_t)rec * 8 + x.c] : T(0);
      const T d = T(1) + xd + dsum;
      const T q = d * pv - off;
      pnew[x.i] = pv;
      pq.add(pv, q);
    } else {
      pnew[x.i] = T(0);
    }
  }
}

// k_upd, CG phase: q = (I + dt A) p, r = D z - alpha q, z = r / D, e += alpha p,
// partials r.z, r.r (and the max relative change for the paper rule).
template <typename T, bool kPaper>
__device__ __forceinline__ void upd_inner_pass(const SolveDev &sd, int ob, int oct_end, T h, T alpha,
                                               const T *__restrict__ p, Acc<T> &rz, Acc<T> &rr,
                                               double &maxchg) {
  const T *__restrict__ KT = (const T *)sd.KT;
  T *__restrict__ z = (T *)sd.z;
  T *__restrict__ e = (T *)sd.e;
  const CellCtx x = cell_ctx(ob, oct_end);
  int nb[3];
  load_nbr(sd.nbr, x, nb);
  T kv = T(-1), pv = T(0);
  int rec = -1;
  if (x.valid) {
    kv = KT[x.i];
    pv = p[x.i];
    rec = __ldg(sd.xrec + x.o);
  }
  T kj[3], pj[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    kj[a] = T(-1);
    pj[a] = T(0);
    if (nb[a] >= 0) {
      const int64_t j = (int64_t)nb[a] * 8 + (x.c ^ (1 << a));
      kj[a] = KT[j];
      pj[a] = p[j];
    }
  }
  T dsum = T(0), off = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T pn = __shfl_xor_sync(kFull, pv, 1 << a);
    const T kn = __shfl_xor_sync(kFull, kv, 1 << a);
    if (kn >= T(0)) {
      const T C = h * (kv + kn);
      dsum += C;
      off += C * pn;
    }
    if (kj[a] >= T(0)) {
      const T C = h * (kv + kj[a]);
      dsum += C;
      off += C * pj[a];
    }
  }
  if (x.valid && kv >= T(0)) {
    const T xd = rec >= 0 ? ((const T *)sd.xdT)[(int64_t)rec * 8 + x.c] : T(0);
    const T d = T(1) + xd + dsum;
    const T q = d * pv - off;
    const T zv = z[x.i];
    const T r = d * zv - alpha * q;
    const T zn = r / d;
    const T ev = e[x.i];
    const T step = alpha * pv;
    e[x.i] = ev + step;
    z[x.i] = zn;
    rz.add(r, zn);
    rr.add(r, r);
    if (kPaper) {
      const double xv = sd.x64[x.i] + (double)ev;
      const double chg = fabs((double)step) / fabs(xv);
      maxchg = fmax(maxchg, chg);
    }
  }
}

// k_op, refinement phase: x' = x + e, r = b - (I + dt A) x' in FP64 with the
// FP64 K, xd and b; z = r / D_T in the bulk precision; partials r.r, x'.x', r.z.
template <typename T>
__device__ __forceinline__ void op_refine_pass(const SolveDev &sd, int ob, int oct_end, double h,
                                               double &rr, double &xx, double &rz) {
  const T *__restrict__ e = (const T *)sd.e;
  const T *__restrict__ KT = (const T *)sd.KT;
  T *__restrict__ z = (T *)sd.z;
  const CellCtx x = cell_ctx(ob, oct_end);
  int nb[3];
  load_nbr(sd.nbr, x, nb);
  double kv = -1.0, xv = 0.0;
  T kvT = T(-1);
  int rec = -1;
  if (x.valid) {
    kv = sd.K64[x.i];
    kvT = KT[x.i];
    xv = sd.x64[x.i] + (double)e[x.i];
    rec = __ldg(sd.xrec + x.o);
  }
  double kj[3], xj[3];
  T kjT[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    kj[a] = -1.0;
    xj[a] = 0.0;
    kjT[a] = T(-1);
    if (nb[a] >= 0) {
      const int64_t j = (int64_t)nb[a] * 8 + (x.c ^ (1 << a));
      kj[a] = sd.K64[j];
      kjT[a] = KT[j];
      xj[a] = sd.x64[j] + (double)e[j];
    }
  }
  double dsum = 0.0, off = 0.0;
  T dsumT = T(0);
  const T hT = (T)h;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double xn = __shfl_xor_sync(kFull, xv, 1 << a);
    const double kn = __shfl_xor_sync(kFull, kv, 1 << a);
    const T knT = __shfl_xor_sync(kFull, kvT, 1 << a);
    if (kn >= 0.0) {
      const double C = h * (kv + kn);
      dsum += C;
      off += C * xn;
      dsumT += hT * (kvT + knT);
    }
    if (kj[a] >= 0.0) {
      const double C = h * (kv + kj[a]);
      dsum += C;
      off += C * xj[a];
      dsumT += hT * (kvT + kjT[a]);
    }
  }
  if (x.valid) {
    if (kv >= 0.0) {
      const double xd = rec >= 0 ? sd.xd64[(int64_t)rec * 8 + x.c] : 0.0;
      const double d = 1.0 + xd + dsum;
      const double q = d * xv - off;
      const double r = sd.b64[x.i] - q;
      T zT;
      if (sizeof(T) == sizeof(double)) {
        zT = (T)(r / d);
      } else {
        const T xdT = rec >= 0 ? ((const T *)sd.xdT)[(int64_t)rec * 8 + x.c] : T(0);
        const T dT = T(1) + xdT + dsumT;
        zT = (T)r / dT;
      }
      z[x.i] = zT;
      rr = fma(r, r, rr);
      xx = fma(xv, xv, xx);
      rz = fma(r, (double)zT, rz);
    } else {
      z[x.i] = T(0);
    }
  }
}

// k_upd, refinement phase: x += e, e = 0.
template <typename T>
__device__ __forceinline__ void upd_refine_pass(const SolveDev &sd, int ob, int oct_end) {
  const CellCtx x = cell_ctx(ob, oct_end);
  if (!x.valid) return;
  T *__restrict__ e = (T *)sd.e;
  const T ev = e[x.i];
  sd.x64[x.i] += (double)ev;
  e[x.i] = T(0);
}

}  // namespace

// ---------------------------------------------------------------------------
// the two tick kernels (persistent grid, grid-stride over work items)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kThreads) k_op(const SolveDev *__restrict__ solves,
                                                 SolveScalars *__restrict__ sc,
                                                 const WorkItem *__restrict__ items, int n_items,
                                                 double *__restrict__ partials,
                                                 unsigned long long *__restrict__ cells) {
  __shared__ double red[kThreads / 32][kNumPartials];
  __shared__ int s_last;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const WorkItem item = items[it];
    const int s = item.solve;
    SolveScalars *scs = sc + s;
    const int phase = scs->phase;
    if (phase == kDone) continue;
    const SolveDev &sd = solves[s];
    const int oct_end = item.oct_begin + item.n_oct;
    double v[kNumPartials] = {0.0, 0.0, 0.0, 0.0};
    if (phase == kInner) {
      const T h = (T)sd.h;
      const T beta = (T)scs->beta;
      const bool first = scs->first != 0;
      const int pcur = scs->pcur;
      const T *pold = (const T *)(pcur ? sd.p1 : sd.p0);
      T *pnew = (T *)(pcur ? sd.p0 : sd.p1);
      Acc<T> pq;
      for (int ob = item.oct_begin; ob < oct_end; ob += kOctsPerPass)
        op_inner_pass<T>(sd, ob, oct_end, h, beta, first, pold, pnew, pq);
      v[0] = pq.get();
      if (cells && threadIdx.x == 0) atomicAdd(cells + 0, (unsigned long long)item.n_oct * 8);
    } else {
      double rr = 0.0, xx = 0.0, rz = 0.0;
      for (int ob = item.oct_begin; ob < oct_end; ob += kOctsPerPass)
        op_refine_pass<T>(sd, ob, oct_end, sd.h, rr, xx, rz);
      v[0] = rr;
      v[1] = xx;
      v[2] = rz;
      if (cells && threadIdx.x == 0) atomicAdd(cells + 1, (unsigned long long)item.n_oct * 8);
    }
    block_reduce<false>(v, red);
    if (!publish_item(v, partials, it, scs, sd.n_items, &s_last)) continue;

    // ---- last CTA of solve s: advance the op-side scalars ----
    double tot[kNumPartials];
    solve_reduce<false>(partials, sd.item_begin, sd.n_items, tot, red);
    if (threadIdx.x == 0) {
      scs->counter = 0;
      if (phase == kInner) {
        const double pq = tot[0];
        if (!(pq > 0.0) || !isfinite(pq)) {
          scs->alpha = 0.0;
          scs->status = ATS_ERR_BREAKDOWN;
        } else {
          scs->alpha = scs->rz / pq;
        }
      } else {
        const double rnorm = sqrt(tot[0]);
        const double xnorm = sqrt(tot[1]);
        if (scs->refines == 0) scs->r0 = rnorm;
        scs->refines += 1;
        scs->rnorm = rnorm;
        scs->xnorm = xnorm;
        const double ref = (sd.stop_rule == ATS_STOP_CERTIFIED) ? xnorm : scs->r0;
        const double target = sd.tol * ref;
        if (scs->final_pass) {
          scs->phase_next = kDone;
        } else if (!isfinite(rnorm)) {
          scs->status = ATS_ERR_BREAKDOWN;
          scs->phase_next = kDone;
        } else if (rnorm <= target) {
          scs->phase_next = kDone;
        } else if (scs->refines > sd.max_refine) {
          scs->status = ATS_ERR_NOT_CONVERGED;
          scs->phase_next = kDone;
        } else if (!(tot[2] > 0.0)) {
          scs->status = ATS_ERR_BREAKDOWN;
          scs->phase_next = kDone;
        } else {
          scs->phase_next = kInner;
          scs->rz = tot[2];
          scs->first = 1;
          scs->inner_iters = 0;
          scs->inner_target = fmax(sd.inner_rtol * rnorm, sd.final_safety * target);
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, bool kPaper>
__global__ void __launch_bounds__(kThreads) k_upd(const SolveDev *__restrict__ solves,
                                                  SolveScalars *__restrict__ sc,
                                                  const WorkItem *__restrict__ items, int n_items,
                                                  double *__restrict__ partials, int *n_active,
                                                  unsigned long long *__restrict__ cells) {
  __shared__ double red[kThreads / 32][kNumPartials];
  __shared__ int s_last;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const WorkItem item = items[it];
    const int s = item.solve;
    SolveScalars *scs = sc + s;
    const int phase = scs->phase;
    if (phase == kDone) continue;
    const SolveDev &sd = solves[s];
    const int oct_end = item.oct_begin + item.n_oct;
    double v[kNumPartials] = {0.0, 0.0, 0.0, 0.0};
    if (phase == kInner) {
      const T h = (T)sd.h;
      const T alpha = (T)scs->alpha;
      const T *p = (const T *)(scs->pcur ? sd.p0 : sd.p1);  // written by k_op this tick
      Acc<T> rz, rr;
      double maxchg = 0.0;
      for (int ob = item.oct_begin; ob < oct_end; ob += kOctsPerPass)
        upd_inner_pass<T, kPaper>(sd, ob, oct_end, h, alpha, p, rz, rr, maxchg);
      v[0] = rz.get();
      v[1] = rr.get();
      v[2] = maxchg;
      if (cells && threadIdx.x == 0) atomicAdd(cells + 2, (unsigned long long)item.n_oct * 8);
    } else {
      for (int ob = item.oct_begin; ob < oct_end; ob += kOctsPerPass)
        upd_refine_pass<T>(sd, ob, oct_end);
      if (cells && threadIdx.x == 0) atomicAdd(cells + 3, (unsigned long long)item.n_oct * 8);
    }
    block_reduce<true>(v, red);
    if (!publish_item(v, partials, it, scs, sd.n_items, &s_last)) continue;

    double tot[kNumPartials];
    solve_reduce<true>(partials, sd.item_begin, sd.n_items, tot, red);
    if (threadIdx.x == 0) {
      scs->counter = 0;
      scs->ticks += 1;
      if (phase == kInner) {
        scs->iters += 1;
        scs->inner_iters += 1;
        const double rz_new = tot[0];
        const double rnorm_in = sqrt(tot[1]);
        scs->maxchg = tot[2];
        if (scs->status == ATS_ERR_BREAKDOWN || !isfinite(rz_new) || rz_new < 0.0) {
          scs->status = ATS_ERR_BREAKDOWN;
          scs->phase = kDone;
          atomicSub(n_active, 1);
        } else {
          scs->beta = rz_new / scs->rz;
          scs->rz = rz_new;
          scs->first = 0;
          scs->pcur ^= 1;
          const bool conv = (rnorm_in <= scs->inner_target) && (!kPaper || tot[2] < sd.tol);
          if (conv || rz_new == 0.0) {
            scs->phase = kRefine;
          } else if (scs->iters >= sd.max_iter) {
            scs->status = ATS_ERR_NOT_CONVERGED;
            scs->final_pass = 1;
            scs->phase = kRefine;
          } else if (scs->inner_iters >= sd.inner_max) {
            scs->phase = kRefine;  // restart from the true residual
          }
        }
      } else {
        scs->phase = scs->phase_next;
        if (scs->phase == kDone) atomicSub(n_active, 1);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// coefficient build (one thread per cell)
// ---------------------------------------------------------------------------

__global__ void k_coef_build(CoefArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * a.n_oct) return;
  const int64_t o = i >> 3;
  const int c = (int)(i & 7);
  const bool leaf = a.leaf ? ((a.leaf[o] >> c) & 1) : true;
  const int xr = a.xrec[o];
  if (!leaf) {
    a.K64[i] = -1.0;
    a.K32[i] = -1.0f;
    a.b64[i] = 0.0;
    if (xr >= 0) {
      a.xd64[(int64_t)xr * 8 + c] = 0.0;
      a.xd32[(int64_t)xr * 8 + c] = 0.0f;
    }
    return;
  }
  const double K = a.K[i];
  const double E = a.E_old[i];
  bool ok = (K > 0.0) && isfinite(K) && isfinite(E);
  double xd = a.s ? a.s[i] : 0.0;
  ok = ok && isfinite(xd) && xd >= 0.0;
  double rhs = E + (a.src ? a.src[i] : 0.0);
  const int fr = a.frec[o];
  if (fr >= 0) {
    for (int dir = 0; dir < 6; ++dir) {
      const int f = a.rec_face[(int64_t)fr * 48 + c * 6 + dir];
      if (f < 0) continue;
      const double Kn = a.face_K ? a.face_K[f] : K;
      const double Enb = a.face_E ? a.face_E[f] : 0.0;
      const double F = a.face_F ? a.face_F[f] : 0.0;
      const double alpha = a.face_alpha ? a.face_alpha[f] : 1.0;
      ok = ok && (Kn > 0.0) && isfinite(Kn) && isfinite(Enb) && isfinite(F);
      const double factor = (a.face_rel[f] == ATS_REL_COARSER) ? (2.0 / 3.0) : 1.0;
      const double C = factor * a.h * (K + Kn);
      const int kind = a.face_kind[f];
      if (kind == ATS_FACE_DIRICHLET) {
        xd += C;
        rhs += C * Enb;
      } else if (kind == ATS_FACE_NEUMANN) {
        rhs += F;
      } else {
        xd += alpha * C;
        rhs += alpha * C * Enb + (1.0 - alpha) * F;
      }
    }
  }
  a.K64[i] = K;
  a.K32[i] = (float)K;
  a.b64[i] = rhs;
  if (xr >= 0) {
    a.xd64[(int64_t)xr * 8 + c] = xd;
    a.xd32[(int64_t)xr * 8 + c] = (float)xd;
  }
  if (!ok) atomicOr(a.err_flag, 1);
}

cudaError_t launch_coef_build(const CoefArgs &a, cudaStream_t st) {
  const int64_t N = 8 * a.n_oct;
  const int threads = 256;
  const int64_t blocks = (N + threads - 1) / threads;
  k_coef_build<<<(unsigned)blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// y = (I + dt A) x in FP64 (operator check / residual for callers)
// ---------------------------------------------------------------------------

__global__ void k_apply64(SolveDev sd, const double *__restrict__ x, double *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * (int64_t)sd.n_oct) return;
  const int o = (int)(i >> 3), c = (int)(i & 7);
  const double kv = sd.K64[i];
  if (kv < 0.0) {
    y[i] = 0.0;
    return;
  }
  double dsum = 0.0, off = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int m = 1 << a;
    // in-oct neighbour
    const int64_t jin = (int64_t)o * 8 + (c ^ m);
    const double kin = sd.K64[jin];
    if (kin >= 0.0) {
      const double C = sd.h * (kv + kin);
      dsum += C;
      off += C * x[jin];
    }
    const int nbo = sd.nbr[(int64_t)o * 6 + 2 * a + ((c >> a) & 1)];
    if (nbo >= 0) {
      const int64_t j = (int64_t)nbo * 8 + (c ^ m);
      const double kj = sd.K64[j];
      if (kj >= 0.0) {
        const double C = sd.h * (kv + kj);
        dsum += C;
        off += C * x[j];
      }
    }
  }
  const int rec = sd.xrec[o];
  const double xd = rec >= 0 ? sd.xd64[(int64_t)rec * 8 + c] : 0.0;
  y[i] = (1.0 + xd + dsum) * x[i] - off;
}

cudaError_t launch_apply64(const SolveDev *sd, const double *x, double *y, cudaStream_t st) {
  const int64_t N = 8 * (int64_t)sd->n_oct;
  const int threads = 256;
  k_apply64<<<(unsigned)((N + threads - 1) / threads), threads, 0, st>>>(*sd, x, y);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// tick launcher
// ---------------------------------------------------------------------------

static cudaError_t record(cudaEvent_t ev, cudaStream_t st, bool capture) {
  if (!ev) return cudaSuccess;
  return capture ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) : cudaEventRecord(ev, st);
}

template <typename T, bool kPaper>
static cudaError_t tick_impl(const SolveDev *solves, SolveScalars *sc, const WorkItem *items,
                             int n_items, double *partials, int *n_active, int grid,
                             cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, cudaEvent_t ev2,
                             bool capture, unsigned long long *cells) {
  cudaError_t err;
  if ((err = record(ev0, st, capture)) != cudaSuccess) return err;
  k_op<T><<<grid, kThreads, 0, st>>>(solves, sc, items, n_items, partials, cells);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if ((err = record(ev1, st, capture)) != cudaSuccess) return err;
  k_upd<T, kPaper><<<grid, kThreads, 0, st>>>(solves, sc, items, n_items, partials, n_active, cells);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return record(ev2, st, capture);
}

cudaError_t launch_tick(bool fp64, bool paper, const SolveDev *solves, SolveScalars *sc,
                        const WorkItem *items, int n_items, double *partials, int *n_active,
                        int grid, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1,
                        cudaEvent_t ev2, bool capture, unsigned long long *cells) {
  if (fp64) {
    return paper ? tick_impl<double, true>(solves, sc, items, n_items, partials, n_active, grid, st, ev0, ev1, ev2, capture, cells)
                 : tick_impl<double, false>(solves, sc, items, n_items, partials, n_active, grid, st, ev0, ev1, ev2, capture, cells);
  }
  return paper ? tick_impl<float, true>(solves, sc, items, n_items, partials, n_active, grid, st, ev0, ev1, ev2, capture, cells)
               : tick_impl<float, false>(solves, sc, items, n_items, partials, n_active, grid, st, ev0, ev1, ev2, capture, cells);
}

// ---------------------------------------------------------------------------
// solve start / end over the work list
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_init(const SolveDev *__restrict__ solves, const WorkItem *__restrict__ items,
                       int n_items, const double *const *__restrict__ src) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const WorkItem item = items[it];
    const SolveDev &sd = solves[item.solve];
    const double *xs = src ? src[item.solve] : nullptr;
    T *e = (T *)sd.e;
    const int64_t b = (int64_t)item.oct_begin * 8, n = (int64_t)item.n_oct * 8;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
      e[b + k] = T(0);
      if (xs) sd.x64[b + k] = xs[b + k];
    }
  }
}

__global__ void k_final(const SolveDev *__restrict__ solves, const WorkItem *__restrict__ items,
                        int n_items, double *const *__restrict__ dst) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const WorkItem item = items[it];
    double *xd = dst[item.solve];
    if (!xd) continue;
    const SolveDev &sd = solves[item.solve];
    const int64_t b = (int64_t)item.oct_begin * 8, n = (int64_t)item.n_oct * 8;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) xd[b + k] = sd.x64[b + k];
  }
}

cudaError_t launch_init(bool fp64, const SolveDev *solves, const WorkItem *items, int n_items,
                        const double *const *src, int grid, cudaStream_t st) {
  if (fp64) k_init<double><<<grid, kThreads, 0, st>>>(solves, items, n_items, src);
  else k_init<float><<<grid, kThreads, 0, st>>>(solves, items, n_items, src);
  return cudaGetLastError();
}

cudaError_t launch_final(const SolveDev *solves, const WorkItem *items, int n_items,
                         double *const *dst, int grid, cudaStream_t st) {
  k_final<<<grid, kThreads, 0, st>>>(solves, items, n_items, dst);
  return cudaGetLastError();
}

int tick_blocks_per_sm(bool fp64, bool paper) {
  int a = 0, b = 0;
  if (fp64) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_op<double>, kThreads, 0);
    if (paper) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_upd<double, true>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_upd<double, false>, kThreads, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_op<float>, kThreads, 0);
    if (paper) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_upd<float, true>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_upd<float, false>, kThreads, 0);
  }
  const int m = a < b ? a : b;
  return m > 0 ? m : 1;
}

}  // namespace ats
