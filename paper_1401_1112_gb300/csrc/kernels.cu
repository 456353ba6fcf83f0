// sm_103a kernels of the per-level implicit diffusion solve.
//
//  k_coef_build  cell diffusion coefficients, interface diagonal extras and the
//                right-hand side b (Sect. 3.1, Eq. Er_imp1; Sect. 3.2 rows).
//  k_op / k_ref / k_upd  one device "tick" of every solve in a work list.  A
//                solve in its CG phase does one iteration of the diagonal-
//                preconditioned CG of Sect. 3.3.4 (k_op: p = z + beta p,
//                q = (I + dt A) p, p.q; k_upd: e += alpha p, r = D z - alpha q,
//                z = D^-1 r, r.z, r.r); a solve in its refinement phase does
//                one FP64 true-residual pass r = b - (I + dt A) x (k_ref, on a
//                second stream beside k_op), the k_upd of its last inner
//                iteration having added x += e.
//
// Layout: a level is an array of octs; cell c = ix + 2 iy + 4 iz of oct o is
// element 8 o + c.  One thread owns one oct: its eight cells of every vector
// come in as one 32-byte load (two in FP64), the twelve in-oct faces are
// computed in registers, and the three out-of-oct faces of each cell come
// from the six face-neighbour octs (index table), of which only the four
// facing cells are loaded.  K < 0 marks a cell that is not an unknown of the
// level (refined cell); its vectors are kept at zero so it drops out.
//
// Work: a solve is split into work items (runs of octs); the tick kernels
// walk a device-side list of the items of the solves still running, which
// the update kernel rebuilds as solves finish.
//
// The operator is matrix-free: an interior face contributes
// C = dt/dx^2 (K_i + K_j)/2 = h (K_i + K_j); the diagonal is
// d_i = 1 + xd_i + sum_f C_f with xd_i (coupling shift + interface w C) read
// from a sparse per-oct record.
//
// Reductions: each work item (a run of octs of one solve) writes its partial
// sums; every CTA that needs a solve's totals in the next kernel reduces all
// of that solve's item partials itself in a fixed order (so all agree
// bitwise), and the CTA owning the solve's first item writes the solve's next
// state (double-buffered by tick parity).  No CTA ever waits for another.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <stdint.h>
#include <vector>

#include "ats_internal.h"

#ifndef ATS_BOUNDS_CHECK
#define ATS_BOUNDS_CHECK 0
#endif

namespace ats {

#if ATS_BOUNDS_CHECK
__device__ unsigned long long g_bound_violations;
#endif

namespace {

// Bounds-checked build (ATS_BOUNDS_CHECK=1): a gathered index (neighbour oct,
// record, face, work item, list entry) is tested against the length of the
// array it indexes before use; an index out of range is counted and the
// caller skips the access (a neighbour becomes "no neighbour", a work item
// becomes empty), so no kernel reads or writes outside its buffers.  In the
// default build the test is constant true and compiles away.
__device__ __forceinline__ bool idx_ok(long long i, long long n) {
#if ATS_BOUNDS_CHECK
  if (i >= 0 && i < n) return true;
  atomicAdd(&g_bound_violations, 1ull);
  return false;
#else
  (void)i;
  (void)n;
  return true;
#endif
}

// Neighbour octs: -1 (none) or an oct of the level.
__device__ __forceinline__ void check_nbr6(int (&nb)[6], int64_t n_oct) {
#pragma unroll
  for (int k = 0; k < 6; ++k)
    if (nb[k] >= 0 && !idx_ok(nb[k], n_oct)) nb[k] = -1;
}

// Octs of a work item that lie inside its solve's level (all of them unless
// the bounds-checked build finds the item out of range).
__device__ __forceinline__ int item_octs(const WorkItem &item, const SolveDev &sd) {
  if (!idx_ok(item.oct_begin, (long long)sd.n_oct + 1) || !idx_ok(item.n_oct, (long long)sd.n_oct + 1) ||
      !idx_ok((long long)item.oct_begin + item.n_oct, (long long)sd.n_oct + 1))
    return 0;
  return item.n_oct;
}

constexpr unsigned kFull = 0xffffffffu;
// resident CTAs per SM the CG tick kernels are compiled for (caps
// registers); the FP64 bulk path needs twice the registers per value.
#ifndef ATS_MINB_OP
#define ATS_MINB_OP 4
#endif
#ifndef ATS_MINB_UPD
#define ATS_MINB_UPD 4
#endif
template <typename T>
struct MinBlocks {  // k_op
  static constexpr int value = sizeof(T) == 4 ? ATS_MINB_OP : 3;
};
template <typename T>
struct MinBlocksUpd {
  static constexpr int value = sizeof(T) == 4 ? ATS_MINB_UPD : 3;
};

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
  __device__ __forceinline__ void add_value(double v) { s += v; }
  __device__ __forceinline__ void merge(const Acc<double> &o) { s += o.s; }
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ double val() const { return s; }
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
  // add one value exactly (TwoSum), the error going to the low part
  __device__ __forceinline__ void add_value(float v) {
    const float t = __fadd_rn(s, v);
    const float zz = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, zz)), __fsub_rn(v, zz));
    s = t;
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ void merge(const Acc<float> &o) {
    const float t = __fadd_rn(s, o.s);
    const float zz = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, zz)), __fsub_rn(o.s, zz));
    s = t;
    c = __fadd_rn(c, __fadd_rn(o.c, e));
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
  // the sum rounded to FP32 (no FP64 instruction)
  __device__ __forceinline__ float val() const { return __fadd_rn(s, c); }
};

// Warp reduction of a compensated FP32 accumulator: the (hi, lo) pairs are
// combined with TwoSum (error-free), so no FP64 instruction is issued per
// lane; lane 0 ends with the warp's pair.
__device__ __forceinline__ void warp_reduce_acc(Acc<float> &a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float s2 = __shfl_down_sync(kFull, a.s, off);
    const float c2 = __shfl_down_sync(kFull, a.c, off);
    const float t = __fadd_rn(a.s, s2);
    const float zz = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, zz)), __fsub_rn(s2, zz));
    a.s = t;
    a.c = __fadd_rn(a.c, __fadd_rn(c2, err));
  }
}
__device__ __forceinline__ void warp_reduce_acc(Acc<double> &a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a.s += __shfl_down_sync(kFull, a.s, off);
}


// ---------------------------------------------------------------------------
// oct-wise vector I/O (one thread owns the eight cells of one oct)
// ---------------------------------------------------------------------------

// 256-bit global accesses (sm_100 and later): the 32 bytes of an FP32 oct are
// one request (one L1 sector access instead of two 16-byte halves), an FP64
// oct is two.  Every oct base is 32-byte aligned: vectors are whole octs in
// device allocations aligned to 256 bytes (a caller's array is read or
// written with them only after its alignment was checked).  Read-only loads use the non-coherent path and may be scheduled
// freely; loads of data this kernel also writes are volatile so that they
// stay ordered with the stores.
__device__ __forceinline__ void ld8_ro(const float *__restrict__ p, float (&v)[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}
__device__ __forceinline__ void ld4_ro(const double *__restrict__ p, double &a, double &b, double &c, double &d) {
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p));
}
__device__ __forceinline__ void ld8_ro(const double *__restrict__ p, double (&v)[8]) {
  ld4_ro(p, v[0], v[1], v[2], v[3]);
  ld4_ro(p + 4, v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void ld8_rw(const float *p, float (&v)[8]) {
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}
__device__ __forceinline__ void ld8_rw(const double *p, double (&v)[8]) {
  asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
  asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
               : "=d"(v[4]), "=d"(v[5]), "=d"(v[6]), "=d"(v[7])
               : "l"(p + 4));
}
__device__ __forceinline__ void st8(float *p, const float (&v)[8]) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void st8(double *p, const double (&v)[8]) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
               : "memory");
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p + 4), "d"(v[4]), "d"(v[5]), "d"(v[6]), "d"(v[7])
               : "memory");
}

// Load the four cells of a neighbour oct that face this oct: the cells whose
// bit A equals NB (A = axis, NB = 1 - side of this oct's face).  v[c] is set
// for exactly those cells c.
template <int A, int NB>
__device__ __forceinline__ void ld_face(const float *__restrict__ p, float (&v)[8]) {
  if (A != 2) {
    ld8_ro(p, v);  // x and y faces: the whole oct in one 32-byte access
  } else {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p + 4 * NB));
    v[4 * NB] = a.x; v[4 * NB + 1] = a.y; v[4 * NB + 2] = a.z; v[4 * NB + 3] = a.w;
  }
}
template <int A, int NB>
__device__ __forceinline__ void ld_face(const double *__restrict__ p, double (&v)[8]) {
  if (A == 0) {
    ld8_ro(p, v);
  } else if (A == 1) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p + 2 * NB));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p + 4 + 2 * NB));
    v[2 * NB] = a.x; v[2 * NB + 1] = a.y; v[4 + 2 * NB] = b.x; v[5 + 2 * NB] = b.y;
  } else {
    ld4_ro(p + 4 * NB, v[4 * NB], v[4 * NB + 1], v[4 * NB + 2], v[4 * NB + 3]);
  }
}

// Coherent loads for the resident solver (one launch runs every iteration of
// a solve): vectors that another CTA of the cluster wrote earlier in the same
// launch are read from L2 (ld.global.cg) after the step's cluster barrier,
// never through the non-coherent read-only path.  asm volatile keeps them
// after that barrier.
#ifndef ATS_RES_LD
#define ATS_RES_LD ".cg"
#endif
__device__ __forceinline__ void ldc8(const float *p, float (&v)[8]) {
  asm volatile("ld.global" ATS_RES_LD ".v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}
__device__ __forceinline__ void ldc4(const double *p, double &a, double &b, double &c, double &d) {
  asm volatile("ld.global" ATS_RES_LD ".v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p));
}
__device__ __forceinline__ void ldc8(const double *p, double (&v)[8]) {
  ldc4(p, v[0], v[1], v[2], v[3]);
  ldc4(p + 4, v[4], v[5], v[6], v[7]);
}
template <int A, int NB>
__device__ __forceinline__ void ldc_face(const float *p, float (&v)[8]) {
  if (A != 2) {
    ldc8(p, v);
  } else {
    asm volatile("ld.global" ATS_RES_LD ".v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[4 * NB]), "=f"(v[4 * NB + 1]), "=f"(v[4 * NB + 2]), "=f"(v[4 * NB + 3])
                 : "l"(p + 4 * NB));
  }
}
template <int A, int NB>
__device__ __forceinline__ void ldc_face(const double *p, double (&v)[8]) {
  if (A == 0) {
    ldc8(p, v);
  } else if (A == 1) {
    asm volatile("ld.global" ATS_RES_LD ".v2.f64 {%0, %1}, [%2];" : "=d"(v[2 * NB]), "=d"(v[2 * NB + 1]) : "l"(p + 2 * NB));
    asm volatile("ld.global" ATS_RES_LD ".v2.f64 {%0, %1}, [%2];"
                 : "=d"(v[4 + 2 * NB]), "=d"(v[5 + 2 * NB])
                 : "l"(p + 4 + 2 * NB));
  } else {
    ldc4(p + 4 * NB, v[4 * NB], v[4 * NB + 1], v[4 * NB + 2], v[4 * NB + 3]);
  }
}
// kCoh: the vector may have been written by another CTA in this launch.
template <bool kCoh, typename T>
__device__ __forceinline__ void ldv8(const T *p, T (&v)[8]) {
  if (kCoh) ldc8(p, v);
  else ld8_ro(p, v);
}
template <int A, int NB, bool kCoh, typename T>
__device__ __forceinline__ void ldvf(const T *p, T (&v)[8]) {
  if (kCoh) ldc_face<A, NB>(p, v);
  else ld_face<A, NB>(p, v);
}

__device__ __forceinline__ void load_nbr6(const int32_t *__restrict__ nbr, int o, int (&nb)[6]) {
  const int2 *q = reinterpret_cast<const int2 *>(nbr + 6 * o);
  const int2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  nb[0] = a.x; nb[1] = a.y; nb[2] = b.x; nb[3] = b.y; nb[4] = c.x; nb[5] = c.y;
}

// The three in-oct faces of every cell, each cell pair once:
// off += C * v(neighbour), with C = h (K_i + K_j) between leaves.
template <typename T>
__device__ __forceinline__ void in_oct_faces(const T (&K)[8], const T (&v)[8], T h, T (&off)[8]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c & (1 << a)) continue;
      const int d = c | (1 << a);
      const T C = (K[c] >= T(0) && K[d] >= T(0)) ? h * (K[c] + K[d]) : T(0);
      off[c] += C * v[d];
      off[d] += C * v[c];
    }
  }
}

// ---------------------------------------------------------------------------
// per-oct work of each phase
// ---------------------------------------------------------------------------

// k_op, CG phase, out-of-oct face DIR: p_new of the neighbour's facing cells
// is formed on the fly from its z and p_old.
template <int DIR, typename T, bool kCoh = false>
__device__ __forceinline__ void op_face(int n, const T *__restrict__ KT, const T *__restrict__ z,
                                        const T *__restrict__ pold, bool first, T beta, T h,
                                        const T (&K)[8], T (&off)[8]) {
  constexpr int A = DIR >> 1, S = DIR & 1, NB = 1 - S;
  if (n < 0) return;
  T Kn[8], Zn[8], Pn[8];
  ld_face<A, NB>(KT + 8 * n, Kn);
  ldvf<A, NB, kCoh>(z + 8 * n, Zn);
  if (!first) ldvf<A, NB, kCoh>(pold + 8 * n, Pn);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (((c >> A) & 1) != S) continue;
    const int j = c ^ (1 << A);
    const T pj = first ? Zn[j] : fma(beta, Pn[j], Zn[j]);
    const T C = (Kn[j] >= T(0)) ? h * (K[c] + Kn[j]) : T(0);
    off[c] += C * pj;
  }
}

// k_ref, axis A of an oct: FP64 flux sums C (x_i - x_j) with the stored FP64
// face coefficients C = h (K_i + K_j) (row A of this oct for the in-oct pairs
// and the +A face, row A of the -A neighbour for the -A face), and the FP32
// diagonal sums of the bulk precision.
// The approximate reciprocal of the hardware (PTX rcp.approx, within one
// ulp): for the Jacobi step z = D^-1 r of the resident solver's FP32 bulk, one
// fixed value per cell for a whole inner solve, so the preconditioner stays
// a positive diagonal matrix.  D >= 1, so flushing subnormals changes nothing.
__device__ __forceinline__ float rcp_approx(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

template <int A, typename T, bool kCoh = false>
__device__ __forceinline__ void ref_axis(const SolveDev &sd, int o, const int (&nb)[6], const T *__restrict__ KT,
                                         T hT, const T (&KTo)[8], const double (&xv)[8], double (&acc)[8],
                                         T (&dsT)[8]) {
  constexpr int bit = 1 << A;
  double Cu[8];
  ld8_ro(sd.C64 + (3 * (size_t)o + A) * 8, Cu);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (c & bit) continue;
    const int d = c | bit;
    const double df = xv[c] - xv[d];
    acc[c] = fma(Cu[c], df, acc[c]);
    acc[d] = fma(-Cu[c], df, acc[d]);
    if (KTo[c] >= T(0) && KTo[d] >= T(0)) {
      const T Ct = hT * (KTo[c] + KTo[d]);
      dsT[c] += Ct;
      dsT[d] += Ct;
    }
  }
  int n = nb[2 * A + 1];  // +A face: this oct's cells with bit A set, C from row A of this oct
  if (n >= 0) {
    double Xn[8];
    T KTn[8];
    ldvf<A, 0, kCoh>(sd.x64 + 8 * n, Xn);
    ld_face<A, 0>(KT + 8 * n, KTn);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (!(c & bit)) continue;
      const int j = c ^ bit;
      acc[c] = fma(Cu[c], xv[c] - Xn[j], acc[c]);
      if (KTn[j] >= T(0)) dsT[c] += hT * (KTo[c] + KTn[j]);
    }
  }
  n = nb[2 * A];  // -A face: cells with bit A clear, C from row A of the -A neighbour
  if (n >= 0) {
    double Xn[8], Cn[8];
    T KTn[8];
    ldvf<A, 1, kCoh>(sd.x64 + 8 * n, Xn);
    ld_face<A, 1>(sd.C64 + (3 * (size_t)n + A) * 8, Cn);
    ld_face<A, 1>(KT + 8 * n, KTn);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c & bit) continue;
      const int j = c | bit;
      acc[c] = fma(Cn[j], xv[c] - Xn[j], acc[c]);
      if (KTn[j] >= T(0)) dsT[c] += hT * (KTo[c] + KTn[j]);
    }
  }
}

// k_ref: true residual r = b - (I + dt A) x in FP64 with the FP64 xd, b and
// face coefficients, written as r = b - (1 + xd) x - sum_f C_f (x_i - x_j)
// (every product a DFMA); z = r / D_T in the bulk precision, D_T stored for the
// CG kernels of the following inner solve.  Norms for the stopping test (r.r,
// x.x) and r.z are accumulated with compensated bulk-precision dots.
// The values of one oct (zo = z, dv = D); op_refine_oct stores them.
// kRcp (FP32 bulk): z = r x rcp(D_T) instead of the rounded quotient, the
// form the resident solver's CG steps use.
template <typename T, bool kCoh = false, bool kRcp = false>
__device__ __forceinline__ void ref_oct_values(const SolveDev &sd, int o, bool want_x, Acc<T> &rr, Acc<T> &xx,
                                               Acc<T> &rz, T (&zo)[8], T (&dv)[8]) {
  const T *__restrict__ KT = (const T *)sd.KT;
  constexpr bool mixed = sizeof(T) != sizeof(double);
  const T hT = (T)sd.h;
  int nb[6];
  load_nbr6(sd.nbr, o, nb);
  check_nbr6(nb, sd.n_oct);
  int rec = __ldg(sd.xrec + o);
  if (rec >= 0 && !idx_ok(rec, sd.n_xd)) rec = -1;
  double xv[8];
  T KTo[8];
  ldv8<kCoh>(sd.x64 + 8 * o, xv);
  ld8_ro(KT + 8 * o, KTo);
  double acc[8];
  T dsT[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    acc[c] = 0.0;
    dsT[c] = T(0);
  }
  ref_axis<0, T, kCoh>(sd, o, nb, KT, hT, KTo, xv, acc, dsT);
  ref_axis<1, T, kCoh>(sd, o, nb, KT, hT, KTo, xv, acc, dsT);
  ref_axis<2, T, kCoh>(sd, o, nb, KT, hT, KTo, xv, acc, dsT);
  double xd[8], b[8];
  T xdT[8];
  if (rec >= 0) {
    ld8_ro(sd.xd64 + 8 * rec, xd);
    if (mixed) ld8_ro((const T *)sd.xdT + 8 * rec, xdT);
  }
  ld8_ro(sd.b64 + 8 * o, b);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const bool leaf = KTo[c] >= T(0);
    const double base = rec >= 0 ? fma(-(1.0 + xd[c]), xv[c], b[c]) : b[c] - xv[c];
    const double r = base - acc[c];
    const T rT = (T)r;
    // D in the bulk precision, kept for the CG kernels of the following
    // inner solve
    const T dT = T(1) + (rec >= 0 ? (mixed ? xdT[c] : (T)xd[c]) : T(0)) + dsT[c];
    T zc;
    if constexpr (kRcp && sizeof(T) == 4) zc = rT * rcp_approx(dT);
    else zc = rT / dT;
    zo[c] = leaf ? zc : T(0);
    dv[c] = leaf ? dT : T(1);
    if (leaf) {
      rr.add(rT, rT);
      rz.add(rT, zc);
      if (want_x) {
        const T xT = (T)xv[c];
        xx.add(xT, xT);
      }
    }
  }
}

template <typename T, bool kCoh = false>
__device__ __forceinline__ void op_refine_oct(const SolveDev &sd, int o, bool want_x, Acc<T> &rr,
                                              Acc<T> &xx, Acc<T> &rz) {
  T zo[8], dv[8];
  ref_oct_values<T, kCoh>(sd, o, want_x, rr, xx, rz, zo, dv);
  st8((T *)sd.z + 8 * o, zo);
  st8((T *)sd.dg + 8 * o, dv);
}

// k_upd, refinement phase: x += e, e = 0.
template <typename T>
__device__ __forceinline__ void upd_refine_oct(const SolveDev &sd, int o) {
  T *e = (T *)sd.e;
  T ev[8];
  double xv[8];
  ld8_rw(e + 8 * o, ev);
  ld8_rw(sd.x64 + 8 * o, xv);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    xv[c] += (double)ev[c];
    ev[c] = T(0);
  }
  st8(sd.x64 + 8 * o, xv);
  st8(e + 8 * o, ev);
}

// ---------------------------------------------------------------------------
// per-item partial sums
//
// A work item stores kNumPartials sums.  In the FP32 bulk each sum is kept as
// an unevaluated (hi, lo) float pair (error-free TwoSum cascade), stored in
// the 8 bytes of a slot; in the FP64 bulk it is a double.  Every CTA that
// needs a solve's totals reduces all of that solve's item partials itself,
// in the same fixed order, so all CTAs obtain bitwise the same totals and no
// CTA ever signals or waits for another.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

template <typename T>
struct Slot;
template <>
struct Slot<float> {
  static __device__ __forceinline__ void store(double *p, const Acc<float> &a) {
    float2 v = make_float2(a.s, a.c);
    *reinterpret_cast<float2 *>(p) = v;
  }
  static __device__ __forceinline__ void load_add(const double *p, Acc<float> &a) {
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    float s, e;
    two_sum(a.s, v.x, s, e);
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(v.y, e));
  }
};
template <>
struct Slot<double> {
  static __device__ __forceinline__ void store(double *p, const Acc<double> &a) { *p = a.s; }
  static __device__ __forceinline__ void load_add(const double *p, Acc<double> &a) { a.s += __ldcg(p); }
};

// Block sums of three accumulators (and a max) of this CTA's item, reduced
// across warps in the accumulator precision; thread 0 writes the slots.
// There is no barrier after thread 0's merge: callers alternate between two
// red / redmx buffers by item, so a buffer is written again only after the
// next item's barrier, which thread 0 reaches after its merge.
template <typename T>
__device__ __forceinline__ void store_item_partials(double *slots, Acc<T> a0, Acc<T> a1, Acc<T> a2, float mx,
                                                    Acc<T> (*red)[3], float *redmx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_reduce_acc(a0);
  warp_reduce_acc(a1);
  warp_reduce_acc(a2);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_down_sync(kFull, mx, off));
  if (lane == 0) {
    red[warp][0] = a0;
    red[warp][1] = a1;
    red[warp][2] = a2;
    redmx[warp] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) {
#pragma unroll
      for (int k = 0; k < 3; ++k) red[0][k].merge(red[w][k]);
      redmx[0] = fmaxf(redmx[0], redmx[w]);
    }
    Slot<T>::store(slots + 0, red[0][0]);
    Slot<T>::store(slots + 1, red[0][1]);
    Slot<T>::store(slots + 2, red[0][2]);
    slots[3] = (double)redmx[0];
  }
}

// Totals over the items [begin, begin + n) of a solve, in one pass over the
// partials: sum 0 from slot k0 of P0, sums 1 and 2 from slots k1 and k2 of P1
// (a null array or a negative slot leaves the sum at zero) and, with
// want_max, the max of slot 3 of P1.  After one barrier every thread merges
// the warps' results itself, in the same order, so every thread holds
// bitwise the same totals.  red / redmx are not the buffers of
// store_item_partials (a warp may store its item sums while another thread
// still reads these).
template <typename T>
struct Totals {
  Acc<T> s[3];
  float mx;
};
template <typename T>
__device__ __forceinline__ void gather_totals(const double *P0, int k0, const double *P1, int k1, int k2,
                                              bool want_max, int begin, int n, Totals<T> &out, Acc<T> (*red)[3],
                                              float *redmx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Acc<T> acc[3];
  float mx = 0.f;
  for (int it = begin + (int)threadIdx.x; it < begin + n; it += kThreads) {
    const size_t base = (size_t)it * kNumPartials;
    if (P0) Slot<T>::load_add(P0 + base + k0, acc[0]);
    if (P1) {
      if (k1 >= 0) Slot<T>::load_add(P1 + base + k1, acc[1]);
      if (k2 >= 0) Slot<T>::load_add(P1 + base + k2, acc[2]);
      if (want_max) mx = fmaxf(mx, (float)__ldcg(P1 + base + 3));
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) warp_reduce_acc(acc[k]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_down_sync(kFull, mx, off));
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) red[warp][k] = acc[k];
    redmx[warp] = mx;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) out.s[k] = red[0][k];
  out.mx = redmx[0];
#pragma unroll
  for (int w = 1; w < kThreads / 32; ++w) {
#pragma unroll
    for (int k = 0; k < 3; ++k) out.s[k].merge(red[w][k]);
    out.mx = fmaxf(out.mx, redmx[w]);
  }
}

// ---------------------------------------------------------------------------
// per-oct work, split so that an oct's own loads are in flight while the CTA
// reduces the solve totals it needs
// ---------------------------------------------------------------------------

// The diagonal D = 1 + xd + sum C of an inner solve is the one its
// refinement pass stored, so k_op forms only the off-diagonal sums.
template <typename T>
struct OpOwn {
  int nb[6];
  T K[8], z[8], pp[8], d[8];
};

template <typename T, bool kCoh = false>
__device__ __forceinline__ void op_load_own(const SolveDev &sd, int o, bool first, const T *__restrict__ pold,
                                            OpOwn<T> &w) {
  load_nbr6(sd.nbr, o, w.nb);
  check_nbr6(w.nb, sd.n_oct);
  ld8_ro((const T *)sd.KT + 8 * o, w.K);
  ldv8<kCoh>((const T *)sd.z + 8 * o, w.z);
  ldv8<kCoh>((const T *)sd.dg + 8 * o, w.d);
  if (!first) ldv8<kCoh>(pold + 8 * o, w.pp);
}

// k_op, CG phase: p_new = z + beta p_old (first: z), q = (I + dt A) p_new,
// partial p_new . q (per-oct FP32 sum, carried error-free across octs).
template <typename T, bool kCoh = false>
__device__ __forceinline__ void op_compute(const SolveDev &sd, int o, const OpOwn<T> &w, T h, T beta, bool first,
                                           const T *__restrict__ pold, T *__restrict__ pnew, Acc<T> &pq) {
  const T *__restrict__ KT = (const T *)sd.KT;
  const T *__restrict__ z = (const T *)sd.z;
  T pv[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) pv[c] = first ? w.z[c] : fma(beta, w.pp[c], w.z[c]);
  T off[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) off[c] = T(0);
  in_oct_faces(w.K, pv, h, off);
  op_face<0, T, kCoh>(w.nb[0], KT, z, pold, first, beta, h, w.K, off);
  op_face<1, T, kCoh>(w.nb[1], KT, z, pold, first, beta, h, w.K, off);
  op_face<2, T, kCoh>(w.nb[2], KT, z, pold, first, beta, h, w.K, off);
  op_face<3, T, kCoh>(w.nb[3], KT, z, pold, first, beta, h, w.K, off);
  op_face<4, T, kCoh>(w.nb[4], KT, z, pold, first, beta, h, w.K, off);
  op_face<5, T, kCoh>(w.nb[5], KT, z, pold, first, beta, h, w.K, off);
  T local = T(0), qv[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T q = w.d[c] * pv[c] - off[c];
    const bool leaf = w.K[c] >= T(0);
    if (leaf) local = fma(pv[c], q, local);
    qv[c] = leaf ? q : T(0);
  }
  pq.add_value(local);
  st8(pnew + 8 * o, pv);  // non-leaf cells carry z = p = 0
  st8((T *)sd.q + 8 * o, qv);
}

// k_upd, CG phase: nothing but the oct's own values.  q = (I + dt A) p was
// stored by k_op and D by the refinement pass, so no neighbour is read.
template <typename T>
struct UpdOwn {
  T p[8], q[8], d[8], z[8], e[8];
};

template <typename T, bool kCoh = false>
__device__ __forceinline__ void upd_load_own(const SolveDev &sd, int o, const T *__restrict__ p, UpdOwn<T> &w) {
  if (kCoh) {  // every vector is rewritten within a resident launch
    ldc8(p + 8 * o, w.p);
    ldc8((const T *)sd.q + 8 * o, w.q);
    ldc8((const T *)sd.dg + 8 * o, w.d);
    ldc8((const T *)sd.z + 8 * o, w.z);
    ldc8((const T *)sd.e + 8 * o, w.e);
    return;
  }
  // p, q (this tick's k_op) and D (a refinement pass) are read-only here
  ld8_ro(p + 8 * o, w.p);
  ld8_ro((const T *)sd.q + 8 * o, w.q);
  ld8_ro((const T *)sd.dg + 8 * o, w.d);
  ld8_rw((const T *)sd.z + 8 * o, w.z);
  ld8_rw((const T *)sd.e + 8 * o, w.e);
}

// r = D z - alpha q, z = r / D, e += alpha p; partials r.z, r.r (and the max
// relative change for the paper rule).  Off the leaves p = q = z = 0 and
// D = 1, so those cells stay zero.
template <typename T, bool kPaper>
__device__ __forceinline__ void upd_compute(const SolveDev &sd, int o, UpdOwn<T> &w, T alpha, Acc<T> &rz,
                                            Acc<T> &rr, float &maxchg) {
  double xo[8];
  if (kPaper) ld8_rw(sd.x64 + 8 * o, xo);
  T lrz = T(0), lrr = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T r = w.d[c] * w.z[c] - alpha * w.q[c];
    const T zn = r / w.d[c];
    const T step = alpha * w.p[c];
    lrz = fma(r, zn, lrz);
    lrr = fma(r, r, lrr);
    if (kPaper && step != T(0)) maxchg = fmaxf(maxchg, (float)(fabs((double)step) / fabs(xo[c] + (double)w.e[c])));
    w.z[c] = zn;
    w.e[c] += step;
  }
  rz.add_value(lrz);
  rr.add_value(lrr);
  st8((T *)sd.z + 8 * o, w.z);
  st8((T *)sd.e + 8 * o, w.e);
}

}  // namespace

// ---------------------------------------------------------------------------
// the three tick kernels (persistent grid, grid-stride over the active lists)
// ---------------------------------------------------------------------------

// The list of one phase for a parity: lists[(parity * 2 + phase) * n_items].
__device__ __forceinline__ int32_t *phase_list(int32_t *lists, int n_items, int parity, int phase) {
  return lists + (size_t)(parity * 2 + phase) * n_items;
}

// Descriptors of a batch of this CTA's work items, staged in shared memory:
// list positions li0, li0 + G, ... (G = gridDim.x; positions below n0 are in
// list0, the others in list1 at li - n0), each with its item, its solve's
// descriptor and scalars.  The three dependent global reads (list entry,
// item, solve) are paid once per batch instead of once per item.
constexpr int kBatch = 32;
struct ItemSlot {
  SolveDev sd;
  SolveScalars sc;
  WorkItem item;
  int32_t it;
  int32_t inner;  // from list0
  int32_t pad[2];
};
static_assert(sizeof(SolveDev) % 8 == 0 && sizeof(SolveScalars) % 8 == 0, "descriptors are copied as 8-byte words");

__device__ __forceinline__ int stage_items(const TickArgs &a, const int32_t *list0, int n0, const int32_t *list1,
                                           int n, int li0, const SolveScalars *S, ItemSlot *slots) {
  const int G = (int)gridDim.x;
  const int left = (n - li0 + G - 1) / G;
  const int m = left < kBatch ? left : kBatch;
  if ((int)threadIdx.x < m) {
    const int li = li0 + (int)threadIdx.x * G;
    const bool in0 = li < n0;
    int it = in0 ? __ldcg(list0 + li) : __ldcg(list1 + (li - n0));
    if (!idx_ok(it, a.n_items)) it = 0;
    slots[threadIdx.x].it = it;
    slots[threadIdx.x].inner = in0 ? 1 : 0;
    WorkItem item = a.items[it];
    if (!idx_ok(item.solve, a.n_solves)) {
      item.solve = 0;
      item.n_oct = 0;
    }
    slots[threadIdx.x].item = item;
  }
  __syncthreads();
  constexpr int wd = (int)(sizeof(SolveDev) / 8), ws = (int)(sizeof(SolveScalars) / 8);
  for (int w = threadIdx.x; w < m * (wd + ws); w += kThreads) {
    const int k = w / (wd + ws), j = w - k * (wd + ws);
    const int sv = slots[k].item.solve;
    if (j < wd) {
      reinterpret_cast<unsigned long long *>(&slots[k].sd)[j] =
          reinterpret_cast<const unsigned long long *>(a.solves + sv)[j];
    } else {
      reinterpret_cast<unsigned long long *>(&slots[k].sc)[j - wd] =
          __ldcg(reinterpret_cast<const unsigned long long *>(S + sv) + (j - wd));
    }
  }
  __syncthreads();
  return m;
}

// CG items: p = z + beta p, q = (I + dt A) p, partial p.q.  k_op and k_ref
// touch disjoint solves (CG-phase and refinement-phase lists) and may run
// concurrently.
template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_op(TickArgs a) {
  __shared__ Acc<T> red[2][kThreads / 32][3], red2[kThreads / 32][3];
  __shared__ float redmx[2][kThreads / 32], redmx2[kThreads / 32];
  int buf = 0;
  const int cur = __ldcg(&a.ctl->parity);
  const int n_in = __ldcg(&a.ctl->count[cur][kInner]);
  const int32_t *list = phase_list(a.lists, a.n_items, cur, kInner);
  const SolveScalars *S = a.sbuf + (size_t)cur * a.n_solves;
  const double *Pprev = a.p_upd + (size_t)(cur ^ 1) * a.n_items * kNumPartials;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl->count[cur ^ 1][0] = 0;
    a.ctl->count[cur ^ 1][1] = 0;
  }
  __shared__ ItemSlot slots[kBatch];
  for (int li0 = blockIdx.x; li0 < n_in; li0 += kBatch * gridDim.x) {
  const int m = stage_items(a, list, n_in, nullptr, n_in, li0, S, slots);
  for (int bi = 0; bi < m; ++bi) {
    const int it = slots[bi].it;
    const WorkItem item = slots[bi].item;
    const SolveDev &sd = slots[bi].sd;
    const SolveScalars &sc = slots[bi].sc;
    const bool first = sc.first != 0;
    const int pcur = sc.pcur;
    const double rz_prev = sc.rz;
    const T *pold = (const T *)(pcur ? sd.p1 : sd.p0);
    T *pnew = (T *)(pcur ? sd.p0 : sd.p1);
    const int oct_end = item.oct_begin + item_octs(item, sd);
    const int o0 = item.oct_begin + (int)threadIdx.x;
    OpOwn<T> w;
    if (o0 < oct_end) op_load_own(sd, o0, first, pold, w);
    // beta = (r_j . z_j) / (r_{j-1} . z_{j-1}) from the previous update's partials
    // (every thread, in the bulk precision)
    T beta = T(0);
    if (!first) {
      Totals<T> tt;
      gather_totals<T>(nullptr, 0, Pprev, 0, -1, false, sd.item_begin, sd.n_items, tt, red2, redmx2);
      beta = tt.s[1].val() / (T)rz_prev;
    }
    const T h = (T)sd.h;
    Acc<T> pq, none;
    if (o0 < oct_end) op_compute(sd, o0, w, h, beta, first, pold, pnew, pq);
    for (int o = o0 + kThreads; o < oct_end; o += kThreads) {
      op_load_own(sd, o, first, pold, w);
      op_compute(sd, o, w, h, beta, first, pold, pnew, pq);
    }
    store_item_partials<T>(a.p_op + (size_t)it * kNumPartials, pq, none, none, 0.f, red[buf], redmx[buf]);
    buf ^= 1;
    if (a.cells && threadIdx.x == 0) atomicAdd(a.cells + (first ? 4 : 0), (unsigned long long)item.n_oct * 8);
  }
  __syncthreads();  // the slots are restaged
  }
}

// Refinement items: FP64 true residual, z = D^-1 r, partials r.r, x.x, r.z.
template <typename T>
__global__ void __launch_bounds__(kThreads, 3) k_ref(TickArgs a) {
  __shared__ Acc<T> red[2][kThreads / 32][3];
  __shared__ float redmx[2][kThreads / 32];
  int buf = 0;
  const int cur = __ldcg(&a.ctl->parity);
  const int n_rf = __ldcg(&a.ctl->count[cur][kRefine]);
  const int32_t *list = phase_list(a.lists, a.n_items, cur, kRefine);
  const SolveScalars *S = a.sbuf + (size_t)cur * a.n_solves;
  __shared__ ItemSlot slots[kBatch];
  for (int li0 = blockIdx.x; li0 < n_rf; li0 += kBatch * gridDim.x) {
  const int m = stage_items(a, list, n_rf, nullptr, n_rf, li0, S, slots);
  for (int bi = 0; bi < m; ++bi) {
    const int it = slots[bi].it;
    const WorkItem item = slots[bi].item;
    const SolveDev &sd = slots[bi].sd;
    const int oct_end = item.oct_begin + item_octs(item, sd);
    Acc<T> rr, xx, rz;
    const bool want_x = sd.stop_rule == ATS_STOP_CERTIFIED;
    for (int o = item.oct_begin + (int)threadIdx.x; o < oct_end; o += kThreads)
      op_refine_oct<T>(sd, o, want_x, rr, xx, rz);
    store_item_partials<T>(a.p_op + (size_t)it * kNumPartials, rr, xx, rz, 0.f, red[buf], redmx[buf]);
    buf ^= 1;
    if (a.cells && threadIdx.x == 0) atomicAdd(a.cells + 1, (unsigned long long)item.n_oct * 8);
  }
  __syncthreads();  // the slots are restaged
  }
}

// Append a solve's items to the next tick's list of its new phase (the CTA
// that owns the solve's first item), or retire it.
__device__ __forceinline__ void commit_solve(const TickArgs &a, int cur, int s, const SolveDev &sd,
                                             const SolveScalars &next, int *s_base) {
  if (threadIdx.x == 0) {
    a.sbuf[(size_t)(cur ^ 1) * a.n_solves + s] = next;
    if (next.phase == kDone) {
      a.final_sc[s] = next;
      atomicSub(a.n_active, 1);
      *s_base = -1;
    } else {
      *s_base = atomicAdd(&a.ctl->count[cur ^ 1][next.phase], sd.n_items);
    }
  }
  __syncthreads();
  int base = *s_base;
  if (base >= 0 && !idx_ok((long long)base + sd.n_items - 1, a.n_items)) base = -1;
  if (base >= 0) {
    int32_t *nl = phase_list(a.lists, a.n_items, cur ^ 1, next.phase);
    for (int k = threadIdx.x; k < sd.n_items; k += kThreads) nl[base + k] = sd.item_begin + k;
  }
  __syncthreads();
}

// CG items: alpha = r.z / p.q, e += alpha p, r = D z - alpha q, z = r / D;
// partials r.z, r.r (max change).  Before updating, the previous update's
// residual decides whether the inner solve has converged (then nothing is
// updated and the solve goes to refinement).  Refinement items: the decision
// after a true-residual pass.  The CTA owning a solve's first item writes the
// solve's next state and list entries.
template <typename T, bool kPaper>
__global__ void __launch_bounds__(kThreads, MinBlocksUpd<T>::value) k_upd(TickArgs a) {
  __shared__ Acc<T> red[2][kThreads / 32][3], red2[kThreads / 32][3];
  __shared__ float redmx[2][kThreads / 32], redmx2[kThreads / 32];
  __shared__ int s_base;
  int buf = 0;
  const int cur = __ldcg(&a.ctl->parity);
  const int n_in = __ldcg(&a.ctl->count[cur][kInner]);
  const int n_list = n_in + __ldcg(&a.ctl->count[cur][kRefine]);
  const SolveScalars *S = a.sbuf + (size_t)cur * a.n_solves;
  const double *Pprev = a.p_upd + (size_t)(cur ^ 1) * a.n_items * kNumPartials;
  double *Pcur = a.p_upd + (size_t)cur * a.n_items * kNumPartials;
  __shared__ ItemSlot slots[kBatch];
  for (int li0 = blockIdx.x; li0 < n_list; li0 += kBatch * gridDim.x) {
  const int m = stage_items(a, phase_list(a.lists, a.n_items, cur, kInner), n_in,
                            phase_list(a.lists, a.n_items, cur, kRefine), n_list, li0, S, slots);
  for (int bi = 0; bi < m; ++bi) {
    const bool inner = slots[bi].inner != 0;
    const int it = slots[bi].it;
    const WorkItem item = slots[bi].item;
    const int s = item.solve;
    const SolveDev &sd = slots[bi].sd;
    const SolveScalars &sc = slots[bi].sc;
    const bool owner = (it == sd.item_begin);
    if (inner) {
      const bool first = sc.first != 0;
      const T *p = (const T *)(sc.pcur ? sd.p0 : sd.p1);  // written by k_op this tick
      const int oct_end = item.oct_begin + item_octs(item, sd);
      const int o0 = item.oct_begin + (int)threadIdx.x;
      UpdOwn<T> w;
      if (o0 < oct_end) upd_load_own(sd, o0, p, w);
      // p.q of this tick and, after the first iteration, r.z and r.r of the
      // previous update: one pass over the solve's partials
      Totals<T> tt;
      gather_totals<T>(a.p_op, 0, first ? nullptr : Pprev, 0, 1, kPaper && !first, sd.item_begin, sd.n_items, tt,
                       red2, redmx2);
      const T pq = tt.s[0].val();
      const T rz_j = first ? (T)sc.rz : tt.s[1].val();
      const T rr_j = first ? T(0) : tt.s[2].val();
      const float mx = tt.mx;
      // the scalar decisions, taken by every thread from the same totals in
      // the bulk precision (sqrt(r.r) <= target as r.r <= target^2)
      const T target2 = sizeof(T) == 4 ? (T)sc.inner_t2 : (T)(sc.inner_target * sc.inner_target);
      const bool conv = !first && ((rr_j <= target2 && (!kPaper || mx < (float)sd.tol)) || rz_j == T(0));
      const bool brk = !conv && (!(rz_j >= T(0)) || !isfinite(rz_j) || !(pq > T(0)) || !isfinite(pq));
      const T alpha = (conv || brk) ? T(0) : rz_j / pq;
      Acc<T> rz, rr, none;
      float maxchg = 0.f;
      if (!conv && !brk) {
        if (o0 < oct_end) upd_compute<T, kPaper>(sd, o0, w, alpha, rz, rr, maxchg);
        for (int o = o0 + kThreads; o < oct_end; o += kThreads) {
          upd_load_own(sd, o, p, w);
          upd_compute<T, kPaper>(sd, o, w, alpha, rz, rr, maxchg);
        }
      }
      // the inner solve ends here (converged, or an iteration cap sends the
      // solve to a true-residual pass): x += e, e = 0 on this item, so the
      // next tick's k_ref reads the corrected x
      const bool to_ref =
          conv || (!brk && (sc.iters + 1 >= sd.max_iter || sc.inner_iters + 1 >= sd.inner_max));
      if (to_ref) {
        for (int o = o0; o < oct_end; o += kThreads) upd_refine_oct<T>(sd, o);
        if (a.cells && threadIdx.x == 0) atomicAdd(a.cells + 3, (unsigned long long)item.n_oct * 8);
      }
      store_item_partials<T>(Pcur + (size_t)it * kNumPartials, rz, rr, none, maxchg, red[buf], redmx[buf]);
      buf ^= 1;
      if (a.cells && threadIdx.x == 0 && !conv && !brk) atomicAdd(a.cells + 2, (unsigned long long)item.n_oct * 8);
      if (owner) {
        SolveScalars nx = sc;
        nx.ticks += 1;
        if (conv) {
          nx.phase = kRefine;
        } else if (brk) {
          nx.status = ATS_ERR_BREAKDOWN;
          nx.phase = kDone;
        } else {
          nx.iters += 1;
          nx.inner_iters += 1;
          nx.first = 0;
          nx.pcur ^= 1;
          nx.rz = first ? sc.rz : tt.s[1].get();
          nx.maxchg = mx;
          if (nx.iters >= sd.max_iter) {
            nx.status = ATS_ERR_NOT_CONVERGED;
            nx.final_pass = 1;
            nx.phase = kRefine;
          } else if (nx.inner_iters >= sd.inner_max) {
            nx.phase = kRefine;  // restart from the true residual
          }
        }
        commit_solve(a, cur, s, sd, nx, &s_base);
      }
    } else {
      // only the owner CTA decides after a true-residual pass
      if (owner) {
        Totals<T> tt;
        gather_totals<T>(a.p_op, 0, a.p_op, 1, 2, false, sd.item_begin, sd.n_items, tt, red2, redmx2);
        const double t[3] = {tt.s[0].get(), tt.s[1].get(), tt.s[2].get()};
        SolveScalars nx = sc;
        nx.ticks += 1;
        const double rnorm = sqrt(t[0]);
        const double xnorm = sqrt(t[1]);
        if (nx.refines == 0) nx.r0 = rnorm;
        nx.refines += 1;
        nx.rnorm = rnorm;
        nx.xnorm = xnorm;
        const double ref = (sd.stop_rule == ATS_STOP_CERTIFIED) ? xnorm : nx.r0;
        const double target = sd.tol * ref;
        if (nx.final_pass) {
          nx.phase = kDone;
        } else if (!isfinite(rnorm)) {
          nx.status = ATS_ERR_BREAKDOWN;
          nx.phase = kDone;
        } else if (rnorm <= target) {
          nx.phase = kDone;
        } else if (nx.refines > sd.max_refine) {
          nx.status = ATS_ERR_NOT_CONVERGED;
          nx.phase = kDone;
        } else if (!(t[2] > 0.0)) {
          nx.status = ATS_ERR_BREAKDOWN;
          nx.phase = kDone;
        } else {
          nx.phase = kInner;
          nx.rz = t[2];
          nx.first = 1;
          nx.inner_iters = 0;
          nx.inner_target = fmax(sd.inner_rtol * rnorm, sd.final_safety * target);
          nx.inner_t2 = (float)(nx.inner_target * nx.inner_target);
        }
        commit_solve(a, cur, s, sd, nx, &s_base);
      }
    }
  }
  __syncthreads();  // the slots are restaged
  }
  // the last CTA of the grid flips the list parity for the next tick
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.ctl->cta_done, 1) == (int)gridDim.x - 1) {
      a.ctl->cta_done = 0;
      a.ctl->parity = cur ^ 1;
      __threadfence();
    }
  }
}


// ---------------------------------------------------------------------------
// coefficient build (one thread per cell)
// ---------------------------------------------------------------------------

// FP64 coefficients of the +x, +y, +z faces of leaf cell i = 8 o + c from the
// input K (the same values the face-coefficient pass derives from K64):
// h (K_i + K_j) when the +a neighbour j (in-oct partner, or the facing cell
// of the +a neighbour oct) is a leaf, else 0.
__device__ __forceinline__ void coef_faces(const CoefArgs &a, int64_t o, int c, bool leaf, double K) {
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int bit = 1 << ax;
    int64_t oj = -1;
    int cj = c ^ bit;
    if (!(c & bit)) {
      oj = o;
    } else {
      const int n = a.nbr[6 * o + 2 * ax + 1];
      if (n >= 0 && idx_ok(n, a.n_oct)) oj = n;
    }
    double C = 0.0;
    if (leaf && oj >= 0 && (!a.leaf || ((a.leaf[oj] >> cj) & 1))) C = a.h * (K + a.K[8 * oj + cj]);
    a.C64[(3 * o + ax) * 8 + c] = C;
  }
}

__device__ __forceinline__ void coef_cell(const CoefArgs &a, int64_t i) {
  const int64_t o = i >> 3;
  const int c = (int)(i & 7);
  const bool leaf = a.leaf ? ((a.leaf[o] >> c) & 1) : true;
  int xr = a.xrec[o];
  if (xr >= 0 && !idx_ok(xr, a.n_xd)) xr = -1;
  if (!leaf) {
    a.K64[i] = -1.0;
    a.K32[i] = -1.0f;
    a.b64[i] = 0.0;
    coef_faces(a, o, c, false, 0.0);
    if (xr >= 0) {
      a.xd64[(int64_t)xr * 8 + c] = 0.0;
      a.xd32[(int64_t)xr * 8 + c] = 0.0f;
    }
    return;
  }
  const double K = a.K[i];
  coef_faces(a, o, c, true, K);
  const double E = a.E_old[i];
  bool ok = (K > 0.0) && isfinite(K) && isfinite(E);
  double xd = a.s ? a.s[i] : 0.0;
  ok = ok && isfinite(xd) && xd >= 0.0;
  double rhs = E + (a.src ? a.src_scale * a.src[i] : 0.0);
  int fr = a.frec[o];
  if (fr >= 0 && !idx_ok(fr, a.n_rec)) fr = -1;
  if (fr >= 0) {
    for (int dir = 0; dir < 6; ++dir) {
      const int f = a.rec_face[(int64_t)fr * 48 + c * 6 + dir];
      if (f < 0 || !idx_ok(f, a.n_face)) continue;
      const double Kn = a.face_K ? a.face_K[f] : K;
      const double Enb = a.face_E ? a.face_E[f] : 0.0;
      const double F = a.face_F ? a.src_scale * a.face_F[f] : 0.0;
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

__global__ void k_coef_build(CoefArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * a.n_oct) return;
  coef_cell(a, i);
}

// All levels of a batch in one launch: block b belongs to level
// blk_level[b] and covers its cells from (b - blk_first[level]) * blockDim.
__global__ void k_coef_build_batch(const CoefArgs *__restrict__ args, const int32_t *__restrict__ blk_level,
                                   const int32_t *__restrict__ blk_first) {
  // the block's level arguments, copied once into shared memory: every
  // thread reads a dozen of their fields
  static_assert(sizeof(CoefArgs) % 8 == 0, "CoefArgs is copied as 8-byte words");
  __shared__ unsigned long long sa[sizeof(CoefArgs) / 8];
  const int k = blk_level[blockIdx.x];
  const unsigned long long *src = reinterpret_cast<const unsigned long long *>(args + k);
  for (int w = threadIdx.x; w < (int)(sizeof(CoefArgs) / 8); w += blockDim.x) sa[w] = src[w];
  __syncthreads();
  const CoefArgs &a = *reinterpret_cast<const CoefArgs *>(sa);
  const int64_t i = (int64_t)(blockIdx.x - blk_first[k]) * blockDim.x + threadIdx.x;
  if (i < 8 * a.n_oct) coef_cell(a, i);
}

// The FP64 face coefficients of cell i = 8 o + c: for each axis a, the face
// towards +a (the in-oct partner when bit a of c is 0, else the facing cell of
// the +a neighbour oct).
__device__ __forceinline__ void face_coef_cell(const int32_t *__restrict__ nbr, const double *__restrict__ K64,
                                               double h, double *__restrict__ C64, int64_t i, int64_t n_oct) {
  const int64_t o = i >> 3;
  const int c = (int)(i & 7);
  const double Ki = K64[i];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int bit = 1 << ax;
    int64_t j = -1;
    if (!(c & bit)) {
      j = 8 * o + (c | bit);
    } else {
      const int n = nbr[6 * o + 2 * ax + 1];
      if (n >= 0 && idx_ok(n, n_oct)) j = 8 * (int64_t)n + (c ^ bit);
    }
    double C = 0.0;
    if (j >= 0) {
      const double Kj = K64[j];
      if (Ki >= 0.0 && Kj >= 0.0) C = h * (Ki + Kj);
    }
    C64[(3 * o + ax) * 8 + c] = C;
  }
}

__global__ void k_face_coef(int64_t n_oct, const int32_t *__restrict__ nbr, const double *__restrict__ K64,
                            double h, double *__restrict__ C64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 8 * n_oct) face_coef_cell(nbr, K64, h, C64, i, n_oct);
}

__global__ void k_zero_flags(int *const *__restrict__ flags, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) *flags[k] = 0;
}

__global__ void k_gather_flags(const int *const *__restrict__ flags, int n, int *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = *flags[k];
}

cudaError_t launch_coef_build_batch(const CoefArgs *args, const int32_t *blk_level, const int32_t *blk_first,
                                    int n_blocks, int n, int *const *flags, cudaStream_t st) {
  k_zero_flags<<<(n + 255) / 256, 256, 0, st>>>(flags, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_blocks == 0) return e;
  k_coef_build_batch<<<(unsigned)n_blocks, kCoefThreads, 0, st>>>(args, blk_level, blk_first);
  return cudaGetLastError();
}

cudaError_t launch_face_coef(int64_t n_oct, const int32_t *nbr, const double *K64, double h, double *C64,
                             cudaStream_t st) {
  if (n_oct <= 0) return cudaSuccess;
  const int64_t N = 8 * n_oct;
  k_face_coef<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(n_oct, nbr, K64, h, C64);
  return cudaGetLastError();
}

cudaError_t launch_gather_flags(const int *const *flags, int n, int *out, cudaStream_t st) {
  k_gather_flags<<<(n + 255) / 256, 256, 0, st>>>(flags, n, out);
  return cudaGetLastError();
}

cudaError_t launch_coef_build(const CoefArgs &a, cudaStream_t st) {
  const int64_t N = 8 * a.n_oct;
  const int threads = 256;
  const int64_t blocks = (N + threads - 1) / threads;
  k_coef_build<<<(unsigned)blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// AMR level coupling (Sect. 3.3.1-3.3.2): restriction and ghost gather
// ---------------------------------------------------------------------------

// Restriction: the value of a refined cell R of level l is the mean of its
// eight children (the child oct at level l+1), for E and for K.
__global__ void k_flux_store(int n_face, const int32_t *__restrict__ gather4, const int32_t *__restrict__ fcell,
                             const double *__restrict__ x, const double *__restrict__ K,
                             const double *__restrict__ fK, const double *__restrict__ fE, double hf,
                             double *__restrict__ store) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_face) return;
  double acc = 0.0;
  bool any = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int g = gather4[4 * f + k];
    if (g < 0) continue;
    const int cell = fcell[g];
    acc += (2.0 / 3.0) * hf * (K[cell] + fK[g]) * (x[cell] - fE[g]);
    any = true;
  }
  if (any) store[f] += acc / 8.0;
}

cudaError_t launch_flux_store(int n_face, const int32_t *gather4, const int32_t *fcell, const double *x,
                              const double *K, const double *fK, const double *fE, double h_f, double *store,
                              cudaStream_t st) {
  if (n_face <= 0) return cudaSuccess;
  k_flux_store<<<(n_face + 127) / 128, 128, 0, st>>>(n_face, gather4, fcell, x, K, fK, fE, h_f, store);
  return cudaGetLastError();
}

__global__ void k_restrict(int n, const int32_t *__restrict__ cell, const int32_t *__restrict__ child,
                           const double *__restrict__ Ef, const double *__restrict__ Kf,
                           double *__restrict__ Ec, double *__restrict__ Kc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t co = (int64_t)child[i] * 8;
  double se = 0.0, sk = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    se += Ef[co + c];
    sk += Kf[co + c];
  }
  Ec[cell[i]] = se * 0.125;
  Kc[cell[i]] = sk * 0.125;
}

// Ghost gather: the neighbour value and K of every interface face of a level.
// rel 0: a refined cell of the same level (its restricted value);
// rel 1: a coarser leaf, at time t^n + theta (t^{n+1} - t^n) of the coarser
// step (theta = 0 holds the coarse value at E^n).
__global__ void k_gather_faces(int n_face, const int8_t *__restrict__ src_rel, const int32_t *__restrict__ src_cell,
                               const double *__restrict__ E_same, const double *__restrict__ K_same,
                               const double *__restrict__ Ec_old, const double *__restrict__ Ec_new,
                               const double *__restrict__ K_coarse, double theta, double *__restrict__ fE,
                               double *__restrict__ fK, const double *__restrict__ wall) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_face) return;
  const int64_t j = src_cell[f];
  if (src_rel[f] == 0) {
    fE[f] = E_same[j];
    fK[f] = K_same[j];
  } else if (src_rel[f] == 2) {  // Dirichlet side of the domain: the side's ghost value and coefficient
    fE[f] = wall[j];
    fK[f] = wall[6 + j];
  } else {
    const double e0 = Ec_old[j];
    fE[f] = theta == 0.0 ? e0 : e0 + theta * (Ec_new[j] - e0);
    fK[f] = K_coarse[j];
  }
}

// Flux-limited diffusion coefficients and linearised coupling of one level
// (Sect. 2.1; the limiter and linearisation readings are stated with the
// entry point): for every leaf cell, from rho, T and E^n,
//   rho kappa_R = k0 rho^2 / T,  R = |grad E| / (rho kappa_R E),
//   lambda = (2 + R) / (6 + 3 R + R^2),  K = c lambda / (rho kappa_R),
//   sigma = dt kappa_P rho c (kappa_P = kappa_R),  mu = 4 a_R T^3 / (rho c_v),
//   s = sigma / (1 + sigma mu),  src = s a_R T^4;
// grad E by central differences over same-level cells, one-sided where a
// neighbour is missing.  Non-leaf cells keep K (restricted) and get s = src = 0.
__global__ void k_fld_coef(int64_t n_oct, const int32_t *__restrict__ nbr, const uint8_t *__restrict__ leaf,
                           const double *__restrict__ E, const double *__restrict__ rho,
                           const double *__restrict__ T, double dx, double dt, double k0, double *__restrict__ K,
                           double *__restrict__ s_out, double *__restrict__ src_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * n_oct) return;
  const int64_t o = i >> 3;
  const int c = (int)(i & 7);
  if (!((leaf[o] >> c) & 1)) {
    s_out[i] = 0.0;
    src_out[i] = 0.0;
    return;
  }
  const double e = E[i];
  double g2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int m = 1 << a;
    const int b = (c >> a) & 1;
    const double e_in = E[o * 8 + (c ^ m)];  // the other cell of the oct along a
    const int nb = nbr[o * 6 + 2 * a + b];    // the oct on this cell's outer side
    double g;
    if (nb >= 0 && idx_ok(nb, n_oct)) {
      const double e_out = E[(int64_t)nb * 8 + (c ^ m)];
      // b = 0: in-oct neighbour is at +a, outer at -a; b = 1: the reverse
      g = b == 0 ? (e_in - e_out) / (2.0 * dx) : (e_out - e_in) / (2.0 * dx);
    } else {
      g = b == 0 ? (e_in - e) / dx : (e - e_in) / dx;
    }
    g2 += g * g;
  }
  const double r = rho[i], t = T[i];
  const double kr = k0 * r * r / t;
  const double R = sqrt(g2) / (kr * e);
  const double lam = (2.0 + R) / (6.0 + 3.0 * R + R * R);
  K[i] = lam / kr;  // c = 1
  const double sigma = dt * kr;
  const double mu = 4.0 * t * t * t / r;  // a_R = c_v = 1
  const double sv = sigma / (1.0 + sigma * mu);
  s_out[i] = sv;
  src_out[i] = sv * t * t * t * t;
}

// Gas temperature after the radiation solve: T = T_n + sigma (E - a_R T_n^4) /
// (rho c_v (1 + sigma mu)) on leaf cells.
__global__ void k_fld_temperature(int64_t N, const uint8_t *__restrict__ leaf, const double *__restrict__ E,
                                  const double *__restrict__ rho, double *__restrict__ T, double dt, double k0) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || !((leaf[i >> 3] >> (i & 7)) & 1)) return;
  const double r = rho[i], t = T[i];
  const double kr = k0 * r * r / t;
  const double sigma = dt * kr;
  const double mu = 4.0 * t * t * t / r;
  T[i] = t + sigma * (E[i] - t * t * t * t) / (r * (1.0 + sigma * mu));
}

cudaError_t launch_fld_coef(int64_t n_oct, const int32_t *nbr, const uint8_t *leaf, const double *E, const double *rho,
                            const double *T, double dx, double dt, double k0, double *K, double *s, double *src,
                            cudaStream_t st) {
  const int64_t N = 8 * n_oct;
  k_fld_coef<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(n_oct, nbr, leaf, E, rho, T, dx, dt, k0, K, s, src);
  return cudaGetLastError();
}

cudaError_t launch_fld_temperature(int64_t N, const uint8_t *leaf, const double *E, const double *rho, double *T,
                                   double dt, double k0, cudaStream_t st) {
  k_fld_temperature<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, leaf, E, rho, T, dt, k0);
  return cudaGetLastError();
}

cudaError_t launch_restrict(int n, const int32_t *cell, const int32_t *child, const double *Ef, const double *Kf,
                            double *Ec, double *Kc, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_restrict<<<(n + 255) / 256, 256, 0, st>>>(n, cell, child, Ef, Kf, Ec, Kc);
  return cudaGetLastError();
}

cudaError_t launch_gather_faces(int n_face, const int8_t *src_rel, const int32_t *src_cell, const double *E_same,
                                const double *K_same, const double *Ec_old, const double *Ec_new,
                                const double *K_coarse, double theta, double *fE, double *fK, const double *wall,
                                cudaStream_t st) {
  if (n_face <= 0) return cudaSuccess;
  k_gather_faces<<<(n_face + 255) / 256, 256, 0, st>>>(n_face, src_rel, src_cell, E_same, K_same, Ec_old, Ec_new,
                                                        K_coarse, theta, fE, fK, wall);
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
    if (nbo >= 0 && idx_ok(nbo, sd.n_oct)) {
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

cudaError_t record_after(const TickTiming &tt, cudaEvent_t ev, cudaStream_t from, bool capture) {
  cudaError_t err;
  if ((err = cudaEventRecord(tt.mark, from)) != cudaSuccess) return err;
  if ((err = cudaStreamWaitEvent(tt.side, tt.mark, 0)) != cudaSuccess) return err;
  return capture ? cudaEventRecordWithFlags(ev, tt.side, cudaEventRecordExternal) : cudaEventRecord(ev, tt.side);
}

template <typename T, bool kPaper>
static cudaError_t tick_impl(const TickArgs &a, const int grids[3], cudaStream_t st, const TickStreams *fj,
                             const TickTiming *tt, bool capture) {
  cudaError_t err;
  const bool fork = fj && fj->aux;
  cudaStream_t sr = fork ? fj->aux : st;
  if (fork && (err = cudaEventRecord(fj->fork, st)) != cudaSuccess) return err;
  // k_ref first: its FP64-bound items start before k_op's CTAs take the SMs
  if (fork && (err = cudaStreamWaitEvent(sr, fj->fork, 0)) != cudaSuccess) return err;
  k_ref<T><<<grids[1], kThreads, 0, sr>>>(a);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (tt && (err = record_after(*tt, tt->ev[1], sr, capture)) != cudaSuccess) return err;
  k_op<T><<<grids[0], kThreads, 0, st>>>(a);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (tt && (err = record_after(*tt, tt->ev[0], st, capture)) != cudaSuccess) return err;
  if (fork) {
    if ((err = cudaEventRecord(fj->join, sr)) != cudaSuccess) return err;
    if ((err = cudaStreamWaitEvent(st, fj->join, 0)) != cudaSuccess) return err;
  }
  k_upd<T, kPaper><<<grids[2], kThreads, 0, st>>>(a);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (tt && (err = record_after(*tt, tt->ev[2], st, capture)) != cudaSuccess) return err;
  return cudaSuccess;
}

cudaError_t launch_tick(bool fp64, bool paper, const TickArgs &a, const int grids[3], cudaStream_t st,
                        const TickStreams *fj, const TickTiming *tt, bool capture) {
  if (fp64) return paper ? tick_impl<double, true>(a, grids, st, fj, tt, capture) : tick_impl<double, false>(a, grids, st, fj, tt, capture);
  return paper ? tick_impl<float, true>(a, grids, st, fj, tt, capture) : tick_impl<float, false>(a, grids, st, fj, tt, capture);
}

template <typename T, bool kPaper>
static void grids_impl(int sms, int grids[3]) {
  int b[3] = {0, 0, 0};
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[0], k_op<T>, kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[1], k_ref<T>, kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[2], k_upd<T, kPaper>, kThreads, 0);
  for (int k = 0; k < 3; ++k) grids[k] = (b[k] > 0 ? b[k] : 1) * sms;
}

void tick_grids(bool fp64, bool paper, int device, int grids[3]) {
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (sms <= 0) sms = 1;
  if (fp64) paper ? grids_impl<double, true>(sms, grids) : grids_impl<double, false>(sms, grids);
  else paper ? grids_impl<float, true>(sms, grids) : grids_impl<float, false>(sms, grids);
}

// ---------------------------------------------------------------------------
// admission of new solves between ticks (continuous batching)
// ---------------------------------------------------------------------------

__global__ void k_admit(TickArgs a, const int32_t *__restrict__ slots, int n_new) {
  __shared__ int base;
  const int s = slots[blockIdx.x];
  const SolveDev &sd = a.solves[s];
  const int cur = a.ctl->parity;
  if (threadIdx.x == 0) {
    base = atomicAdd(&a.ctl->count[cur][kRefine], sd.n_items);
    atomicAdd(a.n_active, 1);
  }
  __syncthreads();
  if (!idx_ok((long long)base + sd.n_items - 1, a.n_items)) return;
  int32_t *l = a.lists + (size_t)(cur * 2 + kRefine) * a.n_items;
  for (int k = threadIdx.x; k < sd.n_items; k += blockDim.x) l[base + k] = sd.item_begin + k;
}

cudaError_t launch_admit(const TickArgs &a, const int32_t *slots, int n_new, cudaStream_t st) {
  if (n_new <= 0) return cudaSuccess;
  k_admit<<<n_new, 128, 0, st>>>(a, slots, n_new);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// solve start / end over the work list
// ---------------------------------------------------------------------------

// Whether a caller's array can take the 32-byte oct vectors.
__device__ __forceinline__ bool oct_aligned(const void *p) { return ((uintptr_t)p & 31u) == 0; }

// Start of a solve on its work items, one oct per thread: e = 0, and x64 =
// src[solve] (Crank-Nicolson: the guess of E^{n+1} is turned into the guess
// of the half-step root (x + E^n) / 2) where src is given.  The caller's
// arrays take 32-byte vectors when aligned, else one cell per access.
template <typename T>
__global__ void k_init(const SolveDev *__restrict__ solves, const WorkItem *__restrict__ items,
                       int n_items, const double *const *__restrict__ src) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const WorkItem item = items[it];
    const SolveDev &sd = solves[item.solve];
    const double *xs = src ? src[item.solve] : nullptr;
    const bool vec = oct_aligned(xs) && oct_aligned(sd.cn_base);
    const int o_end = item.oct_begin + item_octs(item, sd);
    for (int o = item.oct_begin + (int)threadIdx.x; o < o_end; o += blockDim.x) {
      T z0[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) z0[c] = T(0);
      st8((T *)sd.e + 8 * (int64_t)o, z0);
      if (!xs) continue;
      double v[8];
      if (vec) {
        ld8_ro(xs + 8 * (int64_t)o, v);
        if (sd.cn_base) {
          double cb[8];
          ld8_ro(sd.cn_base + 8 * (int64_t)o, cb);
#pragma unroll
          for (int c = 0; c < 8; ++c) v[c] = 0.5 * (v[c] + cb[c]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int64_t k = 8 * (int64_t)o + c;
          v[c] = sd.cn_base ? 0.5 * (xs[k] + sd.cn_base[k]) : xs[k];
        }
      }
      st8(sd.x64 + 8 * (int64_t)o, v);
    }
  }
}

// End of a solve on its work items, one oct per thread: dst[solve] = x64
// (Crank-Nicolson: 2 x64 - E^n), and neg[solve] = 1 when a value is below
// zero (the warning of the solve).
__global__ void k_final(const SolveDev *__restrict__ solves, const WorkItem *__restrict__ items,
                        int n_items, double *const *__restrict__ dst, int *__restrict__ neg) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const WorkItem item = items[it];
    double *xd = dst[item.solve];
    if (!xd) continue;
    const SolveDev &sd = solves[item.solve];
    const bool vec = oct_aligned(xd) && oct_aligned(sd.cn_base);
    const int o_end = item.oct_begin + item_octs(item, sd);
    bool below = false;
    for (int o = item.oct_begin + (int)threadIdx.x; o < o_end; o += blockDim.x) {
      double v[8];
      ld8_rw(sd.x64 + 8 * (int64_t)o, v);
      if (sd.cn_base) {
        double cb[8];
        if (vec) {
          ld8_ro(sd.cn_base + 8 * (int64_t)o, cb);
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) cb[c] = sd.cn_base[8 * (int64_t)o + c];
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = 2.0 * v[c] - cb[c];
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) below = below || v[c] < 0.0;
      if (vec) {
        st8(xd + 8 * (int64_t)o, v);
      } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) xd[8 * (int64_t)o + c] = v[c];
      }
    }
    if (__syncthreads_or(below) && neg && threadIdx.x == 0) atomicOr(neg + item.solve, 1);
  }
}

cudaError_t launch_init(bool fp64, const SolveDev *solves, const WorkItem *items, int n_items,
                        const double *const *src, int grid, cudaStream_t st) {
  if (fp64) k_init<double><<<grid, kThreads, 0, st>>>(solves, items, n_items, src);
  else k_init<float><<<grid, kThreads, 0, st>>>(solves, items, n_items, src);
  return cudaGetLastError();
}

__global__ void k_cn_extrapolate(int64_t N, const double *__restrict__ x, const double *__restrict__ E,
                                 double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = 2.0 * x[i] - E[i];
}

cudaError_t launch_cn_extrapolate(int64_t N, const double *x, const double *E, double *out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  k_cn_extrapolate<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, x, E, out);
  return cudaGetLastError();
}

cudaError_t launch_final(const SolveDev *solves, const WorkItem *items, int n_items,
                         double *const *dst, int *neg, int grid, cudaStream_t st) {
  k_final<<<grid, kThreads, 0, st>>>(solves, items, n_items, dst, neg);
  return cudaGetLastError();
}

int tick_blocks_per_sm(bool fp64, bool paper) {
  int a = 0, b = 0;
  if (fp64) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_op<double>, kThreads, 0);
    if (paper) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_upd<double, true>, kThreads, 0);  // init / final grid
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_upd<double, false>, kThreads, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_op<float>, kThreads, 0);
    if (paper) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_upd<float, true>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_upd<float, false>, kThreads, 0);
  }
  const int m = a < b ? a : b;
  return m > 0 ? m : 1;
}

// ===========================================================================
// Resident solver: every iteration of a solve inside one launch
// ===========================================================================
//
// A solve runs from its first FP64 residual pass to its final certificate
// inside one persistent kernel.  A thread-block cluster takes a large solve:
// its CTAs split the level's octs into contiguous ranges, and the sums of
// each CG step (p.q; r.z and r.r; the residual norms) travel through
// distributed shared memory, ordered by barrier.cluster (a hardware barrier:
// no CTA spins on memory).  A CTA takes a small solve alone, ordered by
// __syncthreads.  A solve then pays no kernel launch per iteration, and
// solves of any mix of sizes and iteration counts keep the SMs busy until the
// work runs out, instead of advancing in lockstep ticks.
//
// The arithmetic of a solve depends only on its level and on the plan's
// resident shape (threads per CTA, CTAs per cluster, the size that selects a
// CTA or a cluster), never on which cluster or CTA takes it or on what runs
// beside it: sums merge in a fixed order (lanes by a shuffle tree, warps by
// index, CTAs by cluster rank) and every CTA of a cluster merges the CTAs'
// partials itself, so all hold bitwise the same totals and take the same
// decisions.  The CG scalars alpha and beta are formed in FP64 from the
// error-free (Dot2) totals and rounded to the bulk precision for the vector
// updates.
//
// Memory ordering: a vector written in one step and read by another CTA in a
// later one (z, p, D, x) is read with ld.global.cg after the step's cluster
// barrier (release / acquire at cluster scope); arrays no step writes (K, the
// neighbour table, face coefficients, b, diagonal extras) take the read-only
// path.

namespace {

constexpr int kMaxCluster = 16;
constexpr int kResMaxWarps = 512 / 32;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster arrives (release) and waits
// (acquire): the hardware cluster barrier (the non-.aligned form, which
// asks no warp convergence of its callers)
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// shared::cluster address of a variable of this CTA's shared memory in the
// CTA of cluster rank `rank`
__device__ __forceinline__ uint32_t cl_map(const void *p, unsigned rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_st(uint32_t a, const Acc<float> &v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.s), "f"(v.c) : "memory");
}
__device__ __forceinline__ void cl_st(uint32_t a, const Acc<double> &v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v.s) : "memory");
}

// lane 0's accumulator in every lane of the warp
__device__ __forceinline__ void bcast_acc(const Acc<float> &a, Acc<float> &t) {
  t.s = __shfl_sync(kFull, a.s, 0);
  t.c = __shfl_sync(kFull, a.c, 0);
}
__device__ __forceinline__ void bcast_acc(const Acc<double> &a, Acc<double> &t) { t.s = __shfl_sync(kFull, a.s, 0); }

// State of the solve a group (a CTA or a cluster) works on; thread 0 of each
// CTA updates its copy from the group's totals, so all copies agree.
struct ResState {
  int32_t phase, first, pcur, iters, inner_iters, refines, status, final_pass;
  int32_t n_op, n_first, n_xpe, pad;
  double rz, r0, rnorm, xnorm, inner_target, alpha, beta;
  float rzf, t2f, alphaf, betaf;  // the same scalars in FP32 (the FP32 bulk's step decisions)
};

template <typename T>
struct ResShared {
  SolveDev sd;
  ResState st;
  Acc<T> red[kResMaxWarps][3];
  __align__(16) Acc<T> inbox[2][kMaxCluster][3];  // [buffer][sender rank][sum]
  int task;
};

// alpha = r.z / p.q, or a breakdown (p.q not positive, a non-finite value).
template <typename T>
__device__ __forceinline__ void cg_alpha(ResState &st, const Acc<T> &pq_tot, bool f32) {
  if (f32) {
    const float pq = pq_tot.val(), rz = st.rzf;
    if (!(rz >= 0.f) || !isfinite(rz) || !(pq > 0.f) || !isfinite(pq)) {
      st.status = ATS_ERR_BREAKDOWN;
      st.phase = kDone;
    } else {
      st.alphaf = __fdiv_rn(rz, pq);
      st.alpha = st.alphaf;
    }
    return;
  }
  const double pq = pq_tot.get();
  if (!(st.rz >= 0.0) || !isfinite(st.rz) || !(pq > 0.0) || !isfinite(pq)) {
    st.status = ATS_ERR_BREAKDOWN;
    st.phase = kDone;
  } else {
    st.alpha = st.rz / pq;
    st.alphaf = (float)st.alpha;
  }
}
// beta = r'.z' / r.z for the next direction; returns whether the inner
// solve has converged (r'.r' <= target^2, or r'.z' = 0).
template <typename T>
__device__ __forceinline__ bool cg_beta(ResState &st, const Acc<T> &rz_tot, const Acc<T> &rr_tot, bool f32) {
  if (f32) {
    const float rz_new = rz_tot.val(), rr = rr_tot.val();
    st.betaf = __fdiv_rn(rz_new, st.rzf);
    st.beta = st.betaf;
    st.rzf = rz_new;
    st.rz = rz_new;
    return rr <= st.t2f || rz_new == 0.f;
  }
  const double rz_new = rz_tot.get(), rr = rr_tot.get();
  st.beta = rz_new / st.rz;
  st.betaf = (float)st.beta;
  st.rz = rz_new;
  st.rzf = (float)rz_new;
  return rr <= st.inner_target * st.inner_target || rz_new == 0.0;
}


// Sums of NA accumulators over the group: this CTA alone, or every CTA of the
// cluster.  Thread 0 of each CTA ends with the group totals in `out`.  The
// lanes of a warp, the warps of a CTA and the CTAs of a cluster are merged by
// fixed shuffle trees (error-free TwoSum pairs in the FP32 bulk): warp 0
// merges the warps' partials; in a cluster its lanes r < cluster size send
// the CTA's total to CTA r's inbox (buffer `buf`, slot of this CTA's rank),
// and after the cluster barrier warp 0 of every CTA merges its inbox, so all
// CTAs hold bitwise the same totals.  The inbox alternates between two
// buffers: a buffer is written again only two sums later, after a barrier
// that every reader of its previous contents has passed.
template <typename T, int NA, bool kCluster>
__device__ __forceinline__ void group_sum(Acc<T> (&a)[NA], ResShared<T> &sh, int &buf, Acc<T> (&out)[NA]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NA; ++k) warp_reduce_acc(a[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NA; ++k) sh.red[warp][k] = a[k];
  }
  __syncthreads();
  Acc<T> m[NA];
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      if (lane < nw) m[k] = sh.red[lane][k];
      warp_reduce_acc(m[k]);
    }
  }
  if (!kCluster) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NA; ++k) out[k] = m[k];
    }
    return;
  }
  const unsigned cs = cl_size(), cr = cl_rank();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      Acc<T> t;
      bcast_acc(m[k], t);
      if ((unsigned)lane < cs) cl_st(cl_map(&sh.inbox[buf][cr][k], (unsigned)lane), t);
    }
  }
  cl_sync();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      Acc<T> t;
      if ((unsigned)lane < cs) t = sh.inbox[buf][lane][k];
      warp_reduce_acc(t);
      if (lane == 0) out[k] = t;
    }
  }
  buf ^= 1;
}

template <bool kCluster>
__device__ __forceinline__ void group_barrier() {
  if (kCluster) cl_sync();
  else __syncthreads();
}

// x += e, e = 0 on one oct at the end of an inner solve (resident launch).
template <typename T>
__device__ __forceinline__ void res_xpe_oct(const SolveDev &sd, int o) {
  T *e = (T *)sd.e;
  T ev[8];
  double xv[8];
  ldc8(e + 8 * o, ev);
  ldc8(sd.x64 + 8 * o, xv);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    xv[c] += (double)ev[c];
    ev[c] = T(0);
  }
  st8(sd.x64 + 8 * o, xv);
  st8(e + 8 * o, ev);
}

// The per-step CG decisions of the FP32 bulk (alpha, beta, the inner test)
// are taken in FP32 from the error-free totals rounded once to FP32 -- the
// tick kernels' form -- unless cg_scalars asks for FP64: one thread takes
// them while the group waits, and the GB300's FP64 pipe makes an FP64
// quotient the longer wait.  A refinement pass's decisions are FP64.

// One solve by one group: the refinement / inner-CG state machine of the tick
// kernels (k_ref, k_op, k_upd), with its decisions taken right after each sum.
template <typename T, bool kCluster>
__device__ void res_solve(const ResArgs &a, int s, ResShared<T> &sh, int &buf) {
  constexpr int wd = (int)(sizeof(SolveDev) / 8);
  for (int w = threadIdx.x; w < wd; w += blockDim.x)
    reinterpret_cast<unsigned long long *>(&sh.sd)[w] = reinterpret_cast<const unsigned long long *>(a.solves + s)[w];
  const unsigned cs = kCluster ? cl_size() : 1u, cr = kCluster ? cl_rank() : 0u;
  if (threadIdx.x == 0) {
    ResState z;
    memset(&z, 0, sizeof(z));
    z.phase = kRefine;
    z.status = ATS_OK;
    sh.st = z;
    if (a.t_solve && cr == 0) a.t_solve[2 * s] = globaltimer_ns();
  }
  __syncthreads();
  const SolveDev &sd = sh.sd;
  const int n = sd.n_oct;
  const int chunk = (int)((n + (int)cs - 1) / (int)cs);
  const int lo = min(n, (int)cr * chunk), hi = min(n, lo + chunk);
  const int o0 = lo + (int)threadIdx.x, stride = (int)blockDim.x;
  const T h = (T)sd.h;
  const bool want_x = sd.stop_rule == ATS_STOP_CERTIFIED;
  const bool f32 = sizeof(T) == 4 && a.cg_scalars == 0;
  for (;;) {
    const int phase = sh.st.phase;
    if (phase == kDone) break;
    if (phase == kRefine) {
      // FP64 true residual of x, z = D^-1 r and D; sums r.r, x.x, r.z
      Acc<T> acc[3], tot[3];
      for (int o = o0; o < hi; o += stride) op_refine_oct<T, true>(sd, o, want_x, acc[0], acc[1], acc[2]);
      group_sum<T, 3, kCluster>(acc, sh, buf, tot);
      if (threadIdx.x == 0) {
        ResState &st = sh.st;
        const double rnorm = sqrt(tot[0].get()), xnorm = sqrt(tot[1].get()), rz = tot[2].get();
        if (st.refines == 0) st.r0 = rnorm;
        st.refines += 1;
        st.rnorm = rnorm;
        st.xnorm = xnorm;
        const double target = sd.tol * (sd.stop_rule == ATS_STOP_CERTIFIED ? xnorm : st.r0);
        if (st.final_pass) {
          st.phase = kDone;
        } else if (!isfinite(rnorm)) {
          st.status = ATS_ERR_BREAKDOWN;
          st.phase = kDone;
        } else if (rnorm <= target) {
          st.phase = kDone;
        } else if (st.refines > sd.max_refine) {
          st.status = ATS_ERR_NOT_CONVERGED;
          st.phase = kDone;
        } else if (!(rz > 0.0)) {
          st.status = ATS_ERR_BREAKDOWN;
          st.phase = kDone;
        } else {
          st.phase = kInner;
          st.rz = rz;
          st.rzf = (float)rz;
          st.first = 1;
          st.inner_iters = 0;
          st.inner_target = fmax(sd.inner_rtol * rnorm, sd.final_safety * target);
          st.t2f = (float)(st.inner_target * st.inner_target);
        }
      }
      __syncthreads();
      continue;
    }
    // inner CG iteration, step 1: p = z + beta p, q = (I + dt A) p, sum p.q
    const bool first = sh.st.first != 0;
    const T beta = sizeof(T) == 4 ? (T)sh.st.betaf : (T)sh.st.beta;
    const int pcur = sh.st.pcur;
    const T *pold = (const T *)(pcur ? sd.p1 : sd.p0);
    T *pnew = (T *)(pcur ? sd.p0 : sd.p1);
    {
      Acc<T> acc[1], tot[1];
      OpOwn<T> w;
      for (int o = o0; o < hi; o += stride) {
        op_load_own<T, true>(sd, o, first, pold, w);
        op_compute<T, true>(sd, o, w, h, beta, first, pold, pnew, acc[0]);
      }
      group_sum<T, 1, kCluster>(acc, sh, buf, tot);
      if (threadIdx.x == 0) {
        ResState &st = sh.st;
        st.n_op += 1;
        st.n_first += first ? 1 : 0;
        cg_alpha(st, tot[0], f32);
      }
      __syncthreads();
    }
    if (sh.st.phase == kDone) break;
    // step 2: e += alpha p, r = D z - alpha q, z = D^-1 r; sums r.z, r.r
    {
      const T alpha = sizeof(T) == 4 ? (T)sh.st.alphaf : (T)sh.st.alpha;
      Acc<T> acc[2], tot[2];
      UpdOwn<T> w;
      float none = 0.f;
      for (int o = o0; o < hi; o += stride) {
        upd_load_own<T, true>(sd, o, pnew, w);
        upd_compute<T, false>(sd, o, w, alpha, acc[0], acc[1], none);
      }
      group_sum<T, 2, kCluster>(acc, sh, buf, tot);
      if (threadIdx.x == 0) {
        ResState &st = sh.st;
        st.iters += 1;
        st.inner_iters += 1;
        st.first = 0;
        st.pcur ^= 1;
        const bool conv = cg_beta(st, tot[0], tot[1], f32);
        if (conv) {
          st.phase = kRefine;
        } else if (st.iters >= sd.max_iter) {
          st.status = ATS_ERR_NOT_CONVERGED;
          st.final_pass = 1;
          st.phase = kRefine;
        } else if (st.inner_iters >= sd.inner_max) {
          st.phase = kRefine;  // restart from the true residual
        }
        if (st.phase == kRefine) st.n_xpe += 1;
      }
      __syncthreads();
    }
    if (sh.st.phase == kRefine) {
      // the inner solve ends: x += e, e = 0; the next residual pass reads the
      // neighbours' x, so the whole group passes a barrier first
      for (int o = o0; o < hi; o += stride) res_xpe_oct<T>(sd, o);
      group_barrier<kCluster>();
    }
  }
  if (threadIdx.x == 0 && cr == 0) {
    const ResState &st = sh.st;
    SolveScalars f;
    memset(&f, 0, sizeof(f));
    f.phase = kDone;
    f.iters = st.iters;
    f.inner_iters = st.inner_iters;
    f.refines = st.refines;
    f.status = st.status;
    f.final_pass = st.final_pass;
    f.ticks = st.n_op + st.iters + st.refines;  // group steps taken
    f.rz = st.rz;
    f.r0 = st.r0;
    f.inner_target = st.inner_target;
    f.rnorm = st.rnorm;
    f.xnorm = st.xnorm;
    a.final_sc[s] = f;
    if (a.t_solve) a.t_solve[2 * s + 1] = globaltimer_ns();
    if (a.cells) {
      const unsigned long long N = 8ull * (unsigned long long)n;
      atomicAdd(a.cells + 0, N * (unsigned long long)(st.n_op - st.n_first));
      atomicAdd(a.cells + 4, N * (unsigned long long)st.n_first);
      atomicAdd(a.cells + 1, N * (unsigned long long)st.refines);
      atomicAdd(a.cells + 2, N * (unsigned long long)st.iters);
      atomicAdd(a.cells + 3, N * (unsigned long long)st.n_xpe);
    }
  }
}

// Small solves, one CTA each, taken from the CTA queue until it is empty.
template <typename T>
__device__ void res_cta_loop(const ResArgs &a, ResShared<T> &sh, int &buf) {
  for (;;) {
    __syncthreads();  // every thread has read the previous task
    if (threadIdx.x == 0) sh.task = atomicAdd(a.tq_head, 1);
    __syncthreads();
    const int t = sh.task;
    if (t >= a.n_tq) break;
    int s = a.tq[t];
    if (!idx_ok(s, a.n_solves)) continue;
    res_solve<T, false>(a, s, sh, buf);
  }
}

template <typename T, int NT>
struct ResMinBlocks {
  static constexpr int value = (sizeof(T) == 4 && NT <= 256) ? 2 : 1;
};

}  // namespace

// The cluster kernel: each cluster takes the large solves of the cluster
// queue one after the other (rank 0 draws the next position and writes it
// into every CTA's shared memory before a cluster barrier); once that queue
// is empty its CTAs take small solves from the CTA queue independently (no
// cluster barrier or distributed shared memory access follows).
template <typename T, int NT>
__global__ void __launch_bounds__(NT, ResMinBlocks<T, NT>::value) k_res_cluster(ResArgs a) {
  __shared__ ResShared<T> sh;
  int buf = 0;
  const unsigned cr = cl_rank(), cs = cl_size();
  for (;;) {
    if (cr == 0 && threadIdx.x == 0) {
      const int t = atomicAdd(a.cq_head, 1);
      for (unsigned r = 0; r < cs; ++r) cl_st(cl_map(&sh.task, r), t);
    }
    cl_sync();
    const int t = sh.task;
    if (t >= a.n_cq) break;
    const int s = a.cq[t];
    if (idx_ok(s, a.n_solves)) res_solve<T, true>(a, s, sh, buf);
  }
  res_cta_loop<T>(a, sh, buf);
}

// The CTA kernel: small solves only (a plan without cluster solves).
template <typename T, int NT>
__global__ void __launch_bounds__(NT, ResMinBlocks<T, NT>::value) k_res_cta(ResArgs a) {
  __shared__ ResShared<T> sh;
  int buf = 0;
  res_cta_loop<T>(a, sh, buf);
}

// ---------------------------------------------------------------------------
// Resident solver with the CG state in shared memory (FP32 bulk)
// ---------------------------------------------------------------------------
//
// Each CTA of the group owns a contiguous run of the level's octs (the
// group's octs split by cluster rank) and keeps K, z and p of the first
// kRes2Cap3 of them in shared memory for the whole solve, each array as eight
// planes (plane c holds cell c of every oct: a warp's accesses to one cell of
// consecutive octs are conflict-free, and a face reads exactly its four
// cells), with each oct's six neighbours coded as (owning rank, local index).  A step reads its own octs
// from its shared memory and the neighbours' faces from the owning CTA's
// shared memory (distributed shared memory inside the cluster): no iteration
// reads K, z or p from L2 or HBM.  D, q and e -- read and written only by the
// thread that owns an oct -- are kept there too when the CTA's share is at
// most kRes2Cap6 octs, so a CG iteration then touches no global memory (else
// they stay in global memory); the FP64 arrays of the refinement pass stay in
// global memory.  Octs beyond a CTA's capacity use the level's global arrays.  Where an oct's values live does not change what is computed, so
// the capacity does not enter the arithmetic.
//
// A CG iteration takes one of two forms (cg_form), equal in exact
// arithmetic.  From p, three group synchronisations:
//   1. p = z + beta p on the own octs (an inner solve's first: p = z), then
//      a group barrier;
//   2. q = (I + dt A) p from the own and the neighbours' p, the sum p.q;
//   3. r = D z - alpha q, z = D^-1 r, e += alpha p, the sums r.z and r.r.
// By the q recurrence, two: since p = z + beta p_prev,
// (I + dt A) p = (I + dt A) z + beta q_prev, and z -- the only array a step
// reads from the neighbours -- is final once step 3's sum has passed:
//   1+2. w = (I + dt A) z, p = z + beta p, q = w + beta q (first: p = z,
//        q = w) in one pass, the sum p.q;
//   3.   as above.

extern __shared__ __align__(128) unsigned char res2_smem[];
// Two layouts of a CTA's shared memory, chosen per solve from the size of the
// CTA's share: all six arrays K, z, p, D, q, e for up to kRes2Cap6 octs, or
// K, z, p only (D, q, e in global memory) for up to kRes2Cap3 octs.  Each
// array is four pair planes (cells 2k, 2k+1 of each oct side by side) of
// cap + 1 octs (oct `cap`: the stand-in neighbour), followed by the 16-byte
// neighbour codes of the octs.
constexpr int kRes2Cap3 = 2048;
constexpr int kRes2Cap6 = 1100;
constexpr size_t kRes2SmemBytes = (size_t)24 * (kRes2Cap3 + 1) * 4 + (size_t)kRes2Cap3 * 16;
static_assert((size_t)48 * (kRes2Cap6 + 1) * 4 + (size_t)kRes2Cap6 * 16 <= kRes2SmemBytes,
              "the six-array layout fits the three-array one's allocation");

namespace {

constexpr uint16_t kCodeNone = 0xFFFF;      // no neighbour (a wall or interface face)
constexpr uint16_t kCodeGlobal = 0xFFFE;    // a neighbour beyond its CTA's capacity: global arrays

// The layout constants of a solve (capacities, plane stride) as compile-time
// members, so every shared access is a register plus an immediate offset.
template <int kCap, int kCapD>
struct Res2Ctx {
  static constexpr int cap = kCap;    // octs of the CTA's share whose K, z, p are in shared memory
  static constexpr int capD = kCapD;  // ... whose D, q, e are (kCap or 0)
  static constexpr uint32_t S = (uint32_t)(kCap + 1) * 8u;  // bytes of one pair plane
  uint32_t sK, sZ, sP, sD, sQ, sE, sC;  // shared-window addresses of this CTA's planes and codes
  int chunk;                // octs per CTA of the group
  int lo;                   // first oct of this CTA
  unsigned cr;              // this CTA's rank in the group (0 for one CTA)
  unsigned crc;             // the rank neighbour codes give this CTA's octs (cr in a cluster, else 0)
  bool grid;                // a whole-GPU group: octs of other CTAs are read from global memory
  bool qrec;                // q by the recurrence: neighbours read z (published globally in a whole-GPU group)
};
using Res2Six = Res2Ctx<kRes2Cap6, kRes2Cap6>;
using Res2Three = Res2Ctx<kRes2Cap3, 0>;
using Res2Global = Res2Ctx<0, 0>;  // every array in global memory (the stand-in row only in shared)

// The eight cells of an oct from the pair planes of an array: pair plane k
// holds cells 2k and 2k+1 of every oct (8 bytes per oct, S bytes per plane),
// a = the array's address + 8 x the oct's local index (this CTA's shared
// memory, or, with the _c forms, another CTA's through its shared::cluster
// address).  Two cells per access halve the shared-memory instructions of the
// own rows and of the y and z faces.
__device__ __forceinline__ float ldsf(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float ldscf(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
template <bool kRemote>
__device__ __forceinline__ void lds2(uint32_t a, float &x, float &y) {
  if (kRemote) asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a));
  else asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a));
}
__device__ __forceinline__ void lds_cells(uint32_t a, uint32_t S, float (&v)[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) lds2<false>(a + k * S, v[2 * k], v[2 * k + 1]);
}
__device__ __forceinline__ void sts_cells(uint32_t a, uint32_t S, const float (&v)[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a + k * S), "f"(v[2 * k]), "f"(v[2 * k + 1]) : "memory");
}
// The four cells facing across axis A (those with bit A equal to NB): one
// cell of each pair across x, two whole pairs across y or z.
template <int A, int NB, bool kRemote>
__device__ __forceinline__ void lds_face(uint32_t a, uint32_t S, float (&v)[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (A == 0) {
      const uint32_t ak = a + k * S + 4u * NB;
      v[2 * k + NB] = kRemote ? ldscf(ak) : ldsf(ak);
    } else {
      if ((((2 * k) >> A) & 1) != NB) continue;
      lds2<kRemote>(a + k * S, v[2 * k], v[2 * k + 1]);
    }
  }
}

__device__ __forceinline__ uint32_t cl_map_s(uint32_t a, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

// Where a neighbour oct's rows are: kind 0 none, 1 this CTA's shared memory,
// 2 another CTA's (rank r), 3 the global arrays (oct g).
struct Nb {
  int kind;
  uint32_t off;  // byte offset of the oct in each plane of a shared array
  unsigned r;
  int g;
};
template <class Cx>
__device__ __forceinline__ Nb nb_of_global(const Cx &cx, int g) {
  Nb n;
  n.g = g;
  n.r = 0;
  n.off = 0;
  if (g < 0) {
    n.kind = 0;
    return n;
  }
  const int r = g / cx.chunk, l = g - r * cx.chunk;
  if (l >= cx.cap) {
    n.kind = 3;
    return n;
  }
  n.r = (unsigned)r;
  n.off = (uint32_t)l * 8u;
  n.kind = n.r == cx.cr ? 1 : (cx.grid ? 3 : 2);
  return n;
}
template <class Cx>
__device__ __forceinline__ uint16_t code_of_global(const Cx &cx, int g) {
  if (g < 0) return kCodeNone;
  const int r = g / cx.chunk, l = g - r * cx.chunk;
  if (l >= cx.cap || (cx.grid && (unsigned)r != cx.cr)) return kCodeGlobal;
  return (uint16_t)(((cx.grid ? 0u : (unsigned)r) << 12) | (unsigned)l);
}

// The six neighbours of own oct o (local index l).
template <class Cx>
__device__ __forceinline__ void res2_nbs(const Cx &cx, const SolveDev &sd, int o, int l, Nb (&nb)[6]) {
  if (l < cx.cap) {
    uint32_t c01, c23, c45, pad;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(c01), "=r"(c23), "=r"(c45), "=r"(pad)
                 : "r"(cx.sC + (uint32_t)l * 16u));
    const uint32_t w[3] = {c01, c23, c45};
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const uint16_t c = (uint16_t)(w[d >> 1] >> (16 * (d & 1)));
      Nb &n = nb[d];
      n.g = -1;
      n.r = 0;
      n.off = 0;
      if (c == kCodeNone) {
        n.kind = 0;
      } else if (c == kCodeGlobal) {
        int g = __ldg(sd.nbr + 6 * o + d);
        if (g >= 0 && !idx_ok(g, sd.n_oct)) g = -1;
        n = nb_of_global(cx, g);
      } else {
        n.r = c >> 12;
        n.off = (uint32_t)(c & 0xFFF) * 8u;
        n.kind = n.r == cx.crc ? 1 : 2;
      }
    }
  } else {
    int g[6];
    load_nbr6(sd.nbr, o, g);
    check_nbr6(g, sd.n_oct);
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = nb_of_global(cx, g[d]);
  }
}

// The four cells of neighbour n that face this oct across axis A (NB: which
// half), from the shared array at `arr` or the global array `garr`.
template <int A, int NB>
__device__ __forceinline__ void res2_face(const Nb &n, uint32_t arr, uint32_t S, const float *garr, bool coherent,
                                          float (&v)[8]) {
  if (n.kind == 1) {
    lds_face<A, NB, false>(arr + n.off, S, v);
  } else if (n.kind == 2) {
    lds_face<A, NB, true>(cl_map_s(arr + n.off, n.r), S, v);
  } else {
    if (coherent) ldc_face<A, NB>(garr + 8 * n.g, v);
    else ld_face<A, NB>(garr + 8 * n.g, v);
  }
}

// An own oct's row of a shared array, or of its global array beyond the capacity.
template <class Cx>
__device__ __forceinline__ void res2_own(const Cx &cx, uint32_t arr, int cap, int l, const float *garr, int o,
                                         bool coherent, float (&v)[8]) {
  if (l < cap) lds_cells(arr + (uint32_t)l * 8u, cx.S, v);
  else if (coherent) ldc8(garr + 8 * o, v);
  else ld8_ro(garr + 8 * o, v);
}
template <class Cx>
__device__ __forceinline__ void res2_own_store(const Cx &cx, uint32_t arr, int cap, int l, float *garr, int o,
                                               const float (&v)[8]) {
  if (l < cap) sts_cells(arr + (uint32_t)l * 8u, cx.S, v);
  else st8(garr + 8 * o, v);
}

// The resident solver keeps K scaled by h = dt / (2 dx^2) (rounded once per
// cell; the sign, which marks leaf cells, is kept), so a face's coupling is
// C = hK_i + hK_j.  Values read from the level's global K are scaled the same
// way where they are used, so where a value lives does not change the bits.
__device__ __forceinline__ void res2_scale_K(float h, float (&K)[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) K[c] *= h;
}

// The in-oct faces of the resident solver's stencil (K scaled by h).  Unlike
// in_oct_faces it takes no leaf test: every array the stencil reads (p, z)
// is zero on non-leaf cells and in the stand-in row, so a coupling to such a
// cell adds C x 0 (C finite); a non-leaf cell's own row is zeroed afterwards.
__device__ __forceinline__ void res2_in_oct(const float (&K)[8], const float (&v)[8], float (&off)[8]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c & (1 << a)) continue;
      const int d = c | (1 << a);
      const float C = K[c] + K[d];
      off[c] = fmaf(C, v[d], off[c]);
      off[d] = fmaf(C, v[c], off[d]);
    }
  }
}

template <int DIR, bool kRec, class Cx>
__device__ __forceinline__ void res2_op_face(const Cx &cx, const SolveDev &sd, const Nb &n, float h,
                                             const float (&K)[8], float (&off)[8]) {
  constexpr int A = DIR >> 1, S = DIR & 1, NB = 1 - S;
  if (n.kind == 0) return;
  float Kn[8], Pn[8];
  res2_face<A, NB>(n, cx.sK, cx.S, (const float *)sd.KT, false, Kn);
  if (n.kind == 3) res2_scale_K(h, Kn);
  res2_face<A, NB>(n, kRec ? cx.sZ : cx.sP, cx.S, (const float *)(kRec ? sd.z : sd.p0), true, Pn);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (((c >> A) & 1) != S) continue;
    const int j = c ^ (1 << A);
    off[c] = fmaf(K[c] + Kn[j], Pn[j], off[c]);  // Pn is zero on non-leaf cells (see res2_in_oct)
  }
}

// The end of step 2 on own oct o, from the stencil's off-diagonal part off
// of v (the value array the stencil read) and the diagonal d.  q = D p - off
// when v = p.  With the q recurrence v = z: w = D z - off, then
// p = z + beta p_prev and q = w + beta q_prev (an inner solve's first step:
// p = z, q = w).  q is zero on non-leaf cells; stores q (and p), returns p.q
// over the leaf cells.
template <bool kRec, class Cx>
__device__ __forceinline__ float res2_op_end(const Cx &cx, const SolveDev &sd, int o, int l, const float (&K)[8],
                                             const float (&v)[8], const float (&d)[8], const float (&off)[8],
                                             bool first, float beta) {
  float local = 0.f, qv[8];
  if (!kRec) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float q = d[c] * v[c] - off[c];
      const bool leaf = K[c] >= 0.f;
      if (leaf) local = fmaf(v[c], q, local);
      qv[c] = leaf ? q : 0.f;
    }
    res2_own_store(cx, cx.sQ, cx.capD, l, (float *)sd.q, o, qv);
    return local;
  }
  float pp[8], pv[8];
  if (first) {
#pragma unroll
    for (int c = 0; c < 8; ++c) pp[c] = qv[c] = 0.f;
  } else {
    res2_own(cx, cx.sP, cx.cap, l, (const float *)sd.p0, o, true, pp);
    res2_own(cx, cx.sQ, cx.capD, l, (const float *)sd.q, o, true, qv);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float w = d[c] * v[c] - off[c];
    const float pn = first ? v[c] : fmaf(beta, pp[c], v[c]);
    const float qn = first ? w : fmaf(beta, qv[c], w);
    const bool leaf = K[c] >= 0.f;
    if (leaf) local = fmaf(pn, qn, local);
    qv[c] = leaf ? qn : 0.f;
    pv[c] = pn;
  }
  res2_own_store(cx, cx.sP, cx.cap, l, (float *)sd.p0, o, pv);
  res2_own_store(cx, cx.sQ, cx.capD, l, (float *)sd.q, o, qv);
  return local;
}

// Step 2 on own oct o: the stencil of v (p, or z with the q recurrence) from
// the own and the neighbours' rows, then res2_op_end; returns the oct's p.q.
template <bool kRec, class Cx>
__device__ __forceinline__ float res2_op_oct(const Cx &cx, const SolveDev &sd, int o, float h, bool first,
                                             float beta) {
  const int l = o - cx.lo;
  float K[8], v[8], d[8];
  res2_own(cx, cx.sK, cx.cap, l, (const float *)sd.KT, o, false, K);
  if (l >= cx.cap) res2_scale_K(h, K);
  res2_own(cx, kRec ? cx.sZ : cx.sP, cx.cap, l, (const float *)(kRec ? sd.z : sd.p0), o, true, v);
  res2_own(cx, cx.sD, cx.capD, l, (const float *)sd.dg, o, true, d);
  Nb nb[6];
  res2_nbs(cx, sd, o, l, nb);
  float off[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) off[c] = 0.f;
  res2_in_oct(K, v, off);
  res2_op_face<0, kRec>(cx, sd, nb[0], h, K, off);
  res2_op_face<1, kRec>(cx, sd, nb[1], h, K, off);
  res2_op_face<2, kRec>(cx, sd, nb[2], h, K, off);
  res2_op_face<3, kRec>(cx, sd, nb[3], h, K, off);
  res2_op_face<4, kRec>(cx, sd, nb[4], h, K, off);
  res2_op_face<5, kRec>(cx, sd, nb[5], h, K, off);
  return res2_op_end<kRec>(cx, sd, o, l, K, v, d, off, first, beta);
}

// Step 2 on own oct o of the shared rows whose six neighbours are all in
// shared memory (or the stand-in row): every face loads unconditionally, from
// this CTA's rows (one CTA) or the owner's (a cluster).
template <int DIR, bool kCluster>
__device__ __forceinline__ void res2_fast_face(uint32_t aK, uint32_t aP, uint32_t PS, float h, const float (&K)[8],
                                               float (&off)[8]) {
  constexpr int A = DIR >> 1, S = DIR & 1, NB = 1 - S;
  float Kn[8], Pn[8];
  lds_face<A, NB, kCluster>(aK, PS, Kn);
  lds_face<A, NB, kCluster>(aP, PS, Pn);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (((c >> A) & 1) != S) continue;
    const int j = c ^ (1 << A);
    off[c] = fmaf(K[c] + Kn[j], Pn[j], off[c]);  // Pn is zero on non-leaf cells (see res2_in_oct)
  }
}

template <bool kCluster, bool kRec, class Cx>
__device__ __forceinline__ float res2_op_oct_fast(const Cx &cx, const SolveDev &sd, int o, int l,
                                                  const uint32_t (&w)[3], float h, bool first, float beta) {
  const uint32_t sV = kRec ? cx.sZ : cx.sP;
  float K[8], v[8], d[8];
  lds_cells(cx.sK + (uint32_t)l * 8u, cx.S, K);
  lds_cells(sV + (uint32_t)l * 8u, cx.S, v);
  res2_own(cx, cx.sD, cx.capD, l, (const float *)sd.dg, o, true, d);
  uint32_t aK[6], aV[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const uint32_t c = (w[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
    const uint32_t off = (c & 0xFFFu) * 8u;
    if (kCluster) {
      aK[k] = cl_map_s(cx.sK + off, c >> 12);
      aV[k] = cl_map_s(sV + off, c >> 12);
    } else {
      aK[k] = cx.sK + off;
      aV[k] = sV + off;
    }
  }
  float off[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) off[c] = 0.f;
  res2_in_oct(K, v, off);
  res2_fast_face<0, kCluster>(aK[0], aV[0], cx.S, h, K, off);
  res2_fast_face<1, kCluster>(aK[1], aV[1], cx.S, h, K, off);
  res2_fast_face<2, kCluster>(aK[2], aV[2], cx.S, h, K, off);
  res2_fast_face<3, kCluster>(aK[3], aV[3], cx.S, h, K, off);
  res2_fast_face<4, kCluster>(aK[4], aV[4], cx.S, h, K, off);
  res2_fast_face<5, kCluster>(aK[5], aV[5], cx.S, h, K, off);
  return res2_op_end<kRec>(cx, sd, o, l, K, v, d, off, first, beta);
}

// Step 2 on own oct o: the branch-free form when its row and every
// neighbour's are in shared memory, else the general one.
template <bool kCluster, bool kRec, class Cx>
__device__ __forceinline__ float res2_op_any(const Cx &cx, const SolveDev &sd, int o, float h, bool first,
                                             float beta) {
  const int l = o - cx.lo;
  if (l < cx.cap) {
    uint32_t w0, w1, w2, pad;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(pad)
                 : "r"(cx.sC + (uint32_t)l * 16u));
    const uint32_t gl = 0xFFFEu;
    const bool any_global = ((w0 & 0xFFFFu) == gl) | ((w0 >> 16) == gl) | ((w1 & 0xFFFFu) == gl) |
                            ((w1 >> 16) == gl) | ((w2 & 0xFFFFu) == gl) | ((w2 >> 16) == gl);
    if (!any_global) {
      const uint32_t w[3] = {w0, w1, w2};
      return res2_op_oct_fast<kCluster, kRec>(cx, sd, o, l, w, h, first, beta);
    }
  }
  return res2_op_oct<kRec>(cx, sd, o, h, first, beta);
}

// Step 1 on own oct o: p = z + beta p (first: p = z).
// In a whole-GPU group the new p also goes to the global array, where the
// other CTAs read the faces they need.
template <class Cx>
__device__ __forceinline__ void res2_dir_oct(const Cx &cx, const SolveDev &sd, int o, bool first, float beta) {
  const int l = o - cx.lo;
  float z[8], p[8];
  res2_own(cx, cx.sZ, cx.cap, l, (const float *)sd.z, o, true, z);
  if (!first) res2_own(cx, cx.sP, cx.cap, l, (const float *)sd.p0, o, true, p);
#pragma unroll
  for (int c = 0; c < 8; ++c) p[c] = first ? z[c] : fmaf(beta, p[c], z[c]);
  res2_own_store(cx, cx.sP, cx.cap, l, (float *)sd.p0, o, p);
  if (cx.grid && l < cx.cap) st8((float *)sd.p0 + 8 * o, p);
}

// Step 3 on own oct o: r = D z - alpha q, z = r x rcp(D), e += alpha p.
template <class Cx>
__device__ __forceinline__ void res2_upd_oct(const Cx &cx, const SolveDev &sd, int o, float alpha, float &lrz,
                                             float &lrr) {
  const int l = o - cx.lo;
  float p[8], z[8], d[8], q[8], e[8];
  res2_own(cx, cx.sP, cx.cap, l, (const float *)sd.p0, o, true, p);
  res2_own(cx, cx.sZ, cx.cap, l, (const float *)sd.z, o, true, z);
  res2_own(cx, cx.sD, cx.capD, l, (const float *)sd.dg, o, true, d);
  res2_own(cx, cx.sQ, cx.capD, l, (const float *)sd.q, o, true, q);
  res2_own(cx, cx.sE, cx.capD, l, (const float *)sd.e, o, true, e);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float r = d[c] * z[c] - alpha * q[c];
    const float zn = r * rcp_approx(d[c]);
    lrz = fmaf(r, zn, lrz);
    lrr = fmaf(r, r, lrr);
    z[c] = zn;
    e[c] += alpha * p[c];
  }
  res2_own_store(cx, cx.sZ, cx.cap, l, (float *)sd.z, o, z);
  if (cx.qrec && cx.grid && l < cx.cap) st8((float *)sd.z + 8 * o, z);
  res2_own_store(cx, cx.sE, cx.capD, l, (float *)sd.e, o, e);
}

// The FP64 residual pass on own oct o (global arrays; the neighbours' x read
// coherently), z into its shared row, D into global memory.
template <class Cx>
__device__ __forceinline__ void res2_ref_oct(const Cx &cx, const SolveDev &sd, int o, bool want_x, Acc<float> &rr,
                                             Acc<float> &xx, Acc<float> &rz) {
  float zo[8], dv[8];
  ref_oct_values<float, true, true>(sd, o, want_x, rr, xx, rz, zo, dv);
  res2_own_store(cx, cx.sZ, cx.cap, o - cx.lo, (float *)sd.z, o, zo);
  if (cx.qrec && cx.grid && o - cx.lo < cx.cap) st8((float *)sd.z + 8 * o, zo);
  res2_own_store(cx, cx.sD, cx.capD, o - cx.lo, (float *)sd.dg, o, dv);
}

// x += e, e = 0 on own oct o at the end of an inner solve (e in its shared
// planes, or global beyond the capacity).
template <class Cx>
__device__ __forceinline__ void res2_xpe_oct(const Cx &cx, const SolveDev &sd, int o) {
  const int l = o - cx.lo;
  if (l >= cx.capD) {
    res_xpe_oct<float>(sd, o);
    return;
  }
  float e[8], z0[8];
  double xv[8];
  lds_cells(cx.sE + (uint32_t)l * 8u, cx.S, e);
  ldc8(sd.x64 + 8 * o, xv);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    xv[c] += (double)e[c];
    z0[c] = 0.f;
  }
  st8(sd.x64 + 8 * o, xv);
  sts_cells(cx.sE + (uint32_t)l * 8u, cx.S, z0);
}

// ---- whole-GPU group: grid barrier and sums through global memory -------
// Polls of the barrier's arrival counter before a wait gives up: with the
// back-off (at most 128 ns of sleep between polls) a wait ends within about
// half a second whatever happens to the other CTAs; a barrier of a running
// solve takes microseconds.
constexpr long long kGridSpinLimit = 1ll << 21;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// The grid barrier, run by warp 0 of each CTA after a CTA barrier (so that
// lane 0's release covers the whole CTA's writes).  Arrivals go to one
// counter (gbar[0], zero at the launch) that only grows: no CTA arrives at
// barrier k + 1 before barrier k is complete, so the counter's value before
// an arrival, `old`, lies in [k E, (k + 1) E) (E = arrivals per barrier) and
// barrier k is complete once the counter reaches (k + 1) E.  Lane 0 arrives
// with an acquire-release add; the last arrival knows it is complete (its
// other lanes read after lane 0's acquire and a warp barrier), the others
// poll the counter with every lane's acquire loads and a short back-off.
// Returns false, in every lane, when the wait gave up (then *gerr = 1).
__device__ bool grid_arrive_wait(const ResArgs &a) {
  const unsigned expect = a.g_expect > 0 ? (unsigned)a.g_expect : gridDim.x;
  const int lane = threadIdx.x & 31;
  unsigned old = 0;
  if (lane == 0) old = atom_add_acq_rel_u32(a.gbar, 1u);
  old = __shfl_sync(kFull, old, 0);
  __syncwarp();
  const unsigned target = (old / expect + 1u) * expect;
  if (old + 1u == target) return true;
  unsigned ns = 16;
  for (long long it = 0;; ++it) {
    const unsigned v = ld_acquire_u32(a.gbar);
    if (__all_sync(kFull, (int)(v - target) >= 0)) return true;
    if (it >= kGridSpinLimit) {
      if (lane == 0) atomicOr(a.gerr, 1);
      return false;
    }
    __nanosleep(ns);
    if (ns < 128) ns <<= 1;
  }
}

// Every CTA of the cooperative launch waits here until all have arrived; the
// CTA's global writes before it are visible to every CTA after it.  Returns
// false in every thread of a CTA whose wait gave up.
__device__ bool grid_sync(const ResArgs &a, int *flag) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = grid_arrive_wait(a);
    if (threadIdx.x == 0) *flag = ok ? 1 : 0;
  }
  __syncthreads();
  return *flag != 0;
}

// Sums of NA accumulators over every CTA of the launch.  Each CTA's total
// (the same shuffle trees as a cluster's) goes to its slot of gpart (buffer
// `buf`) before the CTA arrives at the grid barrier; once the barrier is
// complete, warp 0 of every CTA merges all slots in rank order -- lane j
// takes ranks j, j + 32, ..., every load issued before the merges -- with a
// shuffle tree, so all CTAs hold bitwise the same totals.  Thread 0 ends
// with them in `out`; the return value (thread 0) is false when its wait gave
// up.  The slots alternate between two buffers: a buffer is written again
// only two sums later, after a barrier that every reader has passed.
constexpr int kGridMaxPerLane = 8;  // up to 256 CTAs in the launch
template <int NA>
__device__ bool grid_sum(Acc<float> (&a)[NA], ResShared<float> &sh, const ResArgs &ra, int &buf,
                         Acc<float> (&out)[NA]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NA; ++k) warp_reduce_acc(a[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NA; ++k) sh.red[warp][k] = a[k];
  }
  __syncthreads();
  bool ok = true;
  if (warp == 0) {
    Acc<float> m[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      if (lane < nw) m[k] = sh.red[lane][k];
      warp_reduce_acc(m[k]);
    }
    const unsigned G = gridDim.x;
    float *slots = ra.gpart + (size_t)buf * (G + 1) * 6;  // [G] CTA slots of 3 (hi, lo) pairs
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        slots[blockIdx.x * 6 + 2 * k] = m[k].s;
        slots[blockIdx.x * 6 + 2 * k + 1] = m[k].c;
      }
    }
    ok = grid_arrive_wait(ra);
    if (ok) {
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        float vs[kGridMaxPerLane], vc[kGridMaxPerLane];
#pragma unroll
        for (int i = 0; i < kGridMaxPerLane; ++i) {
          const unsigned r = (unsigned)lane + 32u * i;
          vs[i] = r < G ? __ldcg(slots + r * 6 + 2 * k) : 0.f;
          vc[i] = r < G ? __ldcg(slots + r * 6 + 2 * k + 1) : 0.f;
        }
        Acc<float> t;
#pragma unroll
        for (int i = 0; i < kGridMaxPerLane; ++i) {
          Acc<float> v;
          v.s = vs[i];
          v.c = vc[i];
          t.merge(v);
        }
        warp_reduce_acc(t);
        if (lane == 0) out[k] = t;
      }
    }
  }
  buf ^= 1;
  return ok;
}

// The group's sum and barrier for group kind kG (0 one CTA, 1 a cluster, 2
// the whole GPU); only the whole-GPU forms can fail: the sum reports it to
// thread 0 (which holds the totals), the barrier to every thread.
template <int NA, int kG>
__device__ __forceinline__ bool res2_sum(Acc<float> (&acc)[NA], ResShared<float> &sh, const ResArgs &a, int &buf,
                                         Acc<float> (&tot)[NA]) {
  if (kG == 2) return grid_sum<NA>(acc, sh, a, buf, tot);
  group_sum<float, NA, kG == 1>(acc, sh, buf, tot);
  return true;
}
template <int kG>
__device__ __forceinline__ bool res2_barrier(const ResArgs &a, ResShared<float> &sh) {
  if (kG == 2) return grid_sync(a, &sh.task);
  group_barrier<kG == 1>();
  return true;
}
// A whole-GPU barrier gave up (thread 0): the solve ends with ATS_ERR_TIMEOUT.
__device__ __forceinline__ void res2_timeout(ResState &st) {
  st.status = ATS_ERR_TIMEOUT;
  st.phase = kDone;
}

// The result of a solve on this CTA's octs [lo, hi), as k_final writes it:
// x (Crank-Nicolson: 2 x' - E^n) to xd, which may be device memory or host
// memory the device can write (then the result reaches the host while other
// solves still run).  *neg is set when a value is negative.
__device__ void res2_copy_out(const SolveDev &sd, double *xd, int lo, int hi, int *neg) {
  const bool vec = oct_aligned(xd) && oct_aligned(sd.cn_base);
  bool below = false;
  for (int o = lo + (int)threadIdx.x; o < hi; o += blockDim.x) {
    double v[8];
    ld8_rw(sd.x64 + 8 * (int64_t)o, v);
    if (sd.cn_base) {
      double cb[8];
      if (vec) {
        ld8_ro(sd.cn_base + 8 * (int64_t)o, cb);
      } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) cb[c] = sd.cn_base[8 * (int64_t)o + c];
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = 2.0 * v[c] - cb[c];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) below = below || v[c] < 0.0;
    if (vec) {
      st8(xd + 8 * (int64_t)o, v);
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) xd[8 * (int64_t)o + c] = v[c];
    }
  }
  if (__syncthreads_or(below) && neg && threadIdx.x == 0) atomicOr(neg, 1);
}

// One solve by one group, the CG state of its first octs in shared memory in
// the layout Cx.  kG: 0 one CTA, 1 a cluster, 2 the whole GPU (every CTA of
// a cooperative launch).  Returns false when a grid barrier wait gave up (the solve then
// ends with ATS_ERR_TIMEOUT).
template <int kG, class Cx>
__device__ bool res2_solve_l(const ResArgs &a, int s, ResShared<float> &sh, int &buf) {
  constexpr bool kCluster = kG == 1;
  constexpr int wd = (int)(sizeof(SolveDev) / 8);
  for (int w = threadIdx.x; w < wd; w += blockDim.x)
    reinterpret_cast<unsigned long long *>(&sh.sd)[w] = reinterpret_cast<const unsigned long long *>(a.solves + s)[w];
  const unsigned cs = kG == 2 ? gridDim.x : (kCluster ? cl_size() : 1u);
  const unsigned cr = kG == 2 ? blockIdx.x : (kCluster ? cl_rank() : 0u);
  if (threadIdx.x == 0) {
    ResState z;
    memset(&z, 0, sizeof(z));
    z.phase = kRefine;
    z.status = ATS_OK;
    sh.st = z;
    if (a.t_solve && cr == 0) a.t_solve[2 * s] = globaltimer_ns();
  }
  __syncthreads();
  const SolveDev &sd = sh.sd;
  const int n = sd.n_oct;
  Cx cx;
  cx.chunk = (int)((n + (int)cs - 1) / (int)cs);
  const bool six = Cx::capD > 0;
  cx.lo = min(n, (int)cr * cx.chunk);
  cx.cr = cr;
  cx.crc = kCluster ? cr : 0u;
  cx.grid = kG == 2;
  cx.qrec = a.q_recur != 0;
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(res2_smem);
  cx.sK = base;
  cx.sZ = base + 4u * cx.S;
  cx.sP = base + 8u * cx.S;
  cx.sD = base + 12u * cx.S;  // the six-array layout only
  cx.sQ = base + 16u * cx.S;
  cx.sE = base + 20u * cx.S;
  cx.sC = base + (six ? 24u : 12u) * cx.S;
  const int hi = min(n, cx.lo + cx.chunk);
  const int o0 = cx.lo + (int)threadIdx.x, stride = (int)blockDim.x;
  const float h = (float)sd.h;
  // stage in: K (scaled by h) and the neighbour codes of the octs kept in shared memory
  // (read by other CTAs only after the first sum's cluster barrier), and the
  // stand-in row a face without a neighbour points to
  if (threadIdx.x == 0) {
    float m1[8], z0[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      m1[c] = -1.f;
      z0[c] = 0.f;
    }
    sts_cells(cx.sK + (uint32_t)cx.cap * 8u, cx.S, m1);
    sts_cells(cx.sZ + (uint32_t)cx.cap * 8u, cx.S, z0);
    sts_cells(cx.sP + (uint32_t)cx.cap * 8u, cx.S, z0);
  }
  const uint16_t code_none = (uint16_t)((cx.crc << 12) | (unsigned)cx.cap);
  for (int o = o0; o < hi && o - cx.lo < cx.cap; o += stride) {
    const int l = o - cx.lo;
    float K[8];
    ld8_ro((const float *)sd.KT + 8 * o, K);
    res2_scale_K(h, K);
    sts_cells(cx.sK + (uint32_t)l * 8u, cx.S, K);
    if (l < cx.capD) {  // the correction of the first inner solve starts at zero
      float z0[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) z0[c] = 0.f;
      sts_cells(cx.sE + (uint32_t)l * 8u, cx.S, z0);
    }
    int g[6];
    load_nbr6(sd.nbr, o, g);
    check_nbr6(g, sd.n_oct);
    uint16_t c[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      c[d] = code_of_global(cx, g[d]);
      if (c[d] == kCodeNone) c[d] = code_none;
    }
    const uint32_t w0 = c[0] | ((uint32_t)c[1] << 16), w1 = c[2] | ((uint32_t)c[3] << 16),
                   w2 = c[4] | ((uint32_t)c[5] << 16);
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(cx.sC + (uint32_t)l * 16u), "r"(w0), "r"(w1),
                 "r"(w2), "r"(0u)
                 : "memory");
  }
  const bool want_x = sd.stop_rule == ATS_STOP_CERTIFIED;
  const bool f32 = a.cg_scalars == 0;
  for (;;) {
    const int phase = sh.st.phase;
    if (phase == kDone) break;
    if (phase == kRefine) {
      Acc<float> acc[3], tot[3];
      for (int o = o0; o < hi; o += stride) res2_ref_oct(cx, sd, o, want_x, acc[0], acc[1], acc[2]);
      const bool ok = res2_sum<3, kG>(acc, sh, a, buf, tot);
      if (threadIdx.x == 0 && !ok) res2_timeout(sh.st);
      if (threadIdx.x == 0 && ok) {
        ResState &st = sh.st;
        const double rnorm = sqrt(tot[0].get()), xnorm = sqrt(tot[1].get()), rz = tot[2].get();
        if (st.refines == 0) st.r0 = rnorm;
        st.refines += 1;
        st.rnorm = rnorm;
        st.xnorm = xnorm;
        const double target = sd.tol * (sd.stop_rule == ATS_STOP_CERTIFIED ? xnorm : st.r0);
        if (st.final_pass) {
          st.phase = kDone;
        } else if (!isfinite(rnorm)) {
          st.status = ATS_ERR_BREAKDOWN;
          st.phase = kDone;
        } else if (rnorm <= target) {
          st.phase = kDone;
        } else if (st.refines > sd.max_refine) {
          st.status = ATS_ERR_NOT_CONVERGED;
          st.phase = kDone;
        } else if (!(rz > 0.0)) {
          st.status = ATS_ERR_BREAKDOWN;
          st.phase = kDone;
        } else {
          st.phase = kInner;
          st.rz = rz;
          st.rzf = (float)rz;
          st.first = 1;
          st.inner_iters = 0;
          st.inner_target = fmax(sd.inner_rtol * rnorm, sd.final_safety * target);
          st.t2f = (float)(st.inner_target * st.inner_target);
        }
      }
      __syncthreads();
      continue;
    }
    // steps 1 and 2: the new direction p and q = (I + dt A) p, the sum p.q.
    // From p: p on the own octs, a group barrier (the neighbours' p), the
    // stencil of p.  By the recurrence: one pass, the stencil of z (final
    // since the last group sum) and p, q from their previous values.
    {
      const bool first = sh.st.first != 0;
      const float beta = sh.st.betaf;
      Acc<float> acc[1], tot[1];
      if (cx.qrec) {
        for (int o = o0; o < hi; o += stride) acc[0].add_value(res2_op_any<kCluster, true>(cx, sd, o, h, first, beta));
      } else {
        for (int o = o0; o < hi; o += stride) res2_dir_oct(cx, sd, o, first, beta);
        if (!res2_barrier<kG>(a, sh)) {
          if (threadIdx.x == 0) res2_timeout(sh.st);
          break;
        }
        for (int o = o0; o < hi; o += stride)
          acc[0].add_value(res2_op_any<kCluster, false>(cx, sd, o, h, first, beta));
      }
      const bool ok = res2_sum<1, kG>(acc, sh, a, buf, tot);
      if (threadIdx.x == 0 && !ok) res2_timeout(sh.st);
      if (threadIdx.x == 0 && ok) {
        ResState &st = sh.st;
        st.n_op += 1;
        st.n_first += st.first ? 1 : 0;
        cg_alpha(st, tot[0], f32);
      }
      __syncthreads();
    }
    if (sh.st.phase == kDone) break;
    // step 3: e += alpha p, r = D z - alpha q, z = D^-1 r; sums r.z, r.r
    {
      const float alpha = sh.st.alphaf;
      Acc<float> acc[2], tot[2];
      for (int o = o0; o < hi; o += stride) {
        float lrz = 0.f, lrr = 0.f;
        res2_upd_oct(cx, sd, o, alpha, lrz, lrr);
        acc[0].add_value(lrz);
        acc[1].add_value(lrr);
      }
      const bool ok = res2_sum<2, kG>(acc, sh, a, buf, tot);
      if (threadIdx.x == 0 && !ok) res2_timeout(sh.st);
      if (threadIdx.x == 0 && ok) {
        ResState &st = sh.st;
        st.iters += 1;
        st.inner_iters += 1;
        st.first = 0;
        const bool conv = cg_beta(st, tot[0], tot[1], f32);
        if (conv) {
          st.phase = kRefine;
        } else if (st.iters >= sd.max_iter) {
          st.status = ATS_ERR_NOT_CONVERGED;
          st.final_pass = 1;
          st.phase = kRefine;
        } else if (st.inner_iters >= sd.inner_max) {
          st.phase = kRefine;
        }
        if (st.phase == kRefine) st.n_xpe += 1;
      }
      __syncthreads();
    }
    if (sh.st.phase == kDone) break;
    if (sh.st.phase == kRefine) {
      for (int o = o0; o < hi; o += stride) res2_xpe_oct(cx, sd, o);
      if (!res2_barrier<kG>(a, sh)) {
        if (threadIdx.x == 0) res2_timeout(sh.st);
        break;
      }
    }
  }
  __syncthreads();  // thread 0's last state update is seen by all
  const bool alive = sh.st.status != ATS_ERR_TIMEOUT;
  // the result of the own octs (each CTA updated only its own octs' x)
  double *xd = a.x_out ? a.x_out[s] : nullptr;
  if (xd) res2_copy_out(sd, xd, cx.lo, hi, a.neg ? a.neg + s : nullptr);
  if (threadIdx.x == 0 && cr == 0) {
    const ResState &st = sh.st;
    SolveScalars f;
    memset(&f, 0, sizeof(f));
    f.phase = kDone;
    f.iters = st.iters;
    f.inner_iters = st.inner_iters;
    f.refines = st.refines;
    f.status = st.status;
    f.final_pass = st.final_pass;
    f.ticks = st.n_op + st.iters + st.refines;
    f.rz = st.rz;
    f.r0 = st.r0;
    f.inner_target = st.inner_target;
    f.rnorm = st.rnorm;
    f.xnorm = st.xnorm;
    a.final_sc[s] = f;
    if (a.t_solve) a.t_solve[2 * s + 1] = globaltimer_ns();
    if (a.cells) {
      const unsigned long long N = 8ull * (unsigned long long)n;
      atomicAdd(a.cells + 0, N * (unsigned long long)(st.n_op - st.n_first));
      atomicAdd(a.cells + 4, N * (unsigned long long)st.n_first);
      atomicAdd(a.cells + 1, N * (unsigned long long)st.refines);
      atomicAdd(a.cells + 2, N * (unsigned long long)st.iters);
      atomicAdd(a.cells + 3, N * (unsigned long long)st.n_xpe);
    }
  }
  return alive;
}

// One solve by one group: all six arrays in shared memory when the CTA's
// share fits, else K, z and p (the share's size decides, the arithmetic is
// the same); kGlobal: every array in global memory (a kernel of its own, so
// that the shared-memory kernels keep their register allocation).
template <int kG, bool kGlobal>
__device__ bool res2_solve(const ResArgs &a, int s, ResShared<float> &sh, int &buf) {
  const unsigned cs = kG == 2 ? gridDim.x : (kG == 1 ? cl_size() : 1u);
  const int n = a.solves[s].n_oct;
  const int chunk = (int)((n + (int)cs - 1) / (int)cs);
  if (kGlobal) return res2_solve_l<kG, Res2Global>(a, s, sh, buf);
  if (chunk <= kRes2Cap6) return res2_solve_l<kG, Res2Six>(a, s, sh, buf);
  return res2_solve_l<kG, Res2Three>(a, s, sh, buf);
}

template <bool kGlobal>
__device__ void res2_cta_loop(const ResArgs &a, ResShared<float> &sh, int &buf) {
  for (;;) {
    __syncthreads();  // every thread has read the previous task and left the previous solve
    if (threadIdx.x == 0) sh.task = atomicAdd(a.tq_head, 1);
    __syncthreads();
    const int t = sh.task;
    if (t >= a.n_tq) break;
    int s = a.tq[t];
    if (!idx_ok(s, a.n_solves)) continue;
    res2_solve<0, kGlobal>(a, s, sh, buf);
  }
}

}  // namespace

template <int NT, bool kGlobal>
__global__ void __launch_bounds__(NT, 1) k_res2_cluster(ResArgs a) {
  __shared__ ResShared<float> sh;
  int buf = 0;
  const unsigned cr = cl_rank(), cs = cl_size();
  for (;;) {
    if (cr == 0 && threadIdx.x == 0) {
      const int t = atomicAdd(a.cq_head, 1);
      for (unsigned r = 0; r < cs; ++r) cl_st(cl_map(&sh.task, r), t);
    }
    cl_sync();
    const int t = sh.task;
    if (t >= a.n_cq) break;
    const int s = a.cq[t];
    if (idx_ok(s, a.n_solves)) res2_solve<1, kGlobal>(a, s, sh, buf);
    cl_sync();  // every CTA is done with the shared rows before the next stage-in rewrites them
  }
  res2_cta_loop<kGlobal>(a, sh, buf);
}

template <int NT, bool kGlobal>
__global__ void __launch_bounds__(NT, 1) k_res2_cta(ResArgs a) {
  __shared__ ResShared<float> sh;
  int buf = 0;
  res2_cta_loop<kGlobal>(a, sh, buf);
}

// The whole-GPU form: every CTA of one cooperative launch takes part in
// every solve of the grid queue, in queue order.  After a barrier wait gave
// up, the remaining solves are not started: CTA 0 records them as timed out.
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_res2_grid(ResArgs a) {
  __shared__ ResShared<float> sh;
  int buf = 0;
  bool alive = true;
  for (int t = 0; t < a.n_gq; ++t) {
    const int s = a.gq[t];
    if (!idx_ok(s, a.n_solves)) continue;
    if (alive) {
      alive = res2_solve<2, false>(a, s, sh, buf);
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
      SolveScalars f;
      memset(&f, 0, sizeof(f));
      f.phase = kDone;
      f.status = ATS_ERR_TIMEOUT;
      a.final_sc[s] = f;
    }
    __syncthreads();  // every thread has left the solve before the next stage-in
  }
}

template <typename T, int NT>
static cudaError_t res_launch_t(int cluster, int grid, const ResArgs &a, cudaStream_t st, bool cta_only) {
  if (a.n_cq > 0 && !cta_only) {
    if (cluster > 8) {
      cudaError_t e = cudaFuncSetAttribute(k_res_cluster<T, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_res_cluster<T, NT>, a);
  }
  k_res_cta<T, NT><<<grid, NT, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int NT>
static int res_clusters_t(int cluster) {
  if (cluster > 8 &&
      cudaFuncSetAttribute(k_res_cluster<T, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cluster * 64));
  cfg.blockDim = dim3(NT);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_res_cluster<T, NT>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T, int NT>
static int res_cta_blocks_t() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_res_cta<T, NT>, NT, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}

template <int NT, bool kG>
static cudaError_t res2_launch_k(int cluster, int grid, const ResArgs &a, cudaStream_t st, bool cta_only,
                                 int priority) {
  const size_t smem = kRes2SmemBytes;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  if (a.n_cq > 0 && !cta_only) {
    cudaError_t e = cudaFuncSetAttribute(k_res2_cluster<NT, kG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && cluster > 8)
      e = cudaFuncSetAttribute(k_res2_cluster<NT, kG>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = (unsigned)cluster;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_res2_cluster<NT, kG>, a);
  }
  cudaError_t e = cudaFuncSetAttribute(k_res2_cta<NT, kG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_res2_cta<NT, kG>, a);
}

template <int NT>
static cudaError_t res2_launch_t(int cluster, int grid, const ResArgs &a, cudaStream_t st, bool cta_only,
                                 int priority) {
  return a.cap == 0 ? res2_launch_k<NT, true>(cluster, grid, a, st, cta_only, priority)
                    : res2_launch_k<NT, false>(cluster, grid, a, st, cta_only, priority);
}

template <int NT>
static int res2_clusters_t(int cluster, int cap) {
  (void)cap;
  const size_t smem = kRes2SmemBytes;
  if (cudaFuncSetAttribute(k_res2_cluster<NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      (cluster > 8 &&
       cudaFuncSetAttribute(k_res2_cluster<NT, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cluster * 64));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_res2_cluster<NT, false>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// kRes2Cap3 when the layouts fit the shared memory a CTA can have beside the
// kernels' static shared memory, else 0 (the shared-memory form is then off).
template <int NT>
static int res2_cap_t(int device) {
  int optin = 0;
  cudaFuncAttributes fa, fb;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_res2_cluster<NT, false>) != cudaSuccess ||
      cudaFuncGetAttributes(&fb, k_res2_cta<NT, false>) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t stat = std::max(fa.sharedSizeBytes, fb.sharedSizeBytes);
  return (size_t)optin >= stat + kRes2SmemBytes ? kRes2Cap3 : 0;
}

cudaError_t launch_resident_smem(int threads, int cluster, int grid, const ResArgs &a, cudaStream_t st, bool cta_only,
                                 int priority) {
  if (a.n_cq + a.n_tq <= 0) return cudaSuccess;
  if (cluster < 1 || cluster > kMaxCluster || grid <= 0 || (a.cap != kRes2Cap3 && a.cap != 0))
    return cudaErrorInvalidValue;
  return threads >= 512 ? res2_launch_t<512>(cluster, grid, a, st, cta_only, priority)
                        : res2_launch_t<256>(cluster, grid, a, st, cta_only, priority);
}

int resident_smem_clusters(int threads, int cluster, int cap) {
  if (cluster < 1 || cluster > kMaxCluster || cap < 0) return 0;
  return threads >= 512 ? res2_clusters_t<512>(cluster, cap) : res2_clusters_t<256>(cluster, cap);
}

int resident_smem_cap(int threads, int device) {
  return threads >= 512 ? res2_cap_t<512>(device) : res2_cap_t<256>(device);
}

template <int NT>
static cudaError_t res2_grid_launch_t(int grid, const ResArgs &a, cudaStream_t st) {
  const size_t smem = kRes2SmemBytes;
  cudaError_t e = cudaFuncSetAttribute(k_res2_grid<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_res2_grid<NT>, a);
}

template <int NT>
static int res2_grid_ctas_t(int device) {
  int b = 0, sms = 0;
  if (cudaFuncSetAttribute(k_res2_grid<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRes2SmemBytes) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_res2_grid<NT>, NT, kRes2SmemBytes) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b * sms;
}

// A one-thread kernel that returns after `ns` nanoseconds of %globaltimer
// (or after 2^20 reads of it, whichever comes first): it holds back the work
// queued behind it on its stream.
__global__ void k_hold(unsigned long long ns) {
  const unsigned long long t0 = globaltimer_ns();
  for (int it = 0; it < (1 << 20) && globaltimer_ns() - t0 < ns; ++it) __nanosleep(256);
}

cudaError_t launch_hold(unsigned long long ns, cudaStream_t st) {
  k_hold<<<1, 1, 0, st>>>(ns);
  return cudaGetLastError();
}

cudaError_t launch_resident_grid(int threads, int grid, const ResArgs &a, cudaStream_t st) {
  if (a.n_gq <= 0) return cudaSuccess;
  if (threads != 512 || grid <= 0 || grid > 32 * kGridMaxPerLane || a.cap != kRes2Cap3 || !a.gbar || !a.gpart ||
      !a.gerr)
    return cudaErrorInvalidValue;
  return res2_grid_launch_t<512>(grid, a, st);
}

int resident_six_cap() { return kRes2Cap6; }

int resident_grid_ctas(int threads, int device) {
  if (threads != 512) return 0;  // compiled for 512-thread CTAs only
  return std::min(32 * kGridMaxPerLane, res2_grid_ctas_t<512>(device));
}

// One grid barrier of the whole-GPU form on its own, every CTA recording
// whether its wait ended normally (out[cta] = 1) or gave up (0).
__global__ void k_grid_barrier_probe(ResArgs a, int *out) {
  __shared__ int flag;
  const bool ok = grid_sync(a, &flag);
  if (threadIdx.x == 0) out[blockIdx.x] = ok ? 1 : 0;
}

cudaError_t launch_grid_barrier_probe(int grid, const ResArgs &a, int *out, cudaStream_t st) {
  if (grid <= 0 || !a.gbar || !a.gerr || !out) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(32);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_grid_barrier_probe, a, out);
}

cudaError_t launch_resident(bool fp64, int threads, int cluster, int grid, const ResArgs &a, cudaStream_t st,
                            bool cta_only) {
  if (a.n_cq + a.n_tq <= 0) return cudaSuccess;
  if (cluster < 1 || cluster > kMaxCluster || grid <= 0) return cudaErrorInvalidValue;
  if (!fp64) return cudaErrorInvalidValue;  // FP32 bulk: launch_resident_smem
  return threads >= 512 ? res_launch_t<double, 512>(cluster, grid, a, st, cta_only)
                        : res_launch_t<double, 256>(cluster, grid, a, st, cta_only);
}

int resident_max_clusters(bool fp64, int threads, int cluster) {
  if (cluster < 1 || cluster > kMaxCluster) return 0;
  if (!fp64) return 0;
  return threads >= 512 ? res_clusters_t<double, 512>(cluster) : res_clusters_t<double, 256>(cluster);
}

int resident_cta_blocks(bool fp64, int threads) {
  if (!fp64) return 0;
  return threads >= 512 ? res_cta_blocks_t<double, 512>() : res_cta_blocks_t<double, 256>();
}

}  // namespace ats

// Out-of-range gathered indices counted by a bounds-checked build since the
// last call (the count restarts at zero); -1 from the default build.
extern "C" ats_status ats_bounds_violations(int device, long long *count) {
  if (!count) return ATS_ERR_INVALID_ARG;
#if ATS_BOUNDS_CHECK
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return ATS_ERR_CUDA;
  }
  unsigned long long v = 0;
  const unsigned long long zero = 0;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpyFromSymbol(&v, ats::g_bound_violations, sizeof(v)) != cudaSuccess ||
      cudaMemcpyToSymbol(ats::g_bound_violations, &zero, sizeof(zero)) != cudaSuccess) {
    cudaGetLastError();
    return ATS_ERR_CUDA;
  }
  *count = (long long)v;
#else
  (void)device;
  *count = -1;
#endif
  return ATS_OK;
}

// One grid barrier of the whole-GPU solver, alone: `ctas` CTAs (0: one per
// SM) wait for ctas + extra arrivals.  With extra > 0 nothing ever completes
// the barrier, so every wait must give up on its own.
extern "C" ats_status ats_grid_barrier_selftest(int device, int ctas, int extra, int *n_normal, int *n_gave_up,
                                                double *ms) {
  if (ctas < 0 || extra < 0 || !n_normal || !n_gave_up || !ms) return ATS_ERR_INVALID_ARG;
  int sms = 0;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return ATS_ERR_CUDA;
  }
  const int grid = ctas > 0 ? ctas : sms;
  if (grid > sms) return ATS_ERR_INVALID_ARG;  // one 32-thread CTA per SM is always co-resident
  unsigned *bar = nullptr;
  int *gerr = nullptr, *out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc(&bar, 2 * sizeof(unsigned));
  if (err == cudaSuccess) err = cudaMalloc(&gerr, sizeof(int));
  if (err == cudaSuccess) err = cudaMalloc(&out, sizeof(int) * grid);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) err = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(gerr, 0, sizeof(int), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(out, 0xFF, sizeof(int) * grid, st);
  ats::ResArgs a;
  std::memset(&a, 0, sizeof(a));
  a.gbar = bar;
  a.gerr = gerr;
  a.g_expect = grid + extra;
  if (err == cudaSuccess) err = cudaEventRecord(e0, st);
  if (err == cudaSuccess) err = ats::launch_grid_barrier_probe(grid, a, out, st);
  if (err == cudaSuccess) err = cudaEventRecord(e1, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  std::vector<int> h(grid, -1);
  int flag = 0;
  float t = 0.f;
  if (err == cudaSuccess) err = cudaMemcpy(h.data(), out, sizeof(int) * grid, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaMemcpy(&flag, gerr, sizeof(int), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(bar);
  cudaFree(gerr);
  cudaFree(out);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return ATS_ERR_CUDA;
  }
  int normal = 0, gave_up = 0;
  for (int v : h) {
    normal += v == 1;
    gave_up += v == 0;
  }
  *n_normal = normal;
  *n_gave_up = gave_up;
  *ms = (double)t;
  // every wait that gave up must have raised the flag
  return (gave_up > 0) == (flag != 0) ? ATS_OK : ATS_ERR_CUDA;
}
