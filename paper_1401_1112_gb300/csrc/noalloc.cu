// ats_solve_noalloc: the single-level FP64 Jacobi-PCG solve without any
// device allocation.
//
// Who needs it: callers that cannot call cudaMalloc -- plug-ins handed a fixed
// memory pool by a host application that owns every device allocation, and
// processes whose device memory belongs to another runtime's allocator (a
// framework's caching allocator) that must not be bypassed or made to give
// memory back.  They pass device pointers for every input and output; the CG
// vectors, reduction partials, work list and per-solve scalars live in one
// file-scope device array defined below, which every GPU that loads this
// library keeps until the process exits.
//
// The call is synchronous: it copies its descriptors from host memory, polls
// the solve's progress from the host and synchronises the caller's stream
// before it returns.  So it cannot run inside a CUDA stream capture; a stream
// that is being captured is rejected with ATS_ERR_INVALID_ARG before any work
// is enqueued on it.
//
// Limits and sharing: at most kNoAllocMaxCells cells per call (larger
// requests are rejected).  All calls share the one array and it keeps the
// last call's contents; each call re-initialises every part it reads before
// use (the correction vector e is zeroed, the scalars and lists are written
// from the host).  Calls whose work overlaps on the GPU (two host threads, or
// two streams) race on the array: serialise them.
//
// Set-up: the first call on each device looks up the device address of the
// array (cudaGetSymbolAddress) with that device current.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <mutex>
#include <string>

#include "ats_internal.h"

namespace ats {
namespace {

constexpr int64_t kNoAllocMaxCells = ATS_NOALLOC_MAX_CELLS;
constexpr int kNoAllocTile = 2 * kThreads;  // octs per work item
constexpr int kNoAllocMaxItems = (int)((kNoAllocMaxCells / 8 + kNoAllocTile - 1) / kNoAllocTile);
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// byte layout of the scratch array
constexpr size_t kOffSolve = 0;
constexpr size_t kOffScal = align256(kOffSolve + sizeof(SolveDev));  // [2] by parity, then [1] final
constexpr size_t kOffCtl = align256(kOffScal + 3 * sizeof(SolveScalars));
constexpr size_t kOffActive = align256(kOffCtl + sizeof(TickCtl));
constexpr size_t kOffItems = align256(kOffActive + sizeof(int));
constexpr size_t kOffLists = align256(kOffItems + sizeof(WorkItem) * kNoAllocMaxItems);
constexpr size_t kOffPart = align256(kOffLists + sizeof(int32_t) * 4 * kNoAllocMaxItems);
constexpr size_t kOffXrec = align256(kOffPart + 3 * sizeof(double) * kNumPartials * kNoAllocMaxItems);
constexpr size_t kOffVec = align256(kOffXrec + sizeof(int32_t) * (kNoAllocMaxCells / 8));
constexpr size_t kVecBytes = align256(sizeof(double) * kNoAllocMaxCells);
constexpr size_t kScratchBytes = kOffVec + 9 * kVecBytes;  // e, z, p0, p1, q, D, then C64 (3 vectors)

}  // namespace

// The scratch array (about 19 MB for the default maximum of 2^18 cells).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

__global__ void k_fill_xrec(int32_t *xrec, int n_oct, int identity) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < n_oct) xrec[o] = identity ? o : -1;
}

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace
}  // namespace ats

using namespace ats;

extern "C" ats_status ats_solve_noalloc(int device, void *stream, int64_t n_oct, const int32_t *nbr,
                                        const double *K, const double *xd, double h, const double *b,
                                        double *x, double tol, int max_iter, ats_solve_stats *stats) {
  try {  // no C++ exception leaves the library
    if (!nbr || !K || !b || !x) {
      set_error("ats_solve_noalloc: nbr, K, b and x are required device pointers");
      return ATS_ERR_INVALID_ARG;
    }
    if (n_oct <= 0 || 8 * n_oct > kNoAllocMaxCells) {
      set_error("ats_solve_noalloc: level size must be 1 .. " + std::to_string(kNoAllocMaxCells) +
                " cells (the fixed scratch array holds no more)");
      return ATS_ERR_INVALID_ARG;
    }
    if (!(h > 0.0) || !(tol > 0.0) || device < 0 || device >= kMaxDevices) {
      set_error("ats_solve_noalloc: h and tol must be > 0, device in range");
      return ATS_ERR_INVALID_ARG;
    }
    // the kernels move an oct's eight FP64 values as two 32-byte accesses
    if (((uintptr_t)K | (uintptr_t)xd | (uintptr_t)b | (uintptr_t)x) & 31u) {
      set_error("ats_solve_noalloc: K, xd, b and x must be 32-byte aligned device pointers");
      return ATS_ERR_INVALID_ARG;
    }
    if (max_iter <= 0) max_iter = 20000;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
      set_error(std::string("ats_solve_noalloc: cudaSetDevice: ") + cudaGetErrorString(e));
      return ATS_ERR_CUDA;
    }
    unsigned char *base = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_setup_mutex);
      if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
          set_error(std::string("ats_solve_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
          return ATS_ERR_CUDA;
        }
        g_scratch_ptr[device] = p;
      }
      base = (unsigned char *)g_scratch_ptr[device];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the call synchronises st and reads the solve state back to the host,
    // which a stream capture does not allow: refuse before enqueuing anything
    {
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      e = cudaStreamIsCapturing(st, &cap);
      if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("ats_solve_noalloc: cudaStreamIsCapturing: ") + cudaGetErrorString(e));
        return ATS_ERR_INVALID_ARG;
      }
      if (cap != cudaStreamCaptureStatusNone) {
        set_error("ats_solve_noalloc: the stream is being captured; the call synchronises its stream and cannot "
                  "be captured into a CUDA graph");
        return ATS_ERR_INVALID_ARG;
      }
    }
  
    SolveDev *d_solve = (SolveDev *)(base + kOffSolve);
    SolveScalars *d_sc = (SolveScalars *)(base + kOffScal);
    TickCtl *d_ctl = (TickCtl *)(base + kOffCtl);
    int *d_active = (int *)(base + kOffActive);
    WorkItem *d_items = (WorkItem *)(base + kOffItems);
    int32_t *d_lists = (int32_t *)(base + kOffLists);
    double *d_part = (double *)(base + kOffPart);
    int32_t *d_xrec = (int32_t *)(base + kOffXrec);
    double *vec = (double *)(base + kOffVec);
    const size_t vstride = kVecBytes / sizeof(double);
  
    // host-side descriptors on the stack (no heap either)
    const int n_items = (int)((n_oct + kNoAllocTile - 1) / kNoAllocTile);
    WorkItem items[kNoAllocMaxItems];
    int32_t first_list[kNoAllocMaxItems];
    for (int i = 0; i < n_items; ++i) {
      items[i].solve = 0;
      items[i].oct_begin = i * kNoAllocTile;
      items[i].n_oct = (int32_t)((n_oct - (int64_t)i * kNoAllocTile) < kNoAllocTile ? n_oct - (int64_t)i * kNoAllocTile
                                                                                    : kNoAllocTile);
      items[i].pad = 0;
      first_list[i] = i;
    }
    SolveDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.nbr = nbr;
    sd.xrec = d_xrec;
    sd.n_xd = xd ? (int32_t)n_oct : 0;
    sd.K64 = K;
    sd.KT = K;
    sd.xd64 = xd;
    sd.xdT = xd;
    sd.b64 = b;
    sd.x64 = x;
    sd.e = vec;
    sd.z = vec + vstride;
    sd.p0 = vec + 2 * vstride;
    sd.p1 = vec + 3 * vstride;
    sd.q = vec + 4 * vstride;
    sd.dg = vec + 5 * vstride;
    sd.C64 = vec + 6 * vstride;
    sd.h = h;
    sd.tol = tol;
    sd.inner_rtol = 0.0;
    sd.final_safety = 1.0;
    sd.n_oct = (int32_t)n_oct;
    sd.item_begin = 0;
    sd.n_items = n_items;
    sd.stop_rule = ATS_STOP_RESIDUAL;
    sd.max_iter = max_iter;
    sd.max_refine = 40;
    sd.inner_max = max_iter;
    SolveScalars sc;
    std::memset(&sc, 0, sizeof(sc));
    sc.phase = kRefine;
    sc.status = ATS_OK;
    TickCtl ctl;
    std::memset(&ctl, 0, sizeof(ctl));
    ctl.count[0][kRefine] = n_items;
    const int one = 1;
  
  #define NA_TRY(expr)                                                                      \
    do {                                                                                    \
      cudaError_t _e = (expr);                                                              \
      if (_e != cudaSuccess) {                                                              \
        set_error(std::string("ats_solve_noalloc: ") + cudaGetErrorString(_e) + " at " #expr); \
        return ATS_ERR_CUDA;                                                                \
      }                                                                                     \
    } while (0)
  
    NA_TRY(cudaMemcpyAsync(d_solve, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_sc + 2, &sc, sizeof(sc), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_active, &one, sizeof(int), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_items, items, sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_lists + (size_t)kRefine * n_items, first_list, sizeof(int32_t) * n_items,
                           cudaMemcpyHostToDevice, st));
    k_fill_xrec<<<(unsigned)((n_oct + 255) / 256), 256, 0, st>>>(d_xrec, (int)n_oct, xd != nullptr);
    NA_TRY(cudaGetLastError());
    NA_TRY(launch_face_coef(n_oct, nbr, K, h, vec + 6 * vstride, st));
    NA_TRY(cudaGetLastError());
    int sms = 1, bps = tick_blocks_per_sm(true, false);
    NA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int grid = n_items < bps * sms ? n_items : bps * sms;
    int grids[3];
    tick_grids(true, false, device, grids);
    for (int k = 0; k < 3; ++k) grids[k] = n_items < grids[k] ? n_items : grids[k];
    NA_TRY(launch_init(true, d_solve, d_items, n_items, nullptr, grid, st));
    // the host copies above read stack memory: finish them before it goes away
    NA_TRY(cudaStreamSynchronize(st));
  
    TickArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.solves = d_solve;
    ta.sbuf = d_sc;
    ta.final_sc = d_sc + 2;
    ta.items = d_items;
    ta.lists = d_lists;
    ta.n_items = n_items;
    ta.n_solves = 1;
    ta.ctl = d_ctl;
    ta.p_op = d_part;
    ta.p_upd = d_part + (size_t)n_items * kNumPartials;
    ta.n_active = d_active;
    ta.cells = nullptr;
    const int64_t max_ticks = 2 * ((int64_t)max_iter + 2 * (40 + 2)) + 16;
    int64_t ticks = 0;
    int active = 1;
    while (active > 0 && ticks < max_ticks) {
      for (int t = 0; t < 8; ++t)
        NA_TRY(launch_tick(true, false, ta, grids, st, nullptr, nullptr, false));
      ticks += 8;
      NA_TRY(cudaMemcpyAsync(&active, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
      NA_TRY(cudaStreamSynchronize(st));
    }
    SolveScalars out;
    NA_TRY(cudaMemcpyAsync(&out, d_sc + 2, sizeof(out), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
  #undef NA_TRY
    ats_status status = out.status;
    if (active > 0 && status == ATS_OK) status = ATS_ERR_TIMEOUT;
    if (stats) {
      stats->status = status;
      stats->iterations = out.iters;
      stats->refinements = out.refines;
      stats->ticks = out.ticks;
      stats->r0_norm = out.r0;
      stats->res_norm = out.rnorm;
      stats->x_norm = out.xnorm;
      stats->err_bound = out.xnorm > 0.0 ? out.rnorm / out.xnorm : 0.0;
    }
    if (status != ATS_OK) set_error(std::string("ats_solve_noalloc: ") + ats_status_string(status));
    return status;
  } catch (...) {
    return ats::abi_exception();
  }
}
