// Cell diffusion-coefficient models evaluated on the device.

#include <cuda_runtime.h>

#include <string>

#include "ats_internal.h"

namespace ats {
namespace {

// K_i = K0 E_i^p (the power law of the nonlinear equilibrium test, Sect. 4.2)
__global__ void k_power_law_K(int64_t n, const double *__restrict__ E, double K0, double p, double *__restrict__ K) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) K[i] = K0 * pow(E[i], p);
}

__global__ void k_power_law_K_leaf(int64_t n, const uint8_t *__restrict__ leaf, const double *__restrict__ E, double K0,
                                   double p, double *__restrict__ K) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (leaf && !((leaf[i >> 3] >> (i & 7)) & 1)) return;
  K[i] = K0 * pow(E[i], p);
}

}  // namespace

cudaError_t launch_power_law_K(int64_t n_cell, const uint8_t *leaf, const double *E, double K0, double a, double *K,
                               cudaStream_t st) {
  if (n_cell <= 0) return cudaSuccess;
  k_power_law_K_leaf<<<(unsigned)((n_cell + 255) / 256), 256, 0, st>>>(n_cell, leaf, E, K0, a, K);
  return cudaGetLastError();
}

}  // namespace ats

extern "C" {

ats_status ats_power_law_K(ats_context *ctx, int64_t n, const double *E, double K0, double p, double *K) {
  try {  // no C++ exception leaves the library
    if (!ctx || n < 0 || (n > 0 && (!E || !K))) {
      ats::set_error("ats_power_law_K: bad argument");
      return ATS_ERR_INVALID_ARG;
    }
    if (n == 0) return ATS_OK;
    cudaError_t e = cudaSetDevice(ats::ctx_device(ctx));
    if (e == cudaSuccess) {
      const unsigned blocks = (unsigned)((n + 255) / 256);
      ats::k_power_law_K<<<blocks, 256, 0, ats::ctx_stream(ctx)>>>(n, E, K0, p, K);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      ats::set_error(std::string("ats_power_law_K: ") + cudaGetErrorString(e));
      return ATS_ERR_CUDA;
    }
    return ATS_OK;
  } catch (...) {
    return ats::abi_exception();
  }
}

}  // extern "C"
