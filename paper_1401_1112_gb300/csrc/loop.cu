// Device-side control of the tick loop: the condition kernel of a CUDA graph
// WHILE node (conditional graph node) whose body is one poll interval of
// ticks.  The loop of a solve then runs as one graph launch with no host
// round trip per interval.

#include <cuda_runtime.h>

#include "ats_internal.h"

namespace ats {

namespace {

// After each interval: continue while a solve is active and fewer than
// max_chunks intervals have run.  *chunks counts the intervals (zeroed before
// the graph launch), so the loop ends after at most max_chunks intervals
// whatever the solves do.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int *__restrict__ n_active, int *chunks,
                            int max_chunks) {
  const int c = *chunks + 1;
  *chunks = c;
  const bool more = c >= 1 && c < max_chunks && *n_active > 0;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

}  // namespace

cudaError_t add_while_loop(cudaGraph_t graph, const cudaGraphNode_t *deps, size_t n_deps, cudaGraph_t interval,
                           const int *n_active, int *chunks, int max_chunks, cudaGraphNode_t *node_out) {
  // the handle's default value 1, assigned at every launch of the graph, runs
  // the body once before the first test
  cudaGraphConditionalHandle h;
  cudaError_t err = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  if (err != cudaSuccess) return err;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((err = cudaGraphAddNode(&node, graph, deps, nullptr, n_deps, &np)) != cudaSuccess) return err;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  // body: the interval (cloned), then the condition kernel
  cudaGraphNode_t ticks, cond;
  if ((err = cudaGraphAddChildGraphNode(&ticks, body, nullptr, 0, interval)) != cudaSuccess) return err;
  void *args[4] = {&h, &n_active, &chunks, &max_chunks};
  cudaKernelNodeParams kp = {};
  kp.func = (void *)k_loop_cond;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  if ((err = cudaGraphAddKernelNode(&cond, body, &ticks, 1, &kp)) != cudaSuccess) return err;
  *node_out = node;
  return cudaSuccess;
}

}  // namespace ats
