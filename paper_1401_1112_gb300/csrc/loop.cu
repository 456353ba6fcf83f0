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

cudaError_t make_while_graph(cudaGraph_t *graph, cudaGraph_t *body, cudaGraphConditionalHandle *handle) {
  *graph = nullptr;
  *body = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaGraphCreate(&g, 0);
  if (err != cudaSuccess) return err;
  cudaGraphConditionalHandle h;
  err = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  if (err == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    err = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  }
  if (err != cudaSuccess) {
    cudaGraphDestroy(g);
    return err;
  }
  *graph = g;
  *body = np.conditional.phGraph_out[0];
  *handle = h;
  return cudaSuccess;
}

cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, const int *n_active, int *chunks, int max_chunks,
                             cudaStream_t st) {
  k_loop_cond<<<1, 1, 0, st>>>(h, n_active, chunks, max_chunks);
  return cudaGetLastError();
}

}  // namespace ats
