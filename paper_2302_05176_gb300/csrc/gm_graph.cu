// gm_graph.cu -- one gm_sketch call captured into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <new>

#include "gm.h"
#include "gm_internal.h"

struct gm_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" int gm_graph_create(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                               int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out,
                               void* workspace, size_t workspace_bytes, gm_graph** out) {
  if (!out) return GM_EINVAL;
  *out = nullptr;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return GM_ECUDA;
  // Relaxed mode: the launcher's attribute and occupancy queries run at capture
  // time and are not recorded; only the kernels are.
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaStreamDestroy(st);
    return GM_ECUDA;
  }
  const int rc = gm::launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, workspace,
                                   workspace_bytes, st, false, nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &g);
  cudaStreamDestroy(st);
  if (rc != GM_OK || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != GM_OK ? rc : GM_ECUDA;
  }
  gm_graph* h = new (std::nothrow) gm_graph();
  if (!h) {
    cudaGraphDestroy(g);
    return GM_ENOMEM;
  }
  h->graph = g;
  if (cudaGraphInstantiate(&h->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    delete h;
    cudaGetLastError();
    return GM_ECUDA;
  }
  *out = h;
  return GM_OK;
}

extern "C" int gm_graph_launch(gm_graph* h, void* stream) {
  if (!h || !h->exec) return GM_EINVAL;
  return cudaGraphLaunch(h->exec, (cudaStream_t)stream) == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_graph_destroy(gm_graph* h) {
  if (!h) return GM_EINVAL;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  delete h;
  return GM_OK;
}
