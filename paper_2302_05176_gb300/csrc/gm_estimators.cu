// gm_estimators.cu -- estimators over finished sketches (Sec. 1, Sec. 2.4) and the
// union of sketches (Sec. 2.3, Mergeability).
#include <cuda_runtime.h>

#include "gm.h"
#include "gm_diag.h"
#include "gm_estim.cuh"
#include "gm_internal.h"

namespace gm {

static cudaEvent_t g_aux_before = nullptr, g_aux_after = nullptr;

void aux_events(cudaEvent_t* before, cudaEvent_t* after) {
  *before = g_aux_before;
  *after = g_aux_after;
}

// Launch `launch()` between the registered timing events, if any.
template <class F>
static int timed_launch(cudaStream_t st, F launch) {
  if (g_aux_before) cudaEventRecord(g_aux_before, st);
  launch();
  if (g_aux_after) cudaEventRecord(g_aux_after, st);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

// One warp per pair: count equal, filled registers.
__global__ void jaccard_kernel(const int32_t* __restrict__ sa, const int32_t* __restrict__ sb, int64_t n_pairs,
                               int k, double* __restrict__ out) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); p < n_pairs; p += warps) {
    const double j = warp_jaccard(sa + p * k, sb + p * k, k);
    if ((threadIdx.x & 31) == 0) out[p] = j;
  }
}

// One warp per row: (k - 1) / sum of the registers.
__global__ void cardinality_kernel(const double* __restrict__ y, int n_rows, int k, double* __restrict__ out) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); r < n_rows; r += warps) {
    const double c = warp_cardinality(y + r * k, k);
    if ((threadIdx.x & 31) == 0) out[r] = c;
  }
}

__global__ void merge_kernel(const int32_t* __restrict__ sa, const double* __restrict__ ya,
                             const int32_t* __restrict__ sb, const double* __restrict__ yb, int64_t n,
                             int32_t* s_out, double* y_out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s1 = sa[j], s2 = sb[j];
    const double y1 = ya[j], y2 = yb[j];
    // (y, id) compared as unsigned bit patterns; an unfilled id (-1) sorts last
    const unsigned long long b1 = (unsigned long long)__double_as_longlong(y1);
    const unsigned long long b2 = (unsigned long long)__double_as_longlong(y2);
    const uint32_t i1 = (uint32_t)s1, i2 = (uint32_t)s2;
    const bool take2 = b2 < b1 || (b2 == b1 && i2 < i1);
    s_out[j] = take2 ? s2 : s1;
    y_out[j] = take2 ? y2 : y1;
  }
}

static int grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

}  // namespace gm

extern "C" int gm_jaccard(const int32_t* s_a, const int32_t* s_b, int64_t n_pairs, int32_t k, double* out,
                          void* stream) {
  if (k < 1 || n_pairs < 0) return GM_EINVAL;
  if (n_pairs == 0) return GM_OK;
  if (!s_a || !s_b || !out) return GM_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  return gm::timed_launch(st, [&] {
    gm::jaccard_kernel<<<gm::grid_for(n_pairs, gm::EST_BLOCK / 32), gm::EST_BLOCK, 0, st>>>(s_a, s_b, n_pairs, k,
                                                                                             out);
  });
}

extern "C" int gm_cardinality(const double* y, int32_t n_rows, int32_t k, double* out, void* stream) {
  if (k < 2 || n_rows < 0) return GM_EINVAL;
  if (n_rows == 0) return GM_OK;
  if (!y || !out) return GM_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  return gm::timed_launch(st, [&] {
    gm::cardinality_kernel<<<gm::grid_for(n_rows, gm::EST_BLOCK / 32), gm::EST_BLOCK, 0, st>>>(y, n_rows, k, out);
  });
}

extern "C" int gm_merge(const int32_t* s_a, const double* y_a, const int32_t* s_b, const double* y_b, int64_t n_regs,
                        int32_t* s_out, double* y_out, void* stream) {
  if (n_regs < 0) return GM_EINVAL;
  if (n_regs == 0) return GM_OK;
  if (!s_a || !y_a || !s_b || !y_b || !s_out || !y_out) return GM_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  return gm::timed_launch(st, [&] {
    gm::merge_kernel<<<gm::grid_for(n_regs, gm::EST_BLOCK), gm::EST_BLOCK, 0, st>>>(s_a, y_a, s_b, y_b, n_regs,
                                                                                    s_out, y_out);
  });
}

extern "C" int gm_diag_time_aux_kernels(void* before, void* after) {
  if ((before == nullptr) != (after == nullptr)) return GM_EINVAL;
  gm::g_aux_before = (cudaEvent_t)before;
  gm::g_aux_after = (cudaEvent_t)after;
  return GM_OK;
}
