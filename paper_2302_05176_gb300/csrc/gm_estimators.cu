// gm_estimators.cu -- estimators over finished sketches (Sec. 1, Sec. 2.4) and the
// union of sketches (Sec. 2.3, Mergeability).
#include <cuda_runtime.h>

#include "gm.h"

namespace gm {

constexpr int EST_BLOCK = 256;

// One warp per pair: count equal, filled registers with ballots.
__global__ void jaccard_kernel(const int32_t* __restrict__ sa, const int32_t* __restrict__ sb, int64_t n_pairs,
                               int k, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); p < n_pairs; p += warps) {
    const int32_t* a = sa + p * k;
    const int32_t* b = sb + p * k;
    int hits = 0;
    for (int j = lane; j < k; j += 32) {
      const int32_t x = a[j], y = b[j];
      hits += (x >= 0 && x == y) ? 1 : 0;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) hits += __shfl_xor_sync(0xFFFFFFFFu, hits, d);
    if (lane == 0) out[p] = (double)hits / (double)k;
  }
}

// One CTA per row: FP64 tree sum of the registers, then (k - 1) / sum.
__global__ void cardinality_kernel(const double* __restrict__ y, int n_rows, int k, double* __restrict__ out) {
  __shared__ double part[EST_BLOCK / 32];
  for (int r = blockIdx.x; r < n_rows; r += gridDim.x) {
    const double* row = y + (int64_t)r * k;
    double s = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) s += row[j];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += part[q];
      out[r] = (double)(k - 1) / t;  // an unfilled register (inf) gives 0
    }
    __syncthreads();
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
  gm::jaccard_kernel<<<gm::grid_for(n_pairs, gm::EST_BLOCK / 32), gm::EST_BLOCK, 0, (cudaStream_t)stream>>>(
      s_a, s_b, n_pairs, k, out);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_cardinality(const double* y, int32_t n_rows, int32_t k, double* out, void* stream) {
  if (k < 2 || n_rows < 0) return GM_EINVAL;
  if (n_rows == 0) return GM_OK;
  if (!y || !out) return GM_EINVAL;
  gm::cardinality_kernel<<<gm::grid_for(n_rows, 1), gm::EST_BLOCK, 0, (cudaStream_t)stream>>>(y, n_rows, k, out);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_merge(const int32_t* s_a, const double* y_a, const int32_t* s_b, const double* y_b, int64_t n_regs,
                        int32_t* s_out, double* y_out, void* stream) {
  if (n_regs < 0) return GM_EINVAL;
  if (n_regs == 0) return GM_OK;
  if (!s_a || !y_a || !s_b || !y_b || !s_out || !y_out) return GM_EINVAL;
  gm::merge_kernel<<<gm::grid_for(n_regs, gm::EST_BLOCK), gm::EST_BLOCK, 0, (cudaStream_t)stream>>>(
      s_a, y_a, s_b, y_b, n_regs, s_out, y_out);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}
