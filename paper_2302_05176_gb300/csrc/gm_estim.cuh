// gm_estim.cuh -- per-row estimator reductions over finished sketches (Sec. 1:
// the weighted Jaccard estimate from register collisions; Sec. 2.4: the
// cardinality estimate (k - 1) / sum_j y_j).  Shared by the batch estimators and
// the serving engine's query kernel, so both give the same bits.
#pragma once
#include <cstdint>

namespace gm {

constexpr int EST_BLOCK = 256;  // threads of a cardinality reduction (fixes its summation order)

// Fraction of registers where both sketches hold the same element (one warp).
__device__ __forceinline__ double warp_jaccard(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int k) {
  const int lane = threadIdx.x & 31;
  int hits = 0;
  for (int j = lane; j < k; j += 32) {
    const int32_t x = a[j], y = b[j];
    hits += (x >= 0 && x == y) ? 1 : 0;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) hits += __shfl_xor_sync(0xFFFFFFFFu, hits, d);
  return (double)hits / (double)k;
}

// (k - 1) / sum_j y_j by a block of EST_BLOCK threads: strided partial sums, a
// butterfly per warp, then the warps in order.  part: EST_BLOCK / 32 shared
// doubles.  The result is valid in thread 0; an unfilled register (+inf) gives 0.
__device__ __forceinline__ double block_cardinality(const double* __restrict__ y, int k, double* part) {
  double s = 0.0;
  for (int j = threadIdx.x; j < k; j += EST_BLOCK) s += y[j];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < EST_BLOCK / 32; ++q) t += part[q];
  __syncthreads();
  return (double)(k - 1) / t;
}

}  // namespace gm
