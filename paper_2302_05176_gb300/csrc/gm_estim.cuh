// gm_estim.cuh -- per-row estimator reductions over finished sketches (Sec. 1:
// the weighted Jaccard estimate from register collisions; Sec. 2.4: the
// cardinality estimate (k - 1) / sum_j y_j).  Shared by the batch estimators and
// the serving engine's query kernel, so both give the same bits.
#pragma once
#include <cstdint>

namespace gm {

constexpr int EST_BLOCK = 256;  // threads per CTA of the estimator kernels (8 warps)

// Fraction of registers where both sketches hold the same element (one warp).
// 16-byte loads when both rows are 16-byte aligned and k % 4 == 0, four in
// flight per lane; the count is an integer, so the path does not change it.
__device__ __forceinline__ double warp_jaccard(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int k) {
  const int lane = threadIdx.x & 31;
  int hits = 0;
  if ((k & 3) == 0 && ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u) == 0) {
    const int4* a4 = reinterpret_cast<const int4*>(a);
    const int4* b4 = reinterpret_cast<const int4*>(b);
    const int k4 = k >> 2;
#pragma unroll 4
    for (int j = lane; j < k4; j += 32) {
      const int4 x = __ldg(a4 + j), y = __ldg(b4 + j);
      hits += (x.x >= 0 && x.x == y.x) + (x.y >= 0 && x.y == y.y) + (x.z >= 0 && x.z == y.z) +
              (x.w >= 0 && x.w == y.w);
    }
  } else {
#pragma unroll 4
    for (int j = lane; j < k; j += 32) {
      const int32_t x = __ldg(a + j), y = __ldg(b + j);
      hits += (x >= 0 && x == y) ? 1 : 0;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) hits += __shfl_xor_sync(0xFFFFFFFFu, hits, d);
  return (double)hits / (double)k;
}

// (k - 1) / sum_j y_j by one warp; every lane returns it.  When the row is 16-byte
// aligned and k is even, lane l adds the pairs (y[2j], y[2j+1]) for j = l, l + 32,
// ... into four partial sums (j = l + 64 m and l + 64 m + 32 alternate between two
// pairs of them), so four FP64 add chains run at once and eight 16-byte loads
// are in flight; else y[l], y[l + 32], ... into one sum.  Then the partials in a
// fixed order and a butterfly over the lanes: the same bits on every call.  An
// unfilled register (+inf) gives 0.
__device__ __forceinline__ double warp_cardinality(const double* __restrict__ y, int k) {
  const int lane = threadIdx.x & 31;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if ((k & 1) == 0 && (reinterpret_cast<uintptr_t>(y) & 15u) == 0) {
    const double2* y2 = reinterpret_cast<const double2*>(y);
    const int k2 = k >> 1;
#pragma unroll 4
    for (int j = lane; j < k2; j += 64) {
      const double2 v = __ldg(y2 + j);
      double2 u = make_double2(0.0, 0.0);
      if (j + 32 < k2) u = __ldg(y2 + j + 32);
      s0 += v.x;
      s1 += v.y;
      s2 += u.x;
      s3 += u.y;
    }
  } else {
#pragma unroll 8
    for (int j = lane; j < k; j += 32) s0 += __ldg(y + j);
  }
  double s = (s0 + s1) + (s2 + s3);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  return (double)(k - 1) / s;
}

}  // namespace gm
