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

// 128-bit unsigned accumulator (lo, hi) for the cardinality sums below.
struct Acc128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ void acc_add(Acc128& a, unsigned long long lo, unsigned long long hi) {
  const unsigned long long l = a.lo + lo;
  a.hi += hi + (l < lo ? 1ull : 0ull);
  a.lo = l;
}

// Add the finite non-negative double with bits b to a, in units of 2^(emax - 1135)
// (emax: the largest biased exponent of the row): the 53-bit significand shifted
// left by 60 - (emax - e), or right (truncated) when that is negative.  Every term
// is below 2^113, so k <= 4096 terms fit in 125 bits.
__device__ __forceinline__ void acc_term(Acc128& a, unsigned long long b, int emax) {
  const int ef = (int)(b >> 52);
  if ((b << 1) == 0ull) return;  // +0
  const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
  const int sh = 60 - (emax - (ef ? ef : 1));  // place of the significand's lowest bit
  if (sh >= 64) {
    acc_add(a, 0ull, m << (sh - 64));
  } else if (sh > 0) {
    acc_add(a, m << sh, m >> (64 - sh));
  } else if (sh > -53) {
    acc_add(a, m >> (-sh), 0ull);
  }
}

// The accumulator's value, acc 2^(emax - 1135), rounded to the nearest double
// (ties to even).  acc > 0.
__device__ __forceinline__ double acc_to_double(const Acc128& acc, int emax) {
  // round (hi:lo) to 53 bits, ties to even; value = (hi:lo) 2^(emax - 1135)
  const int lz = acc.hi ? __clzll((long long)acc.hi) : 64 + __clzll((long long)acc.lo);
  const int drop = (127 - lz) - 52;  // bits below the 53-bit significand (the sum is >= 2^60 here)
  unsigned long long mant, rh, rl;    // rh:rl: the dropped bits, left-aligned
  if (drop <= 0) {
    mant = acc.lo << (-drop);
    rh = rl = 0ull;
  } else if (drop < 64) {
    mant = (acc.lo >> drop) | (acc.hi << (64 - drop));
    rh = acc.lo << (64 - drop);
    rl = 0ull;
  } else if (drop == 64) {
    mant = acc.hi;
    rh = acc.lo;
    rl = 0ull;
  } else {
    mant = acc.hi >> (drop - 64);
    rh = (acc.hi << (128 - drop)) | (acc.lo >> (drop - 64));
    rl = acc.lo << (128 - drop);
  }
  const bool rb = (rh >> 63) != 0ull;
  const bool sticky = ((rh << 1) | rl) != 0ull;
  mant += (rb && (sticky || (mant & 1ull))) ? 1ull : 0ull;
  int e2 = emax - 1135 + drop;  // exponent of the significand's lowest bit
  if (mant >> 53) {             // rounding carried into a new binade
    mant >>= 1;
    ++e2;
  }
  const int eb = e2 + 1075;  // biased exponent of the result
  const double sum = (eb >= 1 && eb <= 2046)
                         ? __longlong_as_double((long long)(((unsigned long long)eb << 52) | (mant & 0x000FFFFFFFFFFFFFull)))
                         : ldexp((double)mant, e2);
  return sum;
}

// (k - 1) / sum_j y_j by one warp; every lane returns it.  The sum is formed on
// the integer pipes, not the FP64 unit (whose add rate, not HBM, would bound the
// estimator on GB300): each lane adds its registers into a 128-bit fixed-point
// accumulator aligned to the row's largest exponent (16-byte loads when the row
// is 16-byte aligned and k is even), the lanes' accumulators are added in a
// butterfly, and the total is rounded to the nearest double once.  Terms more
// than 60 binades below the largest are truncated, so the result is the correctly
// rounded sum to within k 2^-60 relative, whatever the order: every call and the
// serving engine's query kernel give the same bits.  An unfilled register
// (+inf) gives 0.
__device__ __forceinline__ double warp_cardinality(const double* __restrict__ y, int k) {
  const int lane = threadIdx.x & 31;
  const bool vec = (k & 1) == 0 && (reinterpret_cast<uintptr_t>(y) & 15u) == 0;
  // pass 1: the largest biased exponent (bits compare like the values)
  unsigned long long bmax = 0ull;
  if (vec) {
    const double2* y2 = reinterpret_cast<const double2*>(y);
#pragma unroll 4
    for (int j = lane; j < (k >> 1); j += 32) {
      const double2 v = __ldg(y2 + j);
      const unsigned long long a = (unsigned long long)__double_as_longlong(v.x);
      const unsigned long long b = (unsigned long long)__double_as_longlong(v.y);
      bmax = a > bmax ? a : bmax;
      bmax = b > bmax ? b : bmax;
    }
  } else {
#pragma unroll 8
    for (int j = lane; j < k; j += 32) {
      const unsigned long long a = (unsigned long long)__double_as_longlong(__ldg(y + j));
      bmax = a > bmax ? a : bmax;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, bmax, d);
    bmax = o > bmax ? o : bmax;
  }
  if (bmax >= 0x7FF0000000000000ull) return 0.0;  // an unfilled register (or a NaN)
  if (bmax == 0ull) return (double)(k - 1) / 0.0;
  const int emax = (int)(bmax >> 52) ? (int)(bmax >> 52) : 1;
  // pass 2: the exact-aligned sum (the row is in L1 / L2 from pass 1)
  Acc128 acc{0ull, 0ull};
  if (vec) {
    const double2* y2 = reinterpret_cast<const double2*>(y);
#pragma unroll 4
    for (int j = lane; j < (k >> 1); j += 32) {
      const double2 v = __ldg(y2 + j);
      acc_term(acc, (unsigned long long)__double_as_longlong(v.x), emax);
      acc_term(acc, (unsigned long long)__double_as_longlong(v.y), emax);
    }
  } else {
#pragma unroll 8
    for (int j = lane; j < k; j += 32) acc_term(acc, (unsigned long long)__double_as_longlong(__ldg(y + j)), emax);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long lo = __shfl_xor_sync(0xFFFFFFFFu, acc.lo, d);
    const unsigned long long hi = __shfl_xor_sync(0xFFFFFFFFu, acc.hi, d);
    acc_add(acc, lo, hi);
  }
  return (double)(k - 1) / acc_to_double(acc, emax);
}


// The same estimates by one CTA of NT threads per row or pair (the batch kernels):
// thread t takes registers t, t + NT, ... (16-byte loads when aligned), so a row
// is read in one round trip; partial results meet in shared memory.  The integer
// hit count and the exactly aligned sum do not depend on the partition, so these
// give the same bits as the warp versions above.
template <int NT>
__device__ __forceinline__ double block_jaccard(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int k,
                                                int* red) {
  const int tid = threadIdx.x;
  int hits = 0;
  if ((k & 3) == 0 && ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u) == 0) {
    const int4* a4 = reinterpret_cast<const int4*>(a);
    const int4* b4 = reinterpret_cast<const int4*>(b);
#pragma unroll 4
    for (int j = tid; j < (k >> 2); j += NT) {
      const int4 x = __ldg(a4 + j), y = __ldg(b4 + j);
      hits += (x.x >= 0 && x.x == y.x) + (x.y >= 0 && x.y == y.y) + (x.z >= 0 && x.z == y.z) +
              (x.w >= 0 && x.w == y.w);
    }
  } else {
#pragma unroll 4
    for (int j = tid; j < k; j += NT) {
      const int32_t x = __ldg(a + j), y = __ldg(b + j);
      hits += (x >= 0 && x == y) ? 1 : 0;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) hits += __shfl_xor_sync(0xFFFFFFFFu, hits, d);
  if ((tid & 31) == 0) red[tid >> 5] = hits;
  __syncthreads();
  int total = 0;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) total += red[q];
  __syncthreads();
  return (double)total / (double)k;
}

template <int NT>
__device__ __forceinline__ double block_cardinality(const double* __restrict__ y, int k, unsigned long long* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool vec = (k & 1) == 0 && (reinterpret_cast<uintptr_t>(y) & 15u) == 0;
  const double2* y2 = reinterpret_cast<const double2*>(y);
  // pass 1: the largest bit pattern (bits compare like the values)
  unsigned long long bmax = 0ull;
  if (vec) {
#pragma unroll 4
    for (int j = tid; j < (k >> 1); j += NT) {
      const double2 v = __ldg(y2 + j);
      const unsigned long long p = (unsigned long long)__double_as_longlong(v.x);
      const unsigned long long q = (unsigned long long)__double_as_longlong(v.y);
      bmax = p > bmax ? p : bmax;
      bmax = q > bmax ? q : bmax;
    }
  } else {
#pragma unroll 4
    for (int j = tid; j < k; j += NT) {
      const unsigned long long p = (unsigned long long)__double_as_longlong(__ldg(y + j));
      bmax = p > bmax ? p : bmax;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, bmax, d);
    bmax = o > bmax ? o : bmax;
  }
  if (lane == 0) red[warp] = bmax;
  __syncthreads();
  bmax = 0ull;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) bmax = red[q] > bmax ? red[q] : bmax;
  __syncthreads();
  if (bmax >= 0x7FF0000000000000ull) return 0.0;  // an unfilled register (or a NaN)
  if (bmax == 0ull) return (double)(k - 1) / 0.0;
  const int emax = (int)(bmax >> 52) ? (int)(bmax >> 52) : 1;
  // pass 2: the aligned sum (the thread's own registers, from L1)
  Acc128 acc{0ull, 0ull};
  if (vec) {
#pragma unroll 4
    for (int j = tid; j < (k >> 1); j += NT) {
      const double2 v = __ldg(y2 + j);
      acc_term(acc, (unsigned long long)__double_as_longlong(v.x), emax);
      acc_term(acc, (unsigned long long)__double_as_longlong(v.y), emax);
    }
  } else {
#pragma unroll 4
    for (int j = tid; j < k; j += NT) acc_term(acc, (unsigned long long)__double_as_longlong(__ldg(y + j)), emax);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long lo = __shfl_xor_sync(0xFFFFFFFFu, acc.lo, d);
    const unsigned long long hi = __shfl_xor_sync(0xFFFFFFFFu, acc.hi, d);
    acc_add(acc, lo, hi);
  }
  if (lane == 0) {
    red[2 * warp] = acc.lo;
    red[2 * warp + 1] = acc.hi;
  }
  __syncthreads();
  Acc128 tot{0ull, 0ull};
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) acc_add(tot, red[2 * q], red[2 * q + 1]);
  __syncthreads();
  return (double)(k - 1) / acc_to_double(tot, emax);
}

}  // namespace gm
