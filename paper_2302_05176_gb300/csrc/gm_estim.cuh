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

// 128-bit unsigned accumulator (lo, hi).
struct Acc128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ void acc_add(Acc128& a, unsigned long long lo, unsigned long long hi) {
  const unsigned long long l = a.lo + lo;
  a.hi += hi + (l < lo ? 1ull : 0ull);
  a.lo = l;
}

// a >>= d (truncating), 0 <= d.
__device__ __forceinline__ void acc_shr(Acc128& a, int d) {
  if (d <= 0) return;
  if (d >= 128) {
    a.lo = a.hi = 0ull;
  } else if (d >= 64) {
    a.lo = a.hi >> (d - 64);
    a.hi = 0ull;
  } else {
    a.lo = (a.lo >> d) | (a.hi << (64 - d));
    a.hi >>= d;
  }
}

// The value acc 2^(e - 1135), rounded to the nearest double (ties to even); acc > 0.
__device__ __forceinline__ double acc_to_double(const Acc128& acc, int e) {
  const int lz = acc.hi ? __clzll((long long)acc.hi) : 64 + __clzll((long long)acc.lo);
  const int drop = (127 - lz) - 52;  // bits below the 53-bit significand
  unsigned long long mant, rh, rl;   // rh:rl: the dropped bits, left-aligned
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
  int e2 = e - 1135 + drop;  // exponent of the significand's lowest bit
  if (mant >> 53) {          // rounding carried into a new binade
    mant >>= 1;
    ++e2;
  }
  const int eb = e2 + 1075;  // biased exponent of the result
  return (eb >= 1 && eb <= 2046)
             ? __longlong_as_double((long long)(((unsigned long long)eb << 52) | (mant & 0x000FFFFFFFFFFFFFull)))
             : ldexp((double)mant, e2);
}

// Add the finite non-negative double with bits b to a lane's accumulator, kept in
// units of 2^(el - 1135) with el the largest biased exponent the lane has seen
// (the accumulator shifts right, truncating, when a larger one comes).  Each term
// is the 53-bit significand shifted to its place: below 2^113, so 128 terms per
// lane and 32 lanes fit in 125 bits.  No branch but the rare rescale.
__device__ __forceinline__ void lane_sum_term(Acc128& a, int& el, unsigned long long b) {
  const int ef = (int)(b >> 52);
  const int e = ef ? ef : 1;
  const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);  // 0 for +0
  if (e > el) {
    acc_shr(a, el ? e - el : 128);
    el = e;
  }
  const int s = 60 - (el - e);
  const int sl = s > 0 ? s : 0;
  const int sr = s < 0 ? (-s < 63 ? -s : 63) : 0;
  const unsigned long long mm = m >> sr;
  acc_add(a, mm << sl, sl ? (mm >> (64 - sl)) : 0ull);
}

// (k - 1) / sum_j y_j by one warp; every lane returns it.  The sum runs on the
// integer pipes, not the FP64 unit (whose add rate, not HBM, bounds an FP64 sum
// on GB300): lane l adds y[l], y[l + 32], ... (16-byte loads y[2j], y[2j+1] when
// the row is 16-byte aligned and k even) into a 128-bit fixed-point accumulator
// (lane_sum_term); the lanes align to the warp's largest exponent and add in a
// butterfly; the total is rounded to the nearest double once.  Terms more than
// 60 binades below the largest lose their low bits, so the result is within
// k 2^-60 of the correctly rounded sum, and the same bits on every call (the
// serving engine's query kernel uses this function too).  An unfilled register
// (+inf) gives 0.
__device__ __forceinline__ double warp_cardinality(const double* __restrict__ y, int k) {
  const int lane = threadIdx.x & 31;
  Acc128 acc{0ull, 0ull};
  int el = 0;
  unsigned long long bmax = 0ull;
  if ((k & 1) == 0 && (reinterpret_cast<uintptr_t>(y) & 15u) == 0) {
    const double2* y2 = reinterpret_cast<const double2*>(y);
#pragma unroll 4
    for (int j = lane; j < (k >> 1); j += 32) {
      const double2 v = __ldg(y2 + j);
      const unsigned long long p = (unsigned long long)__double_as_longlong(v.x);
      const unsigned long long q = (unsigned long long)__double_as_longlong(v.y);
      bmax = p > bmax ? p : bmax;
      bmax = q > bmax ? q : bmax;
      lane_sum_term(acc, el, p < 0x7FF0000000000000ull ? p : 0ull);
      lane_sum_term(acc, el, q < 0x7FF0000000000000ull ? q : 0ull);
    }
  } else {
#pragma unroll 4
    for (int j = lane; j < k; j += 32) {
      const unsigned long long p = (unsigned long long)__double_as_longlong(__ldg(y + j));
      bmax = p > bmax ? p : bmax;
      lane_sum_term(acc, el, p < 0x7FF0000000000000ull ? p : 0ull);
    }
  }
  int emax = el;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, bmax, d);
    bmax = o > bmax ? o : bmax;
    const int oe = __shfl_xor_sync(0xFFFFFFFFu, emax, d);
    emax = oe > emax ? oe : emax;
  }
  if (bmax >= 0x7FF0000000000000ull) return 0.0;  // an unfilled register (or a NaN)
  if (bmax == 0ull) return (double)(k - 1) / 0.0;
  acc_shr(acc, el ? emax - el : 128);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long lo = __shfl_xor_sync(0xFFFFFFFFu, acc.lo, d);
    const unsigned long long hi = __shfl_xor_sync(0xFFFFFFFFu, acc.hi, d);
    acc_add(acc, lo, hi);
  }
  return (double)(k - 1) / acc_to_double(acc, emax);
}

}  // namespace gm
