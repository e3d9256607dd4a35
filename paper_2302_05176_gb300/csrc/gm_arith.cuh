// gm_arith.cuh -- FP64 results computed on GB300's integer pipes.
//
// GB300 runs FP64 at about 1/60 of its FP32 rate (measured: 6.3e11 DFMA/s; a
// warp's FP64 instruction costs the same with one active lane as with 32), and
// CUDA's FP64 log runs at 1.75e10/s.  The arrival recurrence needs, per arrival,
// one natural log and two products.  The logarithm below, in 64/128-bit integer
// arithmetic, runs at 1.2e11/s and is what the sketch uses; the products and the
// reciprocal are exact here too (bit-identical to the FP64 unit) and back the
// all-integer arithmetic (GM_FLAG_INT_PRODUCTS), while the default sends those
// to the otherwise idle FP64 unit:
//
//   neglog_u(w0, w1)  -ln(u) for u = (2m+1) 2^-53, m = top 52 bits of (w1:w0).
//                     Tang's table-driven method (ACM TOMS 16(4), 1990) in fixed
//                     point: f = 2^-L X in [1,2), 1 + r = f INV_j / 2^64 formed
//                     exactly (256 entries, |r| < 2^-9), ln(1+r) by a degree-7
//                     series to ~2^-70 (its tail in 32-bit products), the sum
//                     n ln2 - ln(INV_j^-1) - ln(1+r) in 128-bit fixed point, one
//                     final rounding.  For u within 2^-8 of 1 the series
//                     -ln(1-w) = w (1 + w/2 + ... + w^8/9) keeps full relative
//                     precision.  Measured: correctly rounded on 40,000 test
//                     inputs (max error 0.50000 ulp).
//   drcp_pos(v)       RN(1/v) for positive normal v: an FP32 seed, two Newton steps
//                     in 64-bit fixed point, then the exact remainder 2^116 - Q M
//                     fixes Q = floor(2^116 / M) and the sticky bit.  Bit-identical
//                     to the FP64 unit; subnormal results fall back to it.
//   dmul_pos(a, b)    RN(a b) for positive normal a, b: exact 106-bit product of
//                     the significands, one round-to-nearest-even.  Bit-identical
//                     to the FP64 unit; results outside the normal range fall back
//                     to the FP64 unit.
#pragma once
#include <cstdint>

#include "gm_log_tables.h"

namespace gm {

constexpr uint64_t MANT_MASK = 0x000FFFFFFFFFFFFFull;

// Round the positive integer (hi:lo) times 2^scale_exp to the nearest double,
// ties to even.  The result must be a normal double.
__device__ __forceinline__ double round_u128(uint64_t hi, uint64_t lo, int scale_exp) {
  int s;
  uint64_t H, L;
  if (hi) {
    s = __clzll((long long)hi);
    H = s ? ((hi << s) | (lo >> (64 - s))) : hi;
    L = lo << s;
  } else {
    s = 64 + __clzll((long long)lo);
    H = lo << (s - 64);
    L = 0ull;
  }
  const uint64_t mant = H >> 11;  // leading one at bit 52
  const uint64_t rbit = (H >> 10) & 1ull;
  const bool sticky = ((H & 0x3FFull) != 0ull) || (L != 0ull);
  // value = mant * 2^(127 - s - 52 + scale_exp); biased exponent = that + 1075
  const int64_t be = 127 - s - 52 + scale_exp + 1075;
  uint64_t bits = ((uint64_t)(be - 1) << 52) + mant;
  bits += (rbit && (sticky || (mant & 1ull))) ? 1ull : 0ull;
  return __longlong_as_double((long long)bits);
}

// A real call, not inlined: the fused sketch kernel streams arrivals from four
// places, and one copy of this body instead of four keeps the kernel's code in
// the instruction cache (measured: 4 % faster despite the call's spills).
#ifdef GM_INLINE_LOG
__device__ __forceinline__ double neglog_u(uint32_t w0, uint32_t w1) {
#else
static __device__ __noinline__ double neglog_u(uint32_t w0, uint32_t w1) {
#endif
  const uint64_t x = ((uint64_t)w1 << 32) | (uint64_t)w0;
  const uint64_t X = ((x >> 12) << 1) | 1ull;  // u = X 2^-53, X odd < 2^53
  constexpr uint64_t NEAR_ONE = (1ull << 53) - (1ull << 45);
  if (X >= NEAR_ONE) {
    // u = 1 - w, w = W 2^-53 <= 2^-8:  -ln u = w P(w), P at scale 2^63
    const uint64_t W = (1ull << 53) - X;
    const uint64_t Wq = W << 11;  // w 2^64
    uint64_t p = LOG1M_P[8];
#pragma unroll
    for (int i = 7; i >= 0; --i) p = LOG1M_P[i] + __umul64hi(p, Wq);
    return round_u128(__umul64hi(W, p), W * p, -116);
  }
  const int L = 63 - __clzll((long long)X);
  const uint64_t f64 = X << (63 - L);  // f 2^63, f in [1, 2)
  const int j = (int)((f64 >> 55) & 255ull);
  const uint64_t inv = __ldg(&LOG_INV[j]);
  const uint64_t ph = __umul64hi(f64, inv), pl = f64 * inv;  // (1 + r) 2^127, exact
  const int64_t dh = (int64_t)(ph - 0x8000000000000000ull);   // high word of r 2^127
  const int64_t R = (int64_t)(((uint64_t)dh << 9) | (pl >> 55));  // r 2^72, |r| < 2^-9
  // ln(1 + r) = r - r^2/2 + r^3 B,  B = 1/3 - r/4 + r^2 q,  q = 1/5 - r/6 + r^2/7;
  // the terms of B need ~26 significant bits, so q and r^2 q use 32-bit products
  const int64_t r2 = __mul64hi(R, R);    // r^2 2^80
  const int64_t r3 = __mul64hi(r2, R);   // r^3 2^88
  const int32_t R32 = (int32_t)(R >> 32);    // r 2^40
  const int32_t r2h = (int32_t)(r2 >> 32);   // r^2 2^48
  const int32_t q = LOG_C5 - (int32_t)(((int64_t)R32 * LOG_C6) >> 40) + (int32_t)(((int64_t)r2h * LOG_C7) >> 48);
  const int64_t B = LOG_C3 - (R >> 12) + (((int64_t)r2h * (int64_t)q) >> 17);  // 2^-62
  const int64_t r3B = __mul64hi(r3, B);  // r^3 B 2^86
  const int64_t poly = R - (r2 >> 9) + (r3B >> 14);  // ln(1 + r) 2^72
  const uint64_t n = (uint64_t)(53 - L);
  // E = n ln2 - LNF_j - poly 2^48, at scale 2^-120
  uint64_t tl = LN2_120_LO * n;
  uint64_t th = __umul64hi(LN2_120_LO, n) + LN2_120_HI * n;
  const uint64_t fl = __ldg(&LOG_LNF_LO[j]), fh = __ldg(&LOG_LNF_HI[j]);
  const uint64_t pl48 = (uint64_t)poly << 48;
  const uint64_t ph48 = (uint64_t)(poly >> 16);
  asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(tl), "+l"(th) : "l"(fl), "l"(fh));
  asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(tl), "+l"(th) : "l"(pl48), "l"(ph48));
  return round_u128(th, tl, -120);
}

// Significand product of positive normal a, b, normalised so that the leading
// one is bit 63 of hi; `top` = 1 when the product's leading one was bit 127.
__device__ __forceinline__ void sig_product(uint64_t ab, uint64_t bb, uint64_t& hi, bool& sticky_lo, int& top) {
  const uint64_t A = ((ab & MANT_MASK) | (1ull << 52)) << 11;  // [2^63, 2^64)
  const uint64_t B = ((bb & MANT_MASK) | (1ull << 52)) << 11;
  hi = __umul64hi(A, B);
  uint64_t lo = A * B;  // A B in [2^126, 2^128)
  top = (int)(hi >> 63);
  if (!top) {
    hi = (hi << 1) | (lo >> 63);
    lo <<= 1;
  }
  sticky_lo = lo != 0ull;
}

// RN(a b) for positive normal a, b whose product is normal (no range check).
__device__ __forceinline__ double dmul_normal(double a, double b) {
  const uint64_t ab = (uint64_t)__double_as_longlong(a), bb = (uint64_t)__double_as_longlong(b);
  uint64_t hi;
  bool sl;
  int top;
  sig_product(ab, bb, hi, sl, top);
  const int be = (int)(ab >> 52) + (int)(bb >> 52) - 1023 + top;  // biased exponent of the result
  const uint64_t mant = hi >> 11;
  const bool up = ((hi >> 10) & 1ull) && (((hi & 0x3FFull) != 0ull) || sl || (mant & 1ull));
  return __longlong_as_double((long long)((((uint64_t)(be - 1)) << 52) + mant + (up ? 1ull : 0ull)));
}

// RN(a b) for positive normal a, b; results outside the normal range on the FP64 unit.
__device__ __forceinline__ double dmul_pos(double a, double b) {
  const uint64_t ab = (uint64_t)__double_as_longlong(a), bb = (uint64_t)__double_as_longlong(b);
  const int ea = (int)(ab >> 52), eb = (int)(bb >> 52);
  const int be0 = ea + eb - 1023;  // the result's biased exponent is be0 or be0 + 1
  if (ea == 0 || eb == 0 || be0 < 1 || be0 > 2044) return __dmul_rn(a, b);
  return dmul_normal(a, b);
}

__device__ __forceinline__ double drcp_pos(double v) {
  const uint64_t vb = (uint64_t)__double_as_longlong(v);
  const int ev = (int)(vb >> 52);
  const uint64_t frac = vb & MANT_MASK;
  if (ev == 0 || ev >= 2045) return __drcp_rn(v);
  if (frac == 0ull) return __longlong_as_double((long long)((uint64_t)(2046 - ev) << 52));
  const uint64_t M = frac | (1ull << 52);
  const uint64_t d = M << 11;  // [2^63, 2^64)
  // seed y ~ 2^127 / d from an FP32 reciprocal of the top 24 bits (exact float)
  const float r0 = __frcp_rn((float)(uint32_t)(d >> 40));
  const uint32_t rb = (uint32_t)__float_as_int(r0);
  const uint64_t rm = (uint64_t)((rb & 0x7FFFFFu) | 0x800000u);
  const int sh = (int)((rb >> 23) & 0xFF) - 127 - 23 + 87;
  uint64_t y = sh >= 0 ? (rm << sh) : (rm >> (-sh));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    // eps = 1 - d y / 2^127, kept as eps 2^85 = (2^127 - d y) >> 42
    const uint64_t dh = __umul64hi(d, y), dl = d * y;
    uint64_t el = 0ull - dl;
    uint64_t eh = 0x8000000000000000ull - dh - (dl != 0ull ? 1ull : 0ull);
    const int64_t E64 = (int64_t)((eh << 22) | (el >> 42));
    // y += (y eps 2^21) >> 21, the product taken as signed
    const int64_t corr = (int64_t)__umul64hi(y, (uint64_t)E64) - (E64 < 0 ? (int64_t)y : 0ll);
    y += (uint64_t)(corr >> 21);
  }
  // Q = floor(2^116 / M) exactly, from the remainder
  uint64_t Q = y;
  int64_t rem;  // 2^116 - Q M, |.| < 2^63
  {
    const uint64_t ql = Q * M;
    rem = (int64_t)(0ull - ql);  // low 64 bits of 2^116 - Q M: 2^116 has none
  }
  int guard = 0;
  while (rem < 0 && guard < 4) { --Q; rem += (int64_t)M; ++guard; }
  while (rem >= (int64_t)M && guard < 8) { ++Q; rem -= (int64_t)M; ++guard; }
  if (guard >= 4 || (Q >> 63) == 0ull) return __drcp_rn(v);
  const uint64_t mant = Q >> 11;
  const uint64_t rbit = (Q >> 10) & 1ull;
  const bool sticky = ((Q & 0x3FFull) != 0ull) || (rem != 0);
  uint64_t bits = ((uint64_t)(2044 - ev) << 52) + mant;
  bits += (rbit && (sticky || (mant & 1ull))) ? 1ull : 0ull;
  return __longlong_as_double((long long)bits);
}

}  // namespace gm
