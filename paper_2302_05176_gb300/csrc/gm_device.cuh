// gm_device.cuh -- device building blocks of the GB300 Gumbel-Max sketch.
//
// Arithmetic of one arrival (Sec. 2.2, Eq. biz_dis / Eq. biz_biz-1, with the
// rounding reading stated in include/gm.h):
//   u   = (2m + 1) 2^-53 from the top 52 bits of Philox words 0,1
//   E   = RN(-ln u)
//   t_z = RN(E * C_z),   C_z = RN(1 / (k - z))
//   S_z = RN(exact sum of t_0..t_z)     -- a 128-bit fixed-point accumulator
//   b_z = RN(S_z * R),   R = RN(1 / v)
// The exact sum makes S_z independent of the order in which the terms are
// added, so a warp can form 32 consecutive prefix sums with a shuffle scan and
// get the same bits as a sequential loop.
#pragma once
#include <cstdint>

#include "gm.h"

namespace gm {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint64_t INF_BITS = 0x7FF0000000000000ull;   // +inf: an unfilled register
constexpr uint64_t UNFILLED_ID = 0xFFFFFFFFFFFFFFFFull;  // larger than every id
constexpr uint64_t DBL_MAX_BITS = 0x7FEFFFFFFFFFFFFFull;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter (c0, c1, 0, 0),
// key (k0, k1); ten rounds, Weyl key schedule.
// ---------------------------------------------------------------------------
struct Words {
  uint32_t w0, w1, w2, w3;
};

__device__ __forceinline__ Words philox(uint32_t c0, uint32_t c1, uint32_t k0, uint32_t k1) {
  uint32_t c2 = 0u, c3 = 0u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return Words{c0, c1, c2, c3};
}

// u = (2m+1) 2^-53 with m the top 52 bits of (w1:w0), built from integer ops only
// (an int->double conversion would run on the slow FP64 pipe).
__device__ __forceinline__ double uniform_open(uint32_t w0, uint32_t w1) {
  const uint64_t x = ((uint64_t)w1 << 32) | (uint64_t)w0;
  const uint64_t X = ((x >> 12) << 1) | 1ull;  // odd, < 2^53
  const int lz = __clzll((long long)X);        // 11 .. 63
  const uint64_t mant = X << (lz - 11);        // leading one at bit 52
  const uint64_t bits = ((uint64_t)(1032 - lz) << 52) + mant;
  return __longlong_as_double((long long)bits);
}

// RandInt(z, k): z + floor(r (k - z) / 2^64), r = (w3:w2).
__device__ __forceinline__ int randint(uint32_t w2, uint32_t w3, int z, int k) {
  const uint64_t r = ((uint64_t)w3 << 32) | (uint64_t)w2;
  return z + (int)__umul64hi(r, (uint64_t)(k - z));
}

// ---------------------------------------------------------------------------
// 128-bit unsigned fixed point, value = w0 2^-118 + w1 2^-54.
// For k <= 4096 every term t_z = RN(E C_z) lies in [2^-65, 2^6) (E >= 2^-53,
// E <= 53 ln 2 < 36.74, C_z >= 2^-12), so its lowest mantissa bit is >= 2^-117,
// and every prefix sum is below 36.74 H_4096 < 327 < 2^9: the 128 bits hold each
// prefix sum exactly.
// ---------------------------------------------------------------------------
static_assert(GM_MAX_K <= 4096, "the 128-bit prefix-sum accumulator is exact only for k <= 4096");

struct Fix {
  uint64_t w0, w1;
};

__device__ __forceinline__ Fix fix_zero() { return Fix{0ull, 0ull}; }

// Exact conversion of a positive normal double in [2^-65, 2^10).
__device__ __forceinline__ Fix fix_from(double t) {
  const uint64_t bits = (uint64_t)__double_as_longlong(t);
  const int e = (int)(bits >> 52);
  const uint64_t M = (bits & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
  const int off = e - 957;  // bit index of M's lowest bit: (e - 1075) + 118, >= 1
  Fix f;
  if (off < 64) {
    f.w0 = M << off;
    f.w1 = M >> (64 - off);
  } else {
    f.w0 = 0ull;
    f.w1 = M << (off - 64);
  }
  return f;
}

__device__ __forceinline__ void fix_add(Fix& a, const Fix& b) {
  asm("add.cc.u64 %0, %0, %2;\n\t"
      "addc.u64 %1, %1, %3;"
      : "+l"(a.w0), "+l"(a.w1)
      : "l"(b.w0), "l"(b.w1));
}

// Round a positive fixed-point value (>= 2^-65) to the nearest double, ties to even.
__device__ __forceinline__ double fix_round(const Fix& a) {
  uint64_t hi, lo;
  int base;
  if (a.w1) {
    hi = a.w1; lo = a.w0; base = 64;
  } else {
    hi = a.w0; lo = 0ull; base = 0;
  }
  const int s = __clzll((long long)hi);
  const uint64_t H = s ? ((hi << s) | (lo >> (64 - s))) : hi;
  const uint64_t L = lo << s;
  const int p = base + 63 - s;  // index of the leading one, in units of 2^-118
  const uint64_t mant = H >> 11;
  const uint64_t rbit = (H >> 10) & 1ull;
  const bool sticky = ((H & 0x3FFull) != 0ull) || (L != 0ull);
  uint64_t bits = ((uint64_t)(p + 904) << 52) + mant;  // mant carries the implicit one
  bits += (rbit && (sticky || (mant & 1ull))) ? 1ull : 0ull;
  return __longlong_as_double((long long)bits);
}

// ---------------------------------------------------------------------------
// Registers: 16-byte (y bits, id) pairs in shared memory, updated by a 128-bit
// compare-and-swap to the lexicographic minimum (ties -> smaller id).
// ---------------------------------------------------------------------------
struct alignas(16) Reg {
  unsigned long long y;
  unsigned long long id;
};

__device__ __forceinline__ void cas128_shared(uint32_t saddr, uint64_t ey, uint64_t eid, uint64_t ny,
                                              uint64_t nid, uint64_t& oy, uint64_t& oid) {
  asm volatile(
      "{\n\t.reg .b128 d, cmp, nv;\n\t"
      "mov.b128 cmp, {%2, %3};\n\t"
      "mov.b128 nv, {%4, %5};\n\t"
      "atom.shared.cas.b128 d, [%6], cmp, nv;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(oy), "=l"(oid)
      : "l"(ey), "l"(eid), "l"(ny), "l"(nid), "r"(saddr)
      : "memory");
}

__device__ __forceinline__ void ld_shared_v2(uint32_t saddr, uint64_t& a, uint64_t& b) {
  asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(saddr) : "memory");
}

// Lower register at saddr to (yb, id) if that is smaller.  Lock-free: each failed
// CAS means another thread lowered the register, which can happen only finitely
// often; the cap only guards against a broken invariant.  Returns retries.
constexpr int CAS_CAP = 1 << 16;
__device__ __forceinline__ int reg_lower(uint32_t saddr, uint64_t yb, uint64_t id, bool& gave_up) {
  uint64_t cy, cid;
  ld_shared_v2(saddr, cy, cid);
  int tries = 0;
  while (yb < cy || (yb == cy && id < cid)) {
    uint64_t oy, oid;
    cas128_shared(saddr, cy, cid, yb, id, oy, oid);
    if (oy == cy && oid == cid) break;
    cy = oy;
    cid = oid;
    if (++tries >= CAS_CAP) {
      gave_up = true;
      break;
    }
  }
  return tries;
}

// A cheap, truncating FP32 copy of a non-negative double, from its bits only
// (a double->float conversion runs on the FP64 pipe).  Used for bounds and
// work estimates, never for a register value.
__device__ __forceinline__ float f32_trunc(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -126) return 0.0f;
  if (e > 127) return 3.0e38f;
  const uint32_t fb = ((uint32_t)(e + 127) << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu);
  return __int_as_float((int)fb);
}

// Exact widening of a positive normal float to double, from bits.
__device__ __forceinline__ double f64_from_f32(float f) {
  const uint32_t b = (uint32_t)__float_as_int(f);
  const uint64_t e = (uint64_t)((b >> 23) & 0xFF) + (1023 - 127);
  const uint64_t bits = (e << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

}  // namespace gm
