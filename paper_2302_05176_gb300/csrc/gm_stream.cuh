// gm_stream.cuh -- the arrival stream of one element on the device (Sec. 2.2,
// Eq. biz_dis / Eq. biz_biz-1 and the Fisher-Yates server assignment), shared by
// the sketch kernels and the diagnostic kernels.
#pragma once
#include <cstdint>

#include "gm_arith.cuh"
#include "gm_device.cuh"

namespace gm {

// Arithmetic of an arrival.  ARITH_MIX (the default) takes -ln u from the integer
// pipes (gm_arith.cuh) and the products and 1/v from the FP64 unit, which is
// otherwise idle; ARITH_INT computes the products and 1/v on the integer pipes
// too; ARITH_FP64 uses the FP64 unit throughout (CUDA's log).  Products and
// reciprocals are bit-identical in all three; the logarithms of ARITH_FP64
// differ from the other two by at most an ulp.
constexpr int ARITH_FP64 = 0;
constexpr int ARITH_INT = 1;
constexpr int ARITH_MIX = 2;

template <int ARITH>
__device__ __forceinline__ double arr_neglog(const Words& wd) {
  if constexpr (ARITH != ARITH_FP64)
    return neglog_u(wd.w0, wd.w1);
  else
    return -log(uniform_open(wd.w0, wd.w1));
}
template <int ARITH>
__device__ __forceinline__ double arr_mul(double a, double b) {
  if constexpr (ARITH == ARITH_INT)
    return dmul_pos(a, b);
  else
    return __dmul_rn(a, b);
}
// t = RN(E C): E in [2^-53, 36.74], C in [2^-12, 1], the product always normal
template <int ARITH>
__device__ __forceinline__ double arr_mul_t(double e, double c) {
  if constexpr (ARITH == ARITH_INT)
    return dmul_normal(e, c);
  else
    return __dmul_rn(e, c);
}
template <int ARITH>
__device__ __forceinline__ double arr_rcp(double v) {
  if constexpr (ARITH == ARITH_INT)
    return drcp_pos(v);
  else
    return __drcp_rn(v);
}

// Conservative FP32 screen of a first arrival (Sec. 2.2, FastPrune's stop rule
// applied before any FP64 work).  b_0 = RN(RN(E RN(1/k)) RN(1/v)) with
// E = RN(-ln u) is at least E/(k v) (1 - 2^-50), so b_0 > T whenever
// u < exp(-T k v (1 + 2^-49)).  With v_f the truncated FP32 copy of v (relative
// error < 2^-23 when v_f is a normal float) and T exactly representable in FP32,
// x_f = fl(fl(v_f T) k) >= T k v (1 - 2^-22) as long as v_f T is a normal float;
// the argument is widened by 2^-18 and the result shrunk by 2^-19 to cover fl
// rounding and __expf's error, and u <= (w1 + 1) 2^-32.  Outside that range (v_f
// or v_f T not normal) the screen does not decide.  It only ever skips elements
// whose first arrival exceeds T.
__device__ __forceinline__ bool screen_out(uint32_t w1, float vf, float Tf, float kf) {
  if (!(vf >= 1.17549435e-38f && vf <= 1.0e38f)) return false;
  const float vt = vf * Tf;
  if (!(vt >= 1.0e-30f)) return false;  // also false for NaN
  const float thr = __expf(-(vt * kf) * (1.0f + 0x1p-18f)) * (1.0f - 0x1p-19f);
  const uint32_t thr_i = (uint32_t)(thr * 4294967296.0f);  // floor, thr < 1
  return w1 < thr_i;
}

// --------------------------------------------------------------------------
// SW consecutive arrivals z0 .. z0+SW-1 of one element per SW-lane segment of the
// warp (SW = 8 or 32), one per lane: returns the lane's arrival time (bits; all
// ones when the lane has no arrival) and RandInt target; `carry` (the exact
// prefix sum before z0, the same in every lane of the segment) is advanced past
// the batch.  `act`: the segment streams an element.
// --------------------------------------------------------------------------
// One arrival's term t_z = RN(E C_z) as a fixed-point value and its RandInt target.
template <int ARITH>
__device__ __forceinline__ Fix arrival_term(int32_t id, int z, int k, uint32_t key0, uint32_t key1, const double* __restrict__ ctab, int& J) {
  const Words wd = philox((uint32_t)id, (uint32_t)z, key0, key1);
  J = randint(wd.w2, wd.w3, z, k);
  return fix_from(arr_mul_t<ARITH>(arr_neglog<ARITH>(wd), __ldg(ctab + z)));
}

template <int ARITH, int SW>
__device__ __forceinline__ uint64_t seg_batch(bool act, int32_t id, double R, int z0, int k, uint32_t key0,
                                              uint32_t key1, const double* __restrict__ ctab, Fix& carry, int lane,
                                              int& J) {
  const int sl = lane & (SW - 1);
  const int z = z0 + sl;
  Fix f = fix_zero();
  J = z;
  const bool valid = act && z < k;
  if (valid) f = arrival_term<ARITH>(id, z, k, key0, key1, ctab, J);
#pragma unroll
  for (int d = 1; d < SW; d <<= 1) {
    Fix g;
    g.w0 = __shfl_up_sync(FULL, f.w0, d, SW);
    g.w1 = __shfl_up_sync(FULL, f.w1, d, SW);
    if (sl >= d) fix_add(f, g);
  }
  fix_add(f, carry);
  carry.w0 = __shfl_sync(FULL, f.w0, SW - 1, SW);
  carry.w1 = __shfl_sync(FULL, f.w1, SW - 1, SW);
  return valid ? (uint64_t)__double_as_longlong(arr_mul<ARITH>(fix_round(f), R)) : ~0ull;
}

template <int ARITH>
__device__ __forceinline__ uint64_t warp_batch(int32_t id, double R, int z0, int k, uint32_t key0, uint32_t key1,
                                               const double* __restrict__ ctab, Fix& carry, int lane, int& J) {
  return seg_batch<ARITH, 32>(true, id, R, z0, k, key0, key1, ctab, carry, lane, J);
}

// ---------------------------------------------------------------------------
// The element's Fisher-Yates permutation pi, two storage policies:
//   DensePi:    k u16 entries (pi[j] = j initially) -- long streams;
//   HashPiN<S>: the displaced positions only, in an S-slot open-addressing table
//               of (position << 16 | value) words -- streams of up to ~3S/4
//               steps, 4S bytes instead of 2k.
// ---------------------------------------------------------------------------
struct DensePi {
  uint16_t* a;
  static uint16_t* member_type();
  __device__ __forceinline__ uint32_t get(int p) const { return a[p]; }
  __device__ __forceinline__ void put(int p, uint32_t v) const { a[p] = (uint16_t)v; }
  // pi[j] = j for j < k by the sw lanes of a segment, eight entries per 16-byte
  // store; the caller synchronises the warp afterwards.
  __device__ __forceinline__ void reset_seg(int k, int sl, int sw) const {
    const int k8 = k & ~7;
    for (int j = sl * 8; j < k8; j += 8 * sw) {
      uint4 q;
      q.x = (uint32_t)j | ((uint32_t)(j + 1) << 16);
      q.y = (uint32_t)(j + 2) | ((uint32_t)(j + 3) << 16);
      q.z = (uint32_t)(j + 4) | ((uint32_t)(j + 5) << 16);
      q.w = (uint32_t)(j + 6) | ((uint32_t)(j + 7) << 16);
      *reinterpret_cast<uint4*>(a + j) = q;
    }
    for (int j = k8 + sl; j < k; j += sw) a[j] = (uint16_t)j;
  }
  __device__ __forceinline__ void reset(int k, int lane) const {
    reset_seg(k, lane, 32);
    __syncwarp();
  }
};

constexpr uint32_t HASH_EMPTY = 0xFFFFFFFFu;

template <int SLOTS>
struct HashPiN {
  uint32_t* tab;
  static uint32_t* member_type();
  static constexpr int BITS = SLOTS == 512 ? 9 : (SLOTS == 256 ? 8 : (SLOTS == 128 ? 7 : 6));
  static_assert(SLOTS == 64 || SLOTS == 128 || SLOTS == 256 || SLOTS == 512, "hash size");
  __device__ __forceinline__ static uint32_t slot(uint32_t p) { return (p * 0x9E3779B1u) >> (32 - BITS); }
  __device__ __forceinline__ uint32_t get(int p) const {
    uint32_t s = slot((uint32_t)p);
    for (int probe = 0; probe < SLOTS; ++probe) {
      const uint32_t e = tab[s];
      if (e == HASH_EMPTY) break;
      if ((e >> 16) == (uint32_t)p) return e & 0xFFFFu;
      s = (s + 1u) & (SLOTS - 1);
    }
    return (uint32_t)p;
  }
  __device__ __forceinline__ void put(int p, uint32_t v) const {
    uint32_t s = slot((uint32_t)p);
    const uint32_t ent = ((uint32_t)p << 16) | v;
    for (int probe = 0; probe < SLOTS; ++probe) {
      uint32_t e = tab[s];
      if (e == HASH_EMPTY) {
        e = atomicCAS(&tab[s], HASH_EMPTY, ent);  // another lane may claim the slot first
        if (e == HASH_EMPTY) return;
      }
      if ((e >> 16) == (uint32_t)p) {  // only one lane writes a given position per step
        tab[s] = ent;
        return;
      }
      s = (s + 1u) & (SLOTS - 1);
    }
  }
  // Clear the table with the sw lanes of a segment (sl: lane within it); the
  // caller synchronises the warp afterwards.
  __device__ __forceinline__ void reset_seg(int, int sl, int sw) const {
    uint4* t4 = reinterpret_cast<uint4*>(tab);
    for (int j = sl; j < SLOTS / 4; j += sw) t4[j] = make_uint4(HASH_EMPTY, HASH_EMPTY, HASH_EMPTY, HASH_EMPTY);
  }
  __device__ __forceinline__ void reset(int k, int lane) const {
    reset_seg(k, lane, 32);
    __syncwarp();
  }
};
constexpr int HASH_SLOTS = 512;     // per warp (32-lane segments)
constexpr int HASH_MAX_FILL = 384;  // more displaced positions: the stream moves to a DensePi
using HashPi = HashPiN<HASH_SLOTS>;

// Fisher-Yates steps z0 .. z0+n-1 (n <= SW) on each segment's pi, all segments at
// once; lane l < n of a segment holds J_l (>= z0 + l) and gets the server of
// step z0 + l, exactly as the steps would give in order:
//   a_l = value at position z0+l when step l runs = a_m of the latest earlier lane
//         m that swapped its value into z0+l (J_m = z0+l), else pi[z0+l];
//   c_l = value at J_l when step l runs = a_m of the latest earlier lane m with
//         J_m = J_l, else pi[J_l].
// Chains of a_l are resolved by pointer jumping (log2 SW shuffle rounds);
// afterwards the last lane of each J group stores its a_l at J (positions inside
// the batch window are final and need no store).  n, z0 and pi are per segment.
// Returns the number of stores of the lane's segment.
template <int SW, class PI>
__device__ __forceinline__ int seg_fy_steps(const PI& pi, int z0, int J, int n, int lane, int& c_out) {
  constexpr uint32_t SEGM = SW == 32 ? 0xFFFFFFFFu : ((1u << SW) - 1u);
  const int sl = lane & (SW - 1), base = lane & ~(SW - 1);
  const uint32_t segmask = SEGM << base;
  const bool act = sl < n;
  const uint32_t lt = lanemask_lt();
  const int tgt = (act && (uint32_t)(J - z0) < (uint32_t)SW && J != z0 + sl) ? base + (J - z0) : -1;
  uint32_t W = __ballot_sync(FULL, tgt >= 0);
  uint32_t src_mask = 0u;
  while (W) {  // lanes whose J falls on a later lane's position inside this batch
    const int m = __ffs(W) - 1;
    W &= W - 1u;
    const int t = __shfl_sync(FULL, tgt, m);
    if (lane == t) src_mask |= 1u << m;
  }
  if (!act) src_mask = 0u;
  int src = 31 - __clz(src_mask & lt);  // -1: none
  uint32_t val = act ? pi.get(z0 + sl) : 0u;
#pragma unroll
  for (int r = 0; (1 << r) < SW; ++r) {
    const int from = src < 0 ? lane : src;
    const uint32_t v2 = __shfl_sync(FULL, val, from);
    const int s2 = __shfl_sync(FULL, src, from);
    if (src >= 0) {
      val = v2;
      src = s2;
    }
  }
  const uint32_t same = __match_any_sync(FULL, act ? (int)(((uint32_t)base << 16) | (uint32_t)J) : -1 - lane);
  const int pt = 31 - __clz(same & lt);
  const uint32_t a_pt = __shfl_sync(FULL, val, pt < 0 ? lane : pt);
  c_out = act ? (int)(pt >= 0 ? a_pt : pi.get(J)) : 0;
  __syncwarp();
  const bool store = act && (same & ~(lt | (1u << lane))) == 0u && J >= z0 + SW;
  if (store) pi.put(J, val);
  const int nstores = __popc(__ballot_sync(FULL, store) & segmask);
  __syncwarp();
  return nstores;
}

template <class PI>
__device__ __forceinline__ int warp_fy_steps(const PI& pi, int z0, int J, int n, int lane, int& c_out) {
  return seg_fy_steps<32>(pi, z0, J, n, lane, c_out);
}

}  // namespace gm
