// gm_sketch.cu -- FastGM (Algorithm 1, Sec. 2.2) and the plain O(k n+) sketch on GB300.
//
// Work is cut into units: one per row, plus one per extra chunk of SPLIT_LEN
// elements of a long row.  A persistent grid of CTAs (two of 512 threads per SM,
// or one of 1024 at k = 4096; the kernels for both shapes come from
// gm_fastgm_shape.cuh) takes units from a counter (long-row chunks first).  The
// k registers of a unit live in shared memory as 16-byte (y, id) pairs lowered
// by 128-bit compare-and-swap; the units
// of a long row then merge their registers into global memory with the same
// compare-and-swap, the union of Sec. 2.3 (Mergeability), and the last one writes
// the row.
//
// FastGM, per unit:
//   1. a bound T = q(p) / sum v, q(p) the (1-p) quantile of y* sum v, whose law
//      (1 - e^-t)^k is the one of Sec. 2.3 (Time Complexity).  T plays the role
//      of FastSearch's release horizon R/(k sum v) (Eq. exiri): every arrival
//      <= T is generated, nothing above it.
//   2. warp screening: a warp takes 32 elements, sorts out those whose first
//      arrival is certainly above T (an FP32 test, no FP64 work), those expected
//      to need many arrivals (to the warp path) and the rest, which it hands to
//      its idle lanes.
//   3. light path: every lane walks its own element's ascending arrival stream
//      (Eq. biz_biz-1) until an arrival exceeds T (FastPrune's stopping rule),
//      the Fisher-Yates state a per-lane map of displaced positions.
//   4. warp path: 32 arrivals per step, exact shuffle scan of the prefix sums,
//      parallel Fisher-Yates on a per-warp hash of displaced positions; streams
//      too long for the hash go to one dense permutation per CTA.
//   5. if a register is still empty, no arrival <= T reached it: T is raised and
//      the row is redone (updates are idempotent minima).  Once every register
//      holds an arrival <= T, each holds the minimum over ALL arrivals, so the
//      result equals the full stream whatever T was.
// The plain sketch runs every positive element through the warp path with no
// bound: all k arrivals of every element (Sec. 1, the straightforward method).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "gm.h"
#include "gm_device.cuh"
#include "gm_internal.h"
#include "gm_stream.cuh"
#include "gm_trace.h"

namespace gm {

// Build-time knobs (overridable for experiments): light-lane map capacity, lanes
// per medium segment and its hash table.  The CTA shapes are in gm_fastgm_shape.cuh.
#ifndef GM_COMPACT_LONG
#define GM_COMPACT_LONG 1  // long rows with a fixed bound: screened first, sketched from compact lists
#endif
#ifndef GM_COMPACT_MIN_UNIT
#define GM_COMPACT_MIN_UNIT 8192  // fewest compact-list entries per chunk unit
#endif
#ifndef GM_SPLIT_MEDIUM
#define GM_SPLIT_MEDIUM 1  // compacted rows: medium elements go to the warp-path units, not the chunk units
#endif
#ifndef GM_HEAVY_UNIT
#define GM_HEAVY_UNIT 128  // warp-path elements per warp-path unit (the 8-lane segments of a 1024-thread CTA)
#endif
#ifndef GM_MAPCAP
#define GM_MAPCAP 16
#endif
#ifndef GM_MED_SW
#define GM_MED_SW 8
#endif
// The largest chunk of a long row (rows longer than SPLIT_LEN are cut into chunks
// of a length chosen per launch, chunk_len_for).
#ifndef GM_CHUNK_LEN
#define GM_CHUNK_LEN 65536
#endif
// Elements each lane screens per batch in long-row chunks (1 or 2).
#ifndef GM_SCREEN_PAIR
#define GM_SCREEN_PAIR 1
#endif
// Long-row chunk units per CTA of the persistent grid that chunk_len_for aims at.
#ifndef GM_CHUNK_UNITS_PER_CTA
#define GM_CHUNK_UNITS_PER_CTA 1.75
#endif
// Default routing by the expected number of arrivals below T (gm_tuning): light
// lanes up to LIGHT_MAX, 8-lane segments up to MEDIUM_MAX, 32-lane warps up to
// HEAVY_MAX, dense permutations beyond; first-pass bound at quantile 1 - P_FIRST.
// The values: the best of a grid over the 4,096-row lognormal batch (light 2 ..
// 8, medium 32 .. 128, heavy 128 .. 512): 2.56 ms at k = 1024 and 8.58 ms at
// k = 4096, against 2.62 / 8.80 ms with light 8.
constexpr float LIGHT_MAX = 4.0f;
constexpr float MEDIUM_MAX = 64.0f;
constexpr float HEAVY_MAX = 256.0f;
constexpr float P_FIRST = 0.05f;
constexpr int MED_SW = GM_MED_SW;
constexpr int MED_SLOTS = 16 * MED_SW;  // hash slots per medium segment
constexpr int MED_MAX_FILL = 12 * MED_SW;  // beyond: the element moves to a 32-lane warp
constexpr uint32_t TAG_MEDIUM = 1u << 30, TAG_HEAVY = 2u << 30, TAG_SUPER = 3u << 30;
constexpr uint32_t TAG_MASK = 3u << 30, SLOT_MASK = (1u << 30) - 1u;

// Per-thread counters (the per-warp phase clocks live in shared memory).
struct Counters {
  uint32_t arrivals, elements, screened, heavy, escalated, cas, kept, fallback;
  __device__ void zero() { arrivals = elements = screened = heavy = escalated = cas = kept = fallback = 0u; }
};
constexpr int CLK_LIGHT = 0, CLK_MEDIUM = 1, CLK_HEAVY = 2, CLK_SUPER = 3, CLK_WAIT = 4, CLK_SETUP = 5,
              CLK_FINISH = 6, CLK_TOTAL = 7, NCLK = 8;

struct SketchArgs {
  const int64_t* row_ptr;
  const int32_t* ids;
  const double* w;
  int32_t n_rows;
  int64_t nnz;
  int32_t k;
  uint32_t key0, key1;
  uint32_t flags;
  int32_t* s_out;
  double* y_out;
  WsHeader* hdr;
  const double* ctab;
  uint32_t* list;   // work list of the unit's warp-path elements, at the unit's element range
  uint32_t* plist;  // elements promoted from 8-lane segments to warps, same ranges
  int32_t* long_idx;
  LongRow* longs;
  Reg* long_regs;
  uint32_t* esc;
  int max_long;
  LongPiece* parts;       // per pre-pass piece of the long rows: its sums
  int chunk_len;          // elements per chunk of a long row (a multiple of PIECE_LEN, <= SPLIT_LEN)
  int ndense;             // dense permutations per CTA (warps that take super-heavy elements)
  float q1, q2, q_split;  // normalised bounds: first pass, second pass, long rows (inf = none)
  float grow;             // factor of each later pass's bound over the one before (a power of two)
  int chunk_ladder;       // bound-free: long-row chunks grow their own bound, pruned by the row's y*
  int compact;            // long rows screened first (screen_kernel): chunk units over their compact lists
  const float* t_row;     // learned first-pass bound per row (absolute), or null
  float light_max, medium_max, heavy_max;  // routing thresholds (expected arrivals below T)
  const int32_t* init_s;  // stream mode (one row): registers start from this sketch, else unfilled
  const double* init_y;
  const double* r_row;    // budget pass (plain kernel): FastSearch's R per row, else null
  int fs_delta;           // FastSearch mode (gm_sketch_fastsearch): the rounds' step Delta, else 0
  int32_t* fs_rounds;     // FastSearch mode: rounds each row took (nullable)
};

// FastSearch's release (Algorithm 1): an element of weight v in a row of FP64 sum
// dsum releases the first min(k, ceil(R (v / dsum))) arrivals of its stream by
// budget R (the ratio and the product in FP64, round to nearest, then the ceiling).
__device__ __forceinline__ int fs_budget(double R, double v, double dsum, int k) {
  if (!(R > 0.0)) return 0;
  const double b = ceil(__dmul_rn(R, __ddiv_rn(v, dsum)));
  return b < (double)k ? (int)b : k;
}


__device__ __forceinline__ bool positive_finite(double v) {
  const int64_t b = (int64_t)__double_as_longlong(v);
  return b > 0 && (uint64_t)b < INF_BITS;
}

// --------------------------------------------------------------------------
// Segment path: each SW-lane segment of a warp claims entries of class `want`
// from a work list and streams them SW arrivals per step until an arrival
// exceeds T (arrivals ascend).  An element whose permutation outgrows the
// segment's table is promoted: appended to `promote` (tagged TAG_HEAVY) or,
// without a promote list, retagged TAG_SUPER in place.  Updates are idempotent,
// so a promoted element simply starts again from its first arrival.
// --------------------------------------------------------------------------
// BUDGET: FastSearch's release instead of the bound: each claimed element streams
// exactly its first fs_budget(bR, v, bsum, k) arrivals, all of them kept.
template <int ARITH, int SW, class PI, bool BUDGET = false>
__device__ __forceinline__ void seg_phase(const SketchArgs& a, int64_t lo, uint64_t Tbits, Reg* regs,
                                          uint32_t* list, int count, int* cursor, uint32_t want, const PI& pi,
                                          int fill_limit, uint32_t* promote, int* promote_count, Counters& cnt,
                                          bool& gave_up, double bR = 0.0, double bsum = 0.0) {
  constexpr uint32_t SEGM = SW == 32 ? 0xFFFFFFFFu : ((1u << SW) - 1u);
  const int lane = threadIdx.x & 31, sl = lane & (SW - 1), base = lane & ~(SW - 1);
  const int k = a.k;
  int eidx = -1, z0 = 0, fill = 0;
  int lim = k;  // BUDGET: the element's release
  uint32_t entry = 0u;
  int32_t id = 0;
  double R = 0.0;
  Fix carry = fix_zero();
  bool list_done = false;
  while (true) {
    const bool need = (eidx < 0) && !list_done;  // uniform within the segment
    int h = 0;
    if (need && sl == 0) h = atomicAdd(cursor, 1);
    h = __shfl_sync(FULL, h, base);
    if (need) {
      if (h >= count) {
        list_done = true;
      } else {
        const uint32_t e = list[h];
        if ((e & TAG_MASK) == want) {
          eidx = h;
          entry = e;
          const int64_t g = lo + (e & SLOT_MASK);
          id = a.ids[g];
          const double v = a.w[g];
          R = arr_rcp<ARITH>(v);
          if constexpr (BUDGET) lim = fs_budget(bR, v, bsum, k);
          z0 = 0;
          fill = 0;
          carry = fix_zero();
          pi.reset_seg(k, sl, SW);
          if (sl == 0) ++cnt.heavy;
        }
      }
    }
    __syncwarp();
    const bool act = eidx >= 0;
    if (!__any_sync(FULL, act || !list_done)) break;
    if (!__any_sync(FULL, act)) continue;
    int J;
    const uint64_t bb = seg_batch<ARITH, SW>(act, id, R, z0, k, a.key0, a.key1, a.ctab, carry, lane, J);
    int nkeep;
    if constexpr (BUDGET) {
      nkeep = act ? max(0, min(SW, lim - z0)) : 0;
    } else {
      const uint32_t field = (__ballot_sync(FULL, bb <= Tbits) >> base) & SEGM;
      nkeep = act ? (field == SEGM ? SW : (__ffs(~field) - 1)) : 0;
    }
    if (act && sl == 0) cnt.arrivals += (uint32_t)min(SW, k - z0);
    int c;
    fill += seg_fy_steps<SW>(pi, z0, J, nkeep, lane, c);
    if (sl < nkeep && (!BUDGET || bb <= DBL_MAX_BITS)) {  // a released arrival that is not finite takes no register
      cnt.cas += reg_lower(smem_addr(&regs[c]), bb, (uint64_t)(uint32_t)id, gave_up);
      ++cnt.kept;
    }
    z0 += SW;
    if (act) {
      if (nkeep < SW || z0 >= k || (BUDGET && z0 >= lim)) {
        eidx = -1;
      } else if (fill > fill_limit) {  // too long for this table: promote
        if (sl == 0) {
          if (promote)
            promote[atomicAdd(promote_count, 1)] = (entry & SLOT_MASK) | TAG_HEAVY;
          else
            list[eidx] = (entry & SLOT_MASK) | TAG_SUPER;
        }
        eidx = -1;
      }
    }
  }
}

// SM clock, ordered with the surrounding memory operations and barriers.
__device__ __forceinline__ long long read_clock() {
  long long c;
  asm volatile("mov.u64 %0, %%clock64;" : "=l"(c) : : "memory");
  return c;
}

// A row's first-pass bound from the per-row table: an absolute bound, or (when
// negative) none given, so the closed form applies.
__device__ __forceinline__ bool row_bound(const SketchArgs& a, int row, float& Tf) {
  if (!a.t_row) return false;
  const float t = __ldg(&a.t_row[row]);
  if (!(t >= 0.0f)) return false;
  Tf = t;
  return true;
}

// The bound of every chunk of a long row (from the row's sum, or the table).
__device__ __forceinline__ void chunk_bound(const SketchArgs& a, int row, float sum, uint64_t& Tbits, float& Tf) {
  if (!row_bound(a, row, Tf)) Tf = a.q_split / sum;
  const bool none = !(Tf < 3.0e38f);
  Tbits = none ? DBL_MAX_BITS : (uint64_t)__double_as_longlong(f64_from_f32(Tf));
  if (none) Tf = __int_as_float(0x7F800000);
}

// Row bounds clamped to [0, nnz] so malformed row_ptr never leads out of range.
__device__ __forceinline__ void row_bounds(const SketchArgs& a, int row, int64_t& lo, int64_t& hi) {
  int64_t l = a.row_ptr[row], h = a.row_ptr[row + 1];
  if ((a.flags & GM_FLAG_VALIDATE) && h < l && threadIdx.x == 0) atomicOr(&a.hdr->status, WS_EDATA);
  l = l < 0 ? 0 : (l > a.nnz ? a.nnz : l);
  h = h < l ? l : (h > a.nnz ? a.nnz : h);
  lo = l;
  hi = h;
}

// FP64 sum of the positive weights of [lo, lo+n): per-thread strided sums, warp
// butterflies, then the warps in order.  Block-wide (two barriers).
template <int NT>
__device__ __forceinline__ double block_dsum(const double* w, int64_t lo, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) {
    const double v = w[lo + i];
    if (positive_finite(v)) s += v;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(FULL, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < NT / 32; ++q) t += red[q];
  __syncthreads();
  return t;
}

// Sum of the positive weights of [lo, lo+n) (FP32 from bits, Kahan) and their count;
// validates the elements when asked.  Block-wide; contains __syncthreads.
template <int NT>
__device__ __forceinline__ void block_sum(const SketchArgs& a, int64_t lo, int n, float* red_f, int* red_i,
                                          float& sum, int& npos) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float s = 0.0f, comp = 0.0f;
  int c = 0;
  bool bad = false;
  for (int i = tid; i < n; i += NT) {
    const double v = a.w[lo + i];
    if (positive_finite(v)) {
      const float y = f32_trunc(v) - comp;
      const float t = s + y;
      comp = (t - s) - y;
      s = t;
      ++c;
    } else if (a.flags & GM_FLAG_VALIDATE) {
      const uint64_t b = (uint64_t)__double_as_longlong(v);
      if ((b << 1) != 0ull) bad = true;  // neither +0 nor -0: negative, NaN or inf
    }
    if ((a.flags & GM_FLAG_VALIDATE) && a.ids[lo + i] < 0) bad = true;
  }
  if (bad) atomicOr(&a.hdr->status, WS_EDATA);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    s += __shfl_xor_sync(FULL, s, d);
    c += __shfl_xor_sync(FULL, c, d);
  }
  if (lane == 0) {
    red_f[warp] = s;
    red_i[warp] = c;
  }
  __syncthreads();
  float ts = 0.0f;
  int tc = 0;
  for (int q = 0; q < NT / 32; ++q) {
    ts += red_f[q];
    tc += red_i[q];
  }
  sum = ts;
  npos = tc;
  __syncthreads();
}

// 128-bit compare-and-swap minimum on a global register (the union of Sec. 2.3),
// starting from (cy, cid), a value the register held at some point.
__device__ __forceinline__ void global_lower_from(Reg* r, uint64_t yb, uint64_t id, uint64_t cy, uint64_t cid,
                                                  bool& gave_up) {
  int tries = 0;
  while (yb < cy || (yb == cy && id < cid)) {
    uint64_t oy, oid;
    asm volatile(
        "{\n\t.reg .b128 d, cmp, nv;\n\t"
        "mov.b128 cmp, {%2, %3};\n\t"
        "mov.b128 nv, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], cmp, nv;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(oy), "=l"(oid)
        : "l"(cy), "l"(cid), "l"(yb), "l"(id), "l"(r)
        : "memory");
    if (oy == cy && oid == cid) break;
    cy = oy;
    cid = oid;
    if (++tries >= CAS_CAP) {
      gave_up = true;
      break;
    }
  }
}

__device__ __forceinline__ void global_lower(Reg* r, uint64_t yb, uint64_t id, bool& gave_up) {
  global_lower_from(r, yb, id, __ldcg(&r->y), __ldcg(&r->id), gave_up);
}

// Merge a unit's k shared registers into the row's global ones, every filled
// register by the 128-bit minimum; each thread first loads the current values of
// up to four of its global registers at once, so their latencies overlap.
template <int NT>
__device__ __forceinline__ void merge_to_global(const Reg* regs, Reg* g, int k, bool& gave_up) {
  for (int j0 = threadIdx.x; j0 < k; j0 += 4 * NT) {
    uint64_t cy[4], cid[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + q * NT;
      cy[q] = cid[q] = 0ull;
      if (j < k) {
        cy[q] = __ldcg(&g[j].y);
        cid[q] = __ldcg(&g[j].id);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + q * NT;
      if (j < k) {
        const Reg r = regs[j];
        if (r.y != INF_BITS) global_lower_from(&g[j], r.y, r.id, cy[q], cid[q], gave_up);
      }
    }
  }
}

// Resolve work unit u into (row, chunk, long index).
// Units in dispatch order: the extra chunks of long rows, one unit per row
// (chunk 0 of a long row), then the super-heavy and heavy units of compacted
// long rows (chunk -1 - j for a row's unit j).  The compacted rows' chunk units
// are the longest, so they go first and the shorter heavy units fill the CTAs
// that finish early (measured on 16 x 10^6 Pareto(1.2): 0.299 against 0.317 ms
// per call with the heavy units first).
__device__ __forceinline__ void resolve_unit(const SketchArgs& a, uint32_t u, uint32_t n_hu, uint32_t n_extra,
                                             uint32_t n_long, int& row, int& chunk, int& longi) {
  u = u < n_extra + (uint32_t)a.n_rows ? u + n_hu : u - (n_extra + (uint32_t)a.n_rows);
  if (u < n_hu) {  // a heavy unit: binary search the heavy-unit offsets
    int lo = 0, hi = (int)n_long - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.longs[mid].heavy_off <= u)
        lo = mid;
      else
        hi = mid - 1;
    }
    longi = lo;
    row = (int)a.longs[lo].row;
    chunk = -1 - (int)(u - a.longs[lo].heavy_off);
    return;
  }
  u -= n_hu;
  if (u < n_extra) {  // an extra chunk of a long row: binary search the chunk offsets
    int lo = 0, hi = (int)n_long - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.longs[mid].chunk_off <= u)
        lo = mid;
      else
        hi = mid - 1;
    }
    longi = lo;
    row = (int)a.longs[lo].row;
    chunk = 1 + (int)(u - a.longs[lo].chunk_off);
  } else {
    row = (int)(u - n_extra);
    chunk = 0;
    longi = a.long_idx[row];
  }
}

// MODE_MAIN: all units.  MODE_ESC: the long rows queued for a redo, one CTA each.
constexpr int MODE_MAIN = 0;
constexpr int MODE_ESC = 1;
constexpr int MODE_FS = 2;  // FastSearch's schedule (gm_sketch_fastsearch): every row whole, by one CTA
constexpr int MODE_CMP = 3;  // MODE_MAIN for a launch whose long rows were compacted (screen_kernel)
constexpr int FS_MAX_ROUNDS = 4096;  // then one last pass releases all k arrivals of every element


// C_z = RN(1 / (k - z)); zero the header; check the row_ptr end points.
__global__ void init_kernel(WsHeader* hdr, double* ctab, int k, const int64_t* row_ptr, int n_rows, int64_t nnz,
                            uint32_t flags) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < k) ctab[z] = __drcp_rn((double)(k - z));
  if (z == 0) {
    uint32_t* h = reinterpret_cast<uint32_t*>(hdr);
    for (int q = 0; q < (int)(sizeof(WsHeader) / 4); ++q) h[q] = 0u;
    if ((flags & GM_FLAG_VALIDATE) && (row_ptr[0] != 0 || row_ptr[n_rows] != nnz)) hdr->status |= WS_EDATA;
  }
}

// Find the long rows, number their extra chunks and their pre-pass pieces (one
// CTA of 1024 threads).
constexpr int PLAN_THREADS = 1024;

// Exclusive scan of x over the CTA in blocks of PLAN_THREADS, `carry` the running
// total (shared); returns this thread's offset.  Block-wide.
__device__ __forceinline__ uint32_t plan_scan(uint32_t x, uint32_t* part, uint32_t& carry) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) part[warp] = incl;
  __syncthreads();
  uint32_t wofs = 0u;
  for (int q = 0; q < warp; ++q) wofs += part[q];
  const uint32_t off = carry + wofs + incl - x;
  __syncthreads();
  if (tid == PLAN_THREADS - 1) carry += wofs + incl;
  __syncthreads();
  return off;
}

__global__ void __launch_bounds__(PLAN_THREADS) plan_kernel(SketchArgs a) {
  __shared__ uint32_t part[PLAN_THREADS / 32];
  __shared__ uint32_t carry_c, carry_p;
  const int tid = threadIdx.x;
  for (int r = tid; r < a.n_rows; r += PLAN_THREADS) {
    int64_t lo, hi;
    row_bounds(a, r, lo, hi);
    const int64_t len = hi - lo;
    int32_t li = -1;
    if (len > SPLIT_LEN) {
      const uint32_t i = atomicAdd(&a.hdr->n_long, 1u);
      if ((int)i < a.max_long) {
        li = (int32_t)i;
        LongRow lr;
        lr.row = (uint32_t)r;
        lr.nchunks = (uint32_t)((len + a.chunk_len - 1) / a.chunk_len);
        lr.chunk_off = 0u;
        lr.done = 0u;
        lr.sum = 0.0f;
        lr.npos = 0;
        lr.dsum = 0.0;
        lr.piece_off = 0u;
        lr.npieces = (uint32_t)((len + PIECE_LEN - 1) / PIECE_LEN);
        lr.pieces_done = 0u;
        lr.ncomp = 0u;
        lr.nsuper = 0u;
        lr.nheavy = 0u;
        lr.heavy_off = 0u;
        lr.nhunits = 0u;
        a.longs[i] = lr;
      }
    }
    a.long_idx[r] = li;
  }
  __syncthreads();
  if (tid == 0) {
    carry_c = carry_p = 0u;
    if ((int)a.hdr->n_long > a.max_long) a.hdr->n_long = (uint32_t)a.max_long;  // cannot happen: max_long bounds it
  }
  __syncthreads();
  const uint32_t n_long = a.hdr->n_long;
  for (uint32_t base = 0; base < n_long; base += PLAN_THREADS) {  // exclusive scans of (nchunks - 1), npieces
    const uint32_t i = base + tid;
    const uint32_t xc = i < n_long ? a.longs[i].nchunks - 1u : 0u;
    const uint32_t xp = i < n_long ? a.longs[i].npieces : 0u;
    const uint32_t oc = plan_scan(xc, part, carry_c);
    const uint32_t op = plan_scan(xp, part, carry_p);
    if (i < n_long) {
      a.longs[i].chunk_off = oc;
      a.longs[i].piece_off = op;
    }
  }
  if (tid == 0) {
    a.hdr->n_extra = carry_c;
    a.hdr->n_pieces = carry_p;
  }
}

// Long rows: their global registers set to unfilled (or to the running sketch),
// and the sums of their weights.  One warp per pre-pass piece of PIECE_LEN
// elements: lane l adds elements l, l + 32, ... (FP32 Kahan sum built from the
// bits, the count, the FP64 sum for budget passes; GM_FLAG_VALIDATE's checks),
// the lanes combine in a fixed butterfly, the piece's sums go to parts[], and the
// warp that finishes a row's last piece adds its pieces in piece order.  So the
// sums are the same bits on every call, whatever the scheduling.
constexpr int PREP_THREADS = 256;
__global__ void __launch_bounds__(PREP_THREADS) longprep_kernel(SketchArgs a) {
  const uint32_t n_long = a.hdr->n_long, n_pieces = a.hdr->n_pieces;
  const int k = a.k;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < (int64_t)n_long * k;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(j % k);
    if (a.init_y) {  // stream mode: the one row starts from the running sketch
      a.long_regs[j].y = (uint64_t)__double_as_longlong(a.init_y[r]);
      a.long_regs[j].id = a.init_s[r] < 0 ? UNFILLED_ID : (uint64_t)(uint32_t)a.init_s[r];
    } else {
      a.long_regs[j].y = INF_BITS;
      a.long_regs[j].id = UNFILLED_ID;
    }
  }
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (PREP_THREADS / 32);
  for (uint32_t p = blockIdx.x * (PREP_THREADS / 32) + (threadIdx.x >> 5); p < n_pieces; p += warps) {
    int lo_i = 0, hi_i = (int)n_long - 1;  // the long row owning piece p
    while (lo_i < hi_i) {
      const int mid = (lo_i + hi_i + 1) >> 1;
      if (a.longs[mid].piece_off <= p)
        lo_i = mid;
      else
        hi_i = mid - 1;
    }
    const int li = lo_i;
    int64_t lo, hi;
    row_bounds(a, (int)a.longs[li].row, lo, hi);
    const int64_t plo = lo + (int64_t)(p - a.longs[li].piece_off) * PIECE_LEN;
    const int n = (int)min((int64_t)PIECE_LEN, hi - plo);
    float s = 0.0f, comp = 0.0f;
    double ds = 0.0;
    int c = 0;
    bool bad = false;
    const bool validate = (a.flags & GM_FLAG_VALIDATE) != 0;
    const bool fp64_sum = a.r_row != nullptr;  // budget passes only: FP64 adds are slow on GB300
    for (int base = 0; base < n; base += 32 * 8) {  // eight loads in flight per lane, then their sums
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = base + q * 32 + lane;
        v[q] = i < n ? __ldcs(a.w + plo + i) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (positive_finite(v[q])) {
          const float y = f32_trunc(v[q]) - comp;
          const float t = s + y;
          comp = (t - s) - y;
          s = t;
          if (fp64_sum) ds += v[q];
          ++c;
        } else if (validate) {
          const uint64_t b = (uint64_t)__double_as_longlong(v[q]);
          if ((b << 1) != 0ull) bad = true;  // neither +0 nor -0: negative, NaN or inf
        }
      }
      if (validate) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = base + q * 32 + lane;
          if (i < n && a.ids[plo + i] < 0) bad = true;
        }
      }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&a.hdr->status, WS_EDATA);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      s += __shfl_xor_sync(FULL, s, d);
      if (fp64_sum) ds += __shfl_xor_sync(FULL, ds, d);
      c += __shfl_xor_sync(FULL, c, d);
    }
    unsigned int last = 0u;
    if (lane == 0) {
      a.parts[p] = LongPiece{s, c, ds};
      __threadfence();
      last = (atomicAdd(&a.longs[li].pieces_done, 1u) == a.longs[li].npieces - 1u) ? 1u : 0u;
    }
    if (__shfl_sync(FULL, last, 0)) {  // the row's last piece: add its pieces in order
      __threadfence();
      const uint32_t p0 = a.longs[li].piece_off, np = a.longs[li].npieces;
      float rs = 0.0f, rc = 0.0f;
      double rd = 0.0;
      int rn = 0;
      for (uint32_t q = lane; q < np; q += 32) {
        const LongPiece* pp = a.parts + p0 + q;
        const float y = __ldcg(&pp->sum) - rc;
        const float t = rs + y;
        rc = (t - rs) - y;
        rs = t;
        rd += __ldcg(&pp->dsum);
        rn += __ldcg(&pp->npos);
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        rs += __shfl_xor_sync(FULL, rs, d);
        rd += __shfl_xor_sync(FULL, rd, d);
        rn += __shfl_xor_sync(FULL, rn, d);
      }
      if (lane == 0) {
        a.longs[li].sum = rs;
        a.longs[li].dsum = rd;
        a.longs[li].npos = rn;
      }
    }
  }
}

// Compacted long rows, first step: the first-arrival screen of every element of
// every long row by the whole grid at once (no barriers, no per-chunk registers),
// one warp per sub-piece (a pre-pass piece cut into 1 to 16 parts, enough for
// about two per warp of the grid), eight batches of 32 loads in flight per warp.
// An element is kept when it is positive and either expected to need more than
// a.light_max arrivals below the row's bound or not certainly above it at its
// first arrival (screen_out); the others contribute nothing to the sketch
// (Sec. 2.2, FastPrune at the first arrival).  Kept light elements are listed by
// their offset in the row at the front of the row's range of plist (each warp
// stages up to SCREEN_BUF of them in shared memory and claims their place with
// one atomic add); medium and heavy ones (above a.light_max, for the 8-lane and
// 32-lane paths) at the back of the row's range of list, tagged; super-heavy ones
// (above a.heavy_max, each streamed by a whole CTA) at the back of its range of
// plist.  Entries come in
// no particular order: register updates are order-free minima.  The dropped
// positive elements and the medium and heavy ones are counted here, the light
// ones by the chunk units that stream them.
constexpr int SCREEN_THREADS = 256;
constexpr int SCREEN_BUF = 256;
#ifndef GM_SCREEN_DEPTH
#define GM_SCREEN_DEPTH 8  // batches of 32 loads in flight per warp
#endif
#ifndef GM_SCREEN_MINB
#define GM_SCREEN_MINB 4  // resident CTAs per SM the register budget is sized for
#endif
constexpr int SD = GM_SCREEN_DEPTH;
// Class limits of x = v T: expected arrivals k (1 - exp(-x)) above lim <=> x > -ln(1 - lim / k).
__device__ __forceinline__ float class_limit(float lim, float kf) {
  return lim < kf ? -log1pf(-lim / kf) : __int_as_float(0x7F800000);
}
constexpr int HEAVY_UNIT = GM_HEAVY_UNIT;
__global__ void __launch_bounds__(SCREEN_THREADS, GM_SCREEN_MINB) screen_kernel(SketchArgs a) {
  __shared__ uint32_t buf[SCREEN_THREADS / 32][SCREEN_BUF];
  const uint32_t n_long = a.hdr->n_long, n_pieces = a.hdr->n_pieces;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* wb = buf[warp];
  const float kf = (float)a.k;
  uint32_t n_elem = 0u, n_scr = 0u;
  const uint32_t warps = gridDim.x * (SCREEN_THREADS / 32);
  uint32_t S = 1u;
  while (S < 16u && (uint64_t)n_pieces * S < 2ull * warps) S <<= 1;
  const int sublen = PIECE_LEN / (int)S;
  const uint64_t n_units = (uint64_t)n_pieces * S;
  for (uint64_t q = (uint64_t)blockIdx.x * (SCREEN_THREADS / 32) + warp; q < n_units; q += warps) {
    const uint32_t p = (uint32_t)(q / S), sub = (uint32_t)(q % S);
    int lo_i = 0, hi_i = (int)n_long - 1;  // the long row owning piece p
    while (lo_i < hi_i) {
      const int mid = (lo_i + hi_i + 1) >> 1;
      if (a.longs[mid].piece_off <= p)
        lo_i = mid;
      else
        hi_i = mid - 1;
    }
    const int li = lo_i;
    const int row = (int)a.longs[li].row;
    if (a.longs[li].npos <= 0) continue;  // nothing to sketch in this row
    int64_t lo, hi;
    row_bounds(a, row, lo, hi);
    const uint32_t off = (p - a.longs[li].piece_off) * (uint32_t)PIECE_LEN + sub * (uint32_t)sublen;
    if (lo + off >= hi) continue;
    const int n = (int)min((int64_t)sublen, hi - (lo + off));
    uint64_t Tbits;
    float Tf;
    chunk_bound(a, row, a.longs[li].sum, Tbits, Tf);
    // the classes by x = v T against limits taken once (routing only: the chunk
    // units route by the expected count itself, and either way is exact)
    const float xl = class_limit(a.light_max, kf), xm = class_limit(a.medium_max, kf),
                xh = class_limit(a.heavy_max, kf);
    int nb = 0;  // staged entries (warp-uniform)
    for (int base = 0; base < n; base += SD * 32) {
      double v[SD];
      int32_t id[SD];
#pragma unroll
      for (int r = 0; r < SD; ++r) {
        const int i = base + r * 32 + lane;
        v[r] = i < n ? __ldcs(a.w + lo + off + i) : 0.0;
        id[r] = i < n ? __ldcs(a.ids + lo + off + i) : 0;
      }
#pragma unroll
      for (int r = 0; r < SD; ++r) {
        const int i = base + r * 32 + lane;
        bool keep = false;
        if (i < n && positive_finite(v[r])) {
          // the FP64 pipe is idle here: one truncating conversion there, equal to
          // f32_trunc(v) in FP32's normal range (outside it neither test decides)
          const float vf = __double2float_rz(v[r]);
          const float x = vf * Tf;
          ++n_elem;
          if (x > xh) {  // super-heavy: a unit of its own, dispatched first
            a.plist[hi - 1 - atomicAdd(&a.longs[li].nsuper, 1u)] = off + (uint32_t)i;
          } else if (x > xm) {  // heavy: units of HEAVY_UNIT, dispatched first
            a.list[hi - 1 - atomicAdd(&a.longs[li].nheavy, 1u)] = (off + (uint32_t)i) | TAG_HEAVY;
          } else if (x > xl) {
            if (GM_SPLIT_MEDIUM)
              a.list[hi - 1 - atomicAdd(&a.longs[li].nheavy, 1u)] = (off + (uint32_t)i) | TAG_MEDIUM;
            else
              keep = true;
          } else {
            const Words wd = philox((uint32_t)id[r], 0u, a.key0, a.key1);
            keep = !screen_out(wd.w1, vf, Tf, kf);
            if (!keep) ++n_scr;
          }
          if (keep) --n_elem;  // counted by its chunk unit
        }
        const uint32_t m = __ballot_sync(FULL, keep);
        if (keep) wb[nb + __popc(m & lanemask_lt())] = off + (uint32_t)i;
        nb += __popc(m);
        if (nb > SCREEN_BUF - 32) {  // flush the staged entries
          __syncwarp();
          uint32_t at = 0u;
          if (lane == 0) at = atomicAdd(&a.longs[li].ncomp, (uint32_t)nb);
          at = __shfl_sync(FULL, at, 0);
          for (int j = lane; j < nb; j += 32) a.plist[lo + at + j] = wb[j];
          __syncwarp();
          nb = 0;
        }
      }
    }
    if (nb > 0) {
      __syncwarp();
      uint32_t at = 0u;
      if (lane == 0) at = atomicAdd(&a.longs[li].ncomp, (uint32_t)nb);
      at = __shfl_sync(FULL, at, 0);
      for (int j = lane; j < nb; j += 32) a.plist[lo + at + j] = wb[j];
      __syncwarp();
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    n_elem += __shfl_xor_sync(FULL, n_elem, d);
    n_scr += __shfl_xor_sync(FULL, n_scr, d);
  }
  if (lane == 0 && n_elem) {
    atomicAdd(&a.hdr->counters[1], (unsigned long long)n_elem);
    atomicAdd(&a.hdr->counters[2], (unsigned long long)n_scr);
  }
}

// Compacted long rows, second step (one CTA): every long row's compact list cut
// into chunk units of `cunit` entries, the same for all rows -- about two units
// per CTA of the main kernel's `grid`, between GM_COMPACT_MIN_UNIT and 65,536
// entries -- its super-heavy elements one unit each and its heavy list into
// units of HEAVY_UNIT elements; the units numbered as resolve_unit reads them
// (heavy_off, n_hunits; chunk_off, n_extra).
__global__ void __launch_bounds__(PLAN_THREADS) compact_plan_kernel(SketchArgs a, int grid) {
  __shared__ uint32_t part[PLAN_THREADS / 32];
  __shared__ uint32_t carry_c, carry_h;
  __shared__ unsigned long long total;
  const int tid = threadIdx.x;
  const uint32_t n_long = a.hdr->n_long;
  if (tid == 0) {
    carry_c = carry_h = 0u;
    total = 0ull;
  }
  __syncthreads();
  unsigned long long t = 0ull;
  for (uint32_t i = tid; i < n_long; i += PLAN_THREADS) t += a.longs[i].ncomp;
  atomicAdd(&total, t);
  __syncthreads();
  unsigned long long cu = (total + 2ull * (unsigned long long)grid - 1ull) / (2ull * (unsigned long long)grid);
  cu = cu < GM_COMPACT_MIN_UNIT ? GM_COMPACT_MIN_UNIT : (cu > 65536ull ? 65536ull : cu);
  for (uint32_t base = 0; base < n_long; base += PLAN_THREADS) {
    const uint32_t i = base + tid;
    uint32_t nc = 1u, nh = 0u;
    if (i < n_long) {
      const uint32_t c = a.longs[i].ncomp;
      nc = c == 0u ? 1u : (uint32_t)((c + cu - 1ull) / cu);
      nh = a.longs[i].nsuper + (a.longs[i].nheavy + HEAVY_UNIT - 1u) / HEAVY_UNIT;
    }
    const uint32_t oc = plan_scan(i < n_long ? nc - 1u : 0u, part, carry_c);
    const uint32_t oh = plan_scan(nh, part, carry_h);
    if (i < n_long) {
      a.longs[i].nchunks = nc;
      a.longs[i].chunk_off = oc;
      a.longs[i].nhunits = nh;
      a.longs[i].heavy_off = oh;
    }
  }
  __syncthreads();
  if (tid == 0) {
    a.hdr->n_extra = carry_c;
    a.hdr->n_hunits = carry_h;
    a.hdr->cunit = (uint32_t)cu;
  }
}

static double quantile_bound(double p, int k) {
  // (1 - p) quantile of max of k iid Exp(1):  -ln(1 - (1 - p)^(1/k))
  return -std::log(-std::expm1(std::log1p(-p) / (double)k));
}

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per (kernel, device).  Calls on several host threads with different k
// share the kernel: lowering the limit to one call's size could make another
// call's launch fail, so the limit is only ever raised, and to the top.
static int allow_max_smem(const void* kern) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GM_ECUDA;
  std::lock_guard<std::mutex> g(mu);
  if (done.count({kern, dev})) return GM_OK;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return GM_ECUDA;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return GM_ECUDA;
  // the dynamic part may take what the kernel's static shared memory leaves
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) !=
      cudaSuccess)
    return GM_ECUDA;
  done.insert({kern, dev});
  return GM_OK;
}

// Optional events recorded around the main FastGM (or plain) kernel launch, for
// timing that kernel alone on the call's stream (gm_diag_time_main_kernel).
static cudaEvent_t g_main_before = nullptr, g_main_after = nullptr;


#define GM_SHAPE_NS s512
#define GM_SHAPE_BLOCK 512
#include "gm_fastgm_shape.cuh"
#undef GM_SHAPE_NS
#undef GM_SHAPE_BLOCK
#define GM_SHAPE_NS s1024
#define GM_SHAPE_BLOCK 1024
#include "gm_fastgm_shape.cuh"
#undef GM_SHAPE_NS
#undef GM_SHAPE_BLOCK

// Rows of k >= WIDE_K registers go to 1024-thread CTAs, one per SM: twice the
// warps on a row and the SM's whole shared memory for its permutations (measured
// at k = 4096: 9.83 ms per 4,096-row batch against 11.28 with two 512-thread
// CTAs; at k = 1024: 3.25 against 2.89).  The default arithmetic only; the
// others and the plain sketch keep 512-thread CTAs.
#ifndef GM_WIDE_K
#define GM_WIDE_K 4096
#endif
constexpr int WIDE_K = GM_WIDE_K;

template <int ARITH>
static int launch_shape(const SketchArgs& a, bool plain, int nsm, size_t smem_per_sm, cudaStream_t stream) {
  if constexpr (ARITH == ARITH_MIX)
    if (!plain && a.k >= WIDE_K) return s1024::launch<ARITH>(a, plain, nsm, smem_per_sm, stream);
  return s512::launch<ARITH>(a, plain, nsm, smem_per_sm, stream);
}

// ---------------------------------------------------------------------------
// Tuning table: (k, floor(log2(mean row length))) -> gm_tuning.
// ---------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, gm_tuning> g_tune;

static int tune_bucket(int64_t mean_len) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << (b + 1)) <= mean_len) ++b;
  return b;
}
static bool tuning_ok(const gm_tuning& t) {
  return t.p_first > 0.0f && t.p_first < 1.0f && t.light_max > 0.0f && t.light_max <= t.medium_max &&
         t.medium_max <= t.heavy_max && std::isfinite(t.heavy_max);
}
static gm_tuning tuning_for(int k, int32_t n_rows, int64_t nnz) {
  gm_tuning t{P_FIRST, LIGHT_MAX, MEDIUM_MAX, HEAVY_MAX};
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find({k, tune_bucket(n_rows > 0 ? nnz / n_rows : 0)});
  if (it != g_tune.end()) t = it->second;
  return t;
}

static int launch_sketch_tuned(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                               int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out,
                               void* workspace, size_t workspace_bytes, cudaStream_t stream, bool plain,
                               const float* t_row, const gm_tuning* tuning, const int32_t* init_s = nullptr,
                               const double* init_y = nullptr, const double* r_row = nullptr, int fs_delta = 0,
                               int32_t* fs_rounds = nullptr);

int launch_sketch(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                  int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
                  size_t workspace_bytes, cudaStream_t stream, bool plain, const float* t_row) {
  return launch_sketch_tuned(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, workspace, workspace_bytes,
                             stream, plain, t_row, nullptr);
}

static int launch_sketch_tuned(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                               int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out,
                               void* workspace, size_t workspace_bytes, cudaStream_t stream, bool plain,
                               const float* t_row, const gm_tuning* tuning, const int32_t* init_s,
                               const double* init_y, const double* r_row, int fs_delta, int32_t* fs_rounds) {
  const TraceRange trace(plain ? (r_row ? "gm_sketch_budget" : "gm_sketch_plain")
                               : fs_delta > 0 ? "gm_sketch_fastsearch"
                               : (init_y ? "gm_stream_ingest" : (t_row ? "gm_sketch (per-row bounds)" : "gm_sketch")));
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K) return GM_EINVAL;
  if (init_y && (n_rows != 1 || plain)) return GM_EINVAL;
  if (nnz > 0x7FFFFFFFll) return GM_EINVAL;
  if (!workspace || !ws_aligned(workspace) || !row_ptr || (n_rows > 0 && (!s_out || !y_out)) ||
      (nnz > 0 && (!ids || !w)))
    return GM_EINVAL;
  const uint32_t bound = flags & GM_BOUND_MASK;
  if (!plain && bound == GM_BOUND_LEARNED) return GM_EINVAL;  // needs a trained model
  const size_t need = gm_sketch_workspace_bytes(n_rows, nnz, k, flags);
  if (need == 0) return GM_EINVAL;
  if (workspace_bytes < need) return GM_ENOMEM;
  WsLayout L = ws_layout(workspace, n_rows, nnz, k);

  init_kernel<<<(k + 255) / 256, 256, 0, stream>>>(L.hdr, L.ctab, k, row_ptr, n_rows, nnz, flags);
  if (cudaGetLastError() != cudaSuccess) return GM_ECUDA;
  if (n_rows == 0) return GM_OK;

  SketchArgs a;
  a.row_ptr = row_ptr;
  a.ids = ids;
  a.w = w;
  a.n_rows = n_rows;
  a.nnz = nnz;
  a.k = k;
  a.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
  a.key1 = (uint32_t)(seed >> 32);
  a.flags = flags;
  a.s_out = s_out;
  a.y_out = y_out;
  a.hdr = L.hdr;
  a.ctab = L.ctab;
  a.list = L.list;
  a.plist = L.plist;
  a.long_idx = L.long_idx;
  a.longs = L.longs;
  a.long_regs = reinterpret_cast<Reg*>(L.long_regs);
  a.esc = L.esc;
  a.parts = L.parts;
  a.chunk_len = SPLIT_LEN;  // set per shape by the launcher
  a.max_long = (int)L.max_long;
  a.t_row = plain ? nullptr : t_row;
  a.init_s = init_s;
  a.init_y = init_y;
  a.r_row = plain ? r_row : nullptr;
  a.fs_delta = plain ? 0 : fs_delta;
  a.fs_rounds = fs_rounds;
  const gm_tuning tn = tuning ? *tuning : tuning_for(k, n_rows, nnz);
  if (!tuning_ok(tn)) return GM_EINVAL;
  a.light_max = tn.light_max;
  a.medium_max = tn.medium_max;
  a.heavy_max = tn.heavy_max;
  if (bound == GM_BOUND_NONE) {
    // FastSearch without prior knowledge of y*: the release horizon starts at R = k
    // arrivals per row (T = 1 / sum v) and doubles until every register is filled;
    // long-row chunks run the same ladder on their own registers, pruned by the
    // row's merged y* once it is finite (FastPrune), so no long row is redone.
    a.q1 = 1.0f;
    a.q2 = 2.0f;
    a.grow = 2.0f;
    a.q_split = INFINITY;
    a.chunk_ladder = 1;
  } else {
    a.q1 = (float)quantile_bound((double)tn.p_first, k);
    a.q2 = (float)quantile_bound(1e-6, k);
    a.q_split = (float)quantile_bound(1e-3, k);
    a.grow = 16.0f;
    a.chunk_ladder = 0;
    if (flags & GM_FLAG_TIGHT_BOUND) {
      a.q1 *= 0.125f;
      a.q_split *= 0.125f;
    }
  }
  int dev = 0, nsm = 0, smem_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GM_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GM_ECUDA;
  if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    return GM_ECUDA;
  const size_t smem = (size_t)smem_sm;
  const int rc = (flags & GM_FLAG_FP64_UNIT)      ? launch_shape<ARITH_FP64>(a, plain, nsm, smem, stream)
                 : (flags & GM_FLAG_INT_PRODUCTS) ? launch_shape<ARITH_INT>(a, plain, nsm, smem, stream)
                                                  : launch_shape<ARITH_MIX>(a, plain, nsm, smem, stream);
  if (rc != GM_OK) return rc;
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

}  // namespace gm

extern "C" int gm_diag_time_main_kernel(void* before, void* after) {
  if ((before == nullptr) != (after == nullptr)) return GM_EINVAL;
  gm::g_main_before = (cudaEvent_t)before;
  gm::g_main_after = (cudaEvent_t)after;
  return GM_OK;
}

extern "C" size_t gm_sketch_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k, uint32_t flags) {
  (void)flags;
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K) return 0;
  return gm::ws_bytes(n_rows, nnz, k);
}

extern "C" int gm_sketch(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                         int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
                         size_t workspace_bytes, void* stream) {
  return gm::launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, workspace, workspace_bytes,
                           (cudaStream_t)stream, false, nullptr);
}

extern "C" int gm_sketch_plain(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                               int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out,
                               double* y_out, void* workspace, size_t workspace_bytes, void* stream) {
  return gm::launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, flags & (GM_FLAG_VALIDATE | GM_FLAG_FP64_UNIT | GM_FLAG_INT_PRODUCTS),
                           s_out, y_out, workspace, workspace_bytes, (cudaStream_t)stream, true, nullptr);
}

extern "C" void gm_tuning_default(gm_tuning* t) {
  if (t) *t = gm_tuning{gm::P_FIRST, gm::LIGHT_MAX, gm::MEDIUM_MAX, gm::HEAVY_MAX};
}

extern "C" int gm_tuning_set(int32_t k, int64_t mean_row_len, const gm_tuning* t) {
  if (!t || k < 1 || k > GM_MAX_K || mean_row_len < 0 || !gm::tuning_ok(*t)) return GM_EINVAL;
  std::lock_guard<std::mutex> g(gm::g_tune_mu);
  gm::g_tune[{k, gm::tune_bucket(mean_row_len)}] = *t;
  return GM_OK;
}

extern "C" int gm_tuning_get(int32_t k, int64_t mean_row_len, gm_tuning* out) {
  if (!out || k < 1 || k > GM_MAX_K || mean_row_len < 0) return GM_EINVAL;
  gm_tuning_default(out);
  std::lock_guard<std::mutex> g(gm::g_tune_mu);
  auto it = gm::g_tune.find({k, gm::tune_bucket(mean_row_len)});
  if (it == gm::g_tune.end()) return GM_EINVAL;
  *out = it->second;
  return GM_OK;
}

extern "C" int gm_tuning_clear(void) {
  std::lock_guard<std::mutex> g(gm::g_tune_mu);
  gm::g_tune.clear();
  return GM_OK;
}

// Text: one line per entry, "k bucket p_first light_max medium_max heavy_max".
extern "C" int gm_tuning_save(const char* path) {
  if (!path) return GM_EINVAL;
  FILE* f = std::fopen(path, "w");
  if (!f) return GM_EINVAL;
  bool ok = std::fprintf(f, "# gm_tuning v1: k log2(mean row length) p_first light_max medium_max heavy_max\n") > 0;
  {
    std::lock_guard<std::mutex> g(gm::g_tune_mu);
    for (const auto& kv : gm::g_tune)
      ok = ok && std::fprintf(f, "%d %d %.9g %.9g %.9g %.9g\n", kv.first.first, kv.first.second, kv.second.p_first,
                              kv.second.light_max, kv.second.medium_max, kv.second.heavy_max) > 0;
  }
  return (std::fclose(f) == 0 && ok) ? GM_OK : GM_EINVAL;
}

extern "C" int gm_tuning_load(const char* path) {
  if (!path) return GM_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return GM_EINVAL;
  char line[256];
  std::vector<std::pair<std::pair<int, int>, gm_tuning>> got;
  bool ok = true;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int k = 0, b = 0;
    gm_tuning t{};
    if (std::sscanf(line, "%d %d %f %f %f %f", &k, &b, &t.p_first, &t.light_max, &t.medium_max, &t.heavy_max) != 6 ||
        k < 1 || k > GM_MAX_K || b < 0 || b > 62 || !gm::tuning_ok(t)) {
      ok = false;
      break;
    }
    got.push_back({{k, b}, t});
  }
  std::fclose(f);
  if (!ok) return GM_EDATA;
  std::lock_guard<std::mutex> g(gm::g_tune_mu);
  for (const auto& e : got) gm::g_tune[e.first] = e.second;
  return GM_OK;
}

extern "C" int gm_tune(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                       int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
                       size_t workspace_bytes, gm_tuning* best, double* best_ms, void* stream) {
  if (!best || k < 1 || k > GM_MAX_K || n_rows < 0 || nnz < 0) return GM_EINVAL;
  const gm::TraceRange trace("gm_tune");
  const cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return GM_ECUDA;
  }
  auto run = [&](const gm_tuning& t, float* ms) -> int {
    int rc = gm::launch_sketch_tuned(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, workspace,
                                     workspace_bytes, st, false, nullptr, &t);
    if (rc != GM_OK) return rc;
    float fastest = INFINITY;
    for (int rep = 0; rep < 3; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess) return GM_ECUDA;
      rc = gm::launch_sketch_tuned(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, workspace,
                                   workspace_bytes, st, false, nullptr, &t);
      if (rc != GM_OK) return rc;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return GM_ECUDA;
      float m = 0.0f;
      if (cudaEventElapsedTime(&m, e0, e1) != cudaSuccess) return GM_ECUDA;
      fastest = m < fastest ? m : fastest;
    }
    *ms = fastest;
    return GM_OK;
  };
  gm_tuning cur = gm::tuning_for(k, n_rows, nnz);
  float t_cur = 0.0f;
  int rc = run(cur, &t_cur);
  const float p_cand[] = {0.01f, 0.02f, 0.05f, 0.1f, 0.2f, 0.35f};
  const float l_cand[] = {3.0f, 4.0f, 6.0f, 8.0f, 11.0f};
  const float m_cand[] = {24.0f, 32.0f, 48.0f, 64.0f, 96.0f};
  const float h_cand[] = {128.0f, 256.0f, 512.0f, 1024.0f};
  struct Axis {
    float gm_tuning::*field;
    const float* vals;
    int n;
  } axes[] = {{&gm_tuning::p_first, p_cand, 6}, {&gm_tuning::light_max, l_cand, 5},
              {&gm_tuning::medium_max, m_cand, 5}, {&gm_tuning::heavy_max, h_cand, 4}};
  // coordinate descent, at most two sweeps (the second only if the first moved);
  // a candidate must beat the current choice by 1 %
  for (int sweep = 0; sweep < 2 && rc == GM_OK; ++sweep) {
    bool moved = false;
    for (const Axis& ax : axes) {
      for (int i = 0; i < ax.n && rc == GM_OK; ++i) {
        gm_tuning t = cur;
        t.*(ax.field) = ax.vals[i];
        if (t.*(ax.field) == cur.*(ax.field) || !gm::tuning_ok(t)) continue;
        float ms = 0.0f;
        rc = run(t, &ms);
        if (rc == GM_OK && ms < 0.99f * t_cur) {
          cur = t;
          t_cur = ms;
          moved = true;
        }
      }
    }
    if (!moved) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GM_OK) return rc;
  {
    std::lock_guard<std::mutex> g(gm::g_tune_mu);
    gm::g_tune[{k, gm::tune_bucket(n_rows > 0 ? nnz / n_rows : 0)}] = cur;
  }
  *best = cur;
  if (best_ms) *best_ms = t_cur;
  return GM_OK;
}

// ---------------------------------------------------------------------------
// Stream-FastGM (Algorithm 2): chunks of a stream folded into a running sketch.
// ---------------------------------------------------------------------------
namespace gm {

// row_ptr = {0, n}; the chunk's first-pass bound: the running sketch's y* rounded
// up to FP32 once every register is filled (an arrival above it cannot lower any
// register), else -1 (the closed form of the chunk applies).
__global__ void stream_prep_kernel(const double* __restrict__ y, int k, int64_t n, int64_t* row_ptr, float* t_row) {
  __shared__ unsigned long long red[8];
  unsigned long long m = 0ull;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(y[j]);
    m = b > m ? b : m;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, m, d);
    m = o > m ? o : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = red[q] > m ? red[q] : m;
    row_ptr[0] = 0;
    row_ptr[1] = n;
    const double ys = __longlong_as_double((long long)m);
    // rounded up, and at least the smallest normal float (a larger bound is always safe)
    t_row[0] = (m >= INF_BITS) ? -1.0f : fmaxf(__double2float_ru(ys), 1.17549435e-38f);
  }
}

__global__ void stream_reset_kernel(int32_t* s, double* y, int k) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) {
    s[j] = -1;
    y[j] = __longlong_as_double((long long)INF_BITS);
  }
}

}  // namespace gm

extern "C" size_t gm_stream_workspace_bytes(int64_t n, int32_t k) {
  if (n < 0 || k < 1 || k > GM_MAX_K) return 0;
  return gm::ws_bytes(1, n, k) + 256;
}

extern "C" int gm_stream_reset(int32_t* s, double* y, int32_t k, void* stream) {
  if (!s || !y || k < 1 || k > GM_MAX_K) return GM_EINVAL;
  gm::stream_reset_kernel<<<(k + 255) / 256, 256, 0, (cudaStream_t)stream>>>(s, y, k);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_stream_ingest(int32_t* s, double* y, int32_t k, const int32_t* ids, const double* w, int64_t n,
                                uint64_t seed, uint32_t flags, void* workspace, size_t workspace_bytes, void* stream) {
  if (!s || !y || k < 1 || k > GM_MAX_K || n < 0 || n > 0x7FFFFFFFll || (n > 0 && (!ids || !w)) || !workspace ||
      !gm::ws_aligned(workspace))
    return GM_EINVAL;
  if ((flags & GM_BOUND_MASK) == GM_BOUND_LEARNED) return GM_EINVAL;
  const size_t base = gm::ws_bytes(1, n, k);
  if (workspace_bytes < gm_stream_workspace_bytes(n, k)) return GM_ENOMEM;
  if (n == 0) return GM_OK;
  unsigned char* extra = static_cast<unsigned char*>(workspace) + base;
  int64_t* row_ptr = reinterpret_cast<int64_t*>(extra);
  float* t_row = reinterpret_cast<float*>(extra + 16);
  const cudaStream_t st = (cudaStream_t)stream;
  gm::stream_prep_kernel<<<1, 256, 0, st>>>(y, k, n, row_ptr, t_row);
  if (cudaGetLastError() != cudaSuccess) return GM_ECUDA;
  return gm::launch_sketch_tuned(row_ptr, ids, w, 1, n, k, seed, flags, s, y, workspace, base, st, false, t_row,
                                 nullptr, s, y);
}

// ---------------------------------------------------------------------------
// FastSearch's budgets (Algorithm 1) and caller-given bounds.
// ---------------------------------------------------------------------------
namespace gm {

// Per-row bounds given as doubles -> the sketch's FP32 first-pass bounds, rounded
// up (a larger bound is always safe): > 0 and finite: that bound; +inf: none;
// otherwise (<= 0, NaN): -1, the closed form.
__global__ void bound_prep_kernel(const double* __restrict__ b, int n, float* t_row) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double x = b[r];
  float t = -1.0f;
  if (x > 0.0) t = isinf(x) ? __int_as_float(0x7F800000) : fmaxf(__double2float_ru(x), 1.17549435e-38f);
  t_row[r] = t;
}

// The largest register of each row (+inf if one is unfilled), one warp per row.
__global__ void row_ystar_kernel(const double* __restrict__ y, int n_rows, int k, double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= n_rows) return;
  unsigned long long m = 0ull;
  for (int j = lane; j < k; j += 32) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(y[r * k + j]);
    m = b > m ? b : m;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, m, d);
    m = o > m ? o : m;
  }
  if (lane == 0) out[r] = __longlong_as_double((long long)m);
}

}  // namespace gm

extern "C" int gm_sketch_budget(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                                int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, const double* R_row,
                                int32_t* s_out, double* y_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!R_row && n_rows > 0) return GM_EINVAL;
  return gm::launch_sketch_tuned(row_ptr, ids, w, n_rows, nnz, k, seed,
                                 flags & (GM_FLAG_VALIDATE | GM_FLAG_FP64_UNIT | GM_FLAG_INT_PRODUCTS), s_out, y_out,
                                 workspace, workspace_bytes, (cudaStream_t)stream, true, nullptr, nullptr, nullptr,
                                 nullptr, R_row);
}

extern "C" int gm_sketch_fastsearch(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                                    int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t delta,
                                    int32_t* rounds_out, int32_t* s_out, double* y_out, void* workspace,
                                    size_t workspace_bytes, void* stream) {
  if (delta < 1) return GM_EINVAL;
  return gm::launch_sketch_tuned(row_ptr, ids, w, n_rows, nnz, k, seed,
                                 flags & (GM_FLAG_VALIDATE | GM_FLAG_FP64_UNIT | GM_FLAG_INT_PRODUCTS), s_out, y_out,
                                 workspace, workspace_bytes, (cudaStream_t)stream, false, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, delta, rounds_out);
}

extern "C" size_t gm_sketch_bounded_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k) {
  const size_t base = gm_sketch_workspace_bytes(n_rows, nnz, k, 0u);
  return base ? base + gm::round_up((size_t)(n_rows > 0 ? n_rows : 0) * 4, 256) : 0;
}

extern "C" int gm_sketch_bounded(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                                 int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, const double* bound_row,
                                 int32_t* s_out, double* y_out, void* workspace, size_t workspace_bytes,
                                 void* stream) {
  if (n_rows < 0 || (n_rows > 0 && !bound_row) || !workspace || !gm::ws_aligned(workspace)) return GM_EINVAL;
  if ((flags & GM_BOUND_MASK) == GM_BOUND_LEARNED) return GM_EINVAL;
  const size_t need = gm_sketch_bounded_workspace_bytes(n_rows, nnz, k);
  if (need == 0) return GM_EINVAL;
  if (workspace_bytes < need) return GM_ENOMEM;
  const size_t base = gm_sketch_workspace_bytes(n_rows, nnz, k, 0u);
  float* t_row = reinterpret_cast<float*>(static_cast<unsigned char*>(workspace) + base);
  const cudaStream_t st = (cudaStream_t)stream;
  if (n_rows > 0) {
    gm::bound_prep_kernel<<<(n_rows + 255) / 256, 256, 0, st>>>(bound_row, n_rows, t_row);
    if (cudaGetLastError() != cudaSuccess) return GM_ECUDA;
  }
  return gm::launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, workspace, base, st, false,
                           n_rows > 0 ? t_row : nullptr);
}

extern "C" int gm_row_ystar(const double* y, int32_t n_rows, int32_t k, double* out, void* stream) {
  if (n_rows < 0 || k < 1 || (n_rows > 0 && (!y || !out))) return GM_EINVAL;
  if (n_rows == 0) return GM_OK;
  const int64_t threads = (int64_t)n_rows * 32;
  gm::row_ystar_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(y, n_rows, k, out);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

// ---------------------------------------------------------------------------
// gm_sketch_noalloc: gm_sketch with its scratch in a fixed device array.
//
// Some callers cannot give the library a workspace: code whose device memory
// is owned by a host framework or plugin allocator that forbids foreign
// allocations, serving loops that must never stall on cudaMalloc (it can
// synchronise the device and can fail under memory pressure), and thin
// foreign-function bindings that can only hand over input and output buffers.
// This entry point serves them: it launches the same kernels as gm_sketch, but
// the scratch lives in g_noalloc_scratch below, a file-scope device array that
// every GPU loading the library holds until the process exits.
//
// In host code `g_noalloc_scratch` is only a host-side stand-in for the symbol,
// not a device address, so its device address is looked up with
// cudaGetSymbolAddress with the device current: on every call made outside
// stream capture (so that an address from before a cudaDeviceReset is never
// reused), and taken from the per-device cache during capture.
// ---------------------------------------------------------------------------
#include <mutex>

namespace gm {

constexpr size_t NOALLOC_SCRATCH_BYTES = ws_bytes(GM_NOALLOC_MAX_ROWS, GM_NOALLOC_MAX_NNZ, GM_MAX_K);
// 10,788,096 bytes (about 10.8 MB, 10.3 MiB): two 4 MiB element lists, 2 MiB of
// long-row registers, the per-row index and the small tables.
static_assert(NOALLOC_SCRATCH_BYTES == 10788096, "the documented size of the no-alloc scratch changed");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_noalloc_mutex;

// Device address of g_noalloc_scratch on the current device: looked up afresh
// unless `stream` is capturing, then taken from the cache of an earlier call.
static int noalloc_scratch(cudaStream_t stream, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return GM_ECUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
    cudaGetLastError();  // clear it; use the cache below
    cap = cudaStreamCaptureStatusActive;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cap == cudaStreamCaptureStatusNone || !g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GM_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GM_OK;
}

}  // namespace gm

extern "C" int gm_sketch_noalloc(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                                 int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out,
                                 double* y_out, void* stream) {
  if (nnz > GM_NOALLOC_MAX_NNZ || n_rows > GM_NOALLOC_MAX_ROWS) return GM_ENOMEM;  // beyond the fixed scratch
  const size_t need = gm_sketch_workspace_bytes(n_rows, nnz, k, flags);
  if (need == 0) return GM_EINVAL;
  if (need > gm::NOALLOC_SCRATCH_BYTES) return GM_ENOMEM;
  void* scratch = nullptr;
  const int rc = gm::noalloc_scratch((cudaStream_t)stream, &scratch);
  if (rc != GM_OK) return rc;
  // The first kernel of every call zeroes the scratch header (status, row counter,
  // counters) and rewrites the 1/(k-z) table; the heavy list is written before it
  // is read.  No other state carries over from the previous call.
  return gm::launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, scratch,
                           gm::NOALLOC_SCRATCH_BYTES, (cudaStream_t)stream, false, nullptr);
}

extern "C" int gm_sketch_noalloc_status(gm_stats* stats, void* stream) {
  void* scratch = nullptr;
  const int rc = gm::noalloc_scratch((cudaStream_t)stream, &scratch);
  if (rc != GM_OK) return rc;
  return gm_status(scratch, stats, stream);
}
