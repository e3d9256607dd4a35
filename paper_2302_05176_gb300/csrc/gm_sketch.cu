// gm_sketch.cu -- FastGM (Algorithm 1, Sec. 2.2) and the plain O(k n+) sketch on GB300.
//
// One CTA sketches one row at a time (persistent grid, rows taken from a global
// counter).  The k registers live in shared memory as 16-byte (y, id) pairs.
//
// FastGM, per row:
//   1. sum v over the row (FP32, only used to place the bound) and the bound
//      T = q(p) / sum v, where q(p) is the (1-p) quantile of y* sum v, whose law
//      (1 - e^-t)^k is the one derived in Sec. 2.3 (Time Complexity).  T plays
//      the role of FastSearch's release horizon R/(k sum v) (Eq. exiri): every
//      arrival <= T is generated, nothing above it.
//   2. light path: every lane owns one element at a time and walks its
//      ascending arrival stream (Eq. biz_biz-1) until an arrival exceeds T
//      (FastPrune's stopping rule); when its element is done it takes the next
//      one from the row's pool, so lanes stay busy while streams differ in
//      length.  The Fisher-Yates state is a small per-lane map of displaced
//      positions in shared memory.
//   3. heavy path: elements expected to need many arrivals (or whose map
//      overflowed) are streamed by a whole warp, 32 arrivals per step, with a
//      dense permutation in shared memory and an exact shuffle scan of the
//      prefix sums.
//   4. if a register is still empty, no arrival <= T reached it: T is raised
//      and the row is redone (registers keep their values; every update is an
//      idempotent minimum).  Once every register holds an arrival <= T, each
//      holds the minimum over ALL arrivals: the result equals the full stream.
// The plain sketch runs every positive element through the heavy path with no
// bound, i.e. all k arrivals of every element (Sec. 1, straightforward method).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "gm.h"
#include "gm_device.cuh"
#include "gm_internal.h"

namespace gm {

constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;
constexpr int MAPCAP = 32;             // displaced positions a light lane can track
constexpr float HEAVY_EXPECT = 16.0f;  // expected arrivals above which an element goes to a warp

struct Counters {
  unsigned long long arrivals, elements, screened, heavy, escalated, cas;
  __device__ void zero() { arrivals = elements = screened = heavy = escalated = cas = 0ull; }
};

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
  uint32_t* heavy;
  float q1, q2;  // normalised bounds of the first two passes (inf = no bound)
};

struct SmemScalars {
  int pool, hcount, hnext, row;
  float red_f[WARPS];
  int red_i[WARPS];
};

// --------------------------------------------------------------------------
// Warp-cooperative stream of one element: 32 consecutive arrivals per step.
// --------------------------------------------------------------------------
__device__ __forceinline__ void heavy_element(int32_t id, double v, int k, uint32_t key0, uint32_t key1,
                                              uint64_t Tbits, const double* __restrict__ ctab, Reg* regs,
                                              uint16_t* pi, int* scr, int lane, Counters& cnt,
                                              bool& gave_up) {
  const double R = __drcp_rn(v);
  for (int j = lane; j < k; j += 32) pi[j] = (uint16_t)j;
  __syncwarp();
  Fix carry = fix_zero();
  for (int z0 = 0; z0 < k; z0 += 32) {
    const int z = z0 + lane;
    const bool valid = z < k;
    Fix f = fix_zero();
    int J = z;
    if (valid) {
      const Words wd = philox((uint32_t)id, (uint32_t)z, key0, key1);
      const double u = uniform_open(wd.w0, wd.w1);
      const double t = __dmul_rn(-log(u), __ldg(ctab + z));
      f = fix_from(t);
      J = randint(wd.w2, wd.w3, z, k);
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      Fix g;
      g.w0 = __shfl_up_sync(FULL, f.w0, d);
      g.w1 = __shfl_up_sync(FULL, f.w1, d);
      g.w2 = __shfl_up_sync(FULL, f.w2, d);
      if (lane >= d) fix_add(f, g);
    }
    fix_add(f, carry);
    const double S = fix_round(f);
    const uint64_t bb = (uint64_t)__double_as_longlong(__dmul_rn(S, R));
    const bool keep = valid && bb <= Tbits;
    const uint32_t km = __ballot_sync(FULL, keep);
    const int nkeep = (km == FULL) ? 32 : (__ffs(~km) - 1);  // arrivals ascend: keep is a prefix
    if (lane == 0) cnt.arrivals += (unsigned long long)min(32, k - z0);
    scr[lane] = J;
    __syncwarp();
    if (lane == 0) {
      for (int l = 0; l < nkeep; ++l) {  // Fisher-Yates steps z0 .. z0+nkeep-1, in order
        const int p = z0 + l, j = scr[l];
        const uint16_t a = pi[p];
        const uint16_t c = pi[j];
        pi[j] = a;
        scr[l] = c;
      }
    }
    __syncwarp();
    if (lane < nkeep) cnt.cas += reg_lower(smem_addr(&regs[scr[lane]]), bb, (uint64_t)(uint32_t)id, gave_up);
    carry.w0 = __shfl_sync(FULL, f.w0, 31);
    carry.w1 = __shfl_sync(FULL, f.w1, 31);
    carry.w2 = __shfl_sync(FULL, f.w2, 31);
    __syncwarp();
    if (nkeep < 32) break;
  }
}

__device__ __forceinline__ bool positive_finite(double v) {
  const int64_t b = (int64_t)__double_as_longlong(v);
  return b > 0 && (uint64_t)b < INF_BITS;
}

// --------------------------------------------------------------------------
// Light path: lanes walk their own element's stream, refilling from the pool.
// --------------------------------------------------------------------------
__device__ __forceinline__ void light_phase(const SketchArgs& a, int64_t lo, int n, uint64_t Tbits, float Tf,
                                            Reg* regs, uint32_t* map, SmemScalars& sh, Counters& cnt,
                                            bool& gave_up) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int k = a.k;
  const float kf = (float)k;
  int e = -1, z = 0, msize = 0;
  int32_t id = 0;
  double R = 0.0;
  Fix acc = fix_zero();
  bool pool_done = false;
  while (true) {
    const bool need = (e < 0) && !pool_done;
    const uint32_t nmask = __ballot_sync(FULL, need);
    if (nmask) {
      const int leader = __ffs(nmask) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(&sh.pool, __popc(nmask));
      base = __shfl_sync(FULL, base, leader);
      if (need) {
        const int slot = base + __popc(nmask & lanemask_lt());
        if (slot >= n) {
          pool_done = true;
        } else {
          const int64_t g = lo + slot;
          const double v = a.w[g];
          if (positive_finite(v)) {
            ++cnt.elements;
            const float lam = kf * (1.0f - __expf(-f32_trunc(v) * Tf));
            if (lam > HEAVY_EXPECT) {
              a.heavy[lo + atomicAdd(&sh.hcount, 1)] = (uint32_t)slot;
            } else {
              e = slot;
              id = a.ids[g];
              R = __drcp_rn(v);
              z = 0;
              acc = fix_zero();
              msize = 0;
            }
          }
        }
      }
    }
    const bool active = e >= 0;
    if (!__any_sync(FULL, active || !pool_done)) break;
    if (!active) continue;
    const Words wd = philox((uint32_t)id, (uint32_t)z, a.key0, a.key1);
    const double u = uniform_open(wd.w0, wd.w1);
    const double t = __dmul_rn(-log(u), __ldg(a.ctab + z));
    fix_add(acc, fix_from(t));
    const double S = fix_round(acc);
    const uint64_t bb = (uint64_t)__double_as_longlong(__dmul_rn(S, R));
    ++cnt.arrivals;
    if (bb > Tbits) {  // FastPrune: the rest of this stream is above the bound
      if (z == 0) ++cnt.screened;
      e = -1;
      continue;
    }
    const int J = randint(wd.w2, wd.w3, z, k);
    // Fisher-Yates step z on the sparse map (positions < z are final and dropped)
    int iz = -1;
    for (int i = 0; i < msize; ++i)
      if ((map[i * BLOCK + tid] >> 16) == (uint32_t)z) {
        iz = i;
        break;
      }
    uint32_t vz = (uint32_t)z;
    if (iz >= 0) {
      vz = map[iz * BLOCK + tid] & 0xFFFFu;
      --msize;
      map[iz * BLOCK + tid] = map[msize * BLOCK + tid];
    }
    uint32_t c = vz;
    bool overflow = false;
    if (J != z) {
      int ij = -1;
      for (int i = 0; i < msize; ++i)
        if ((map[i * BLOCK + tid] >> 16) == (uint32_t)J) {
          ij = i;
          break;
        }
      if (ij >= 0) {
        c = map[ij * BLOCK + tid] & 0xFFFFu;
        map[ij * BLOCK + tid] = ((uint32_t)J << 16) | vz;
      } else {
        c = (uint32_t)J;
        if (msize >= MAPCAP) {
          overflow = true;
        } else {
          map[msize * BLOCK + tid] = ((uint32_t)J << 16) | vz;
          ++msize;
        }
      }
    }
    if (overflow) {  // restart this element on the warp path (updates are idempotent)
      a.heavy[lo + atomicAdd(&sh.hcount, 1)] = (uint32_t)e;
      e = -1;
      continue;
    }
    cnt.cas += reg_lower(smem_addr(&regs[c]), bb, (uint64_t)(uint32_t)id, gave_up);
    if (++z >= k) e = -1;
  }
}

__device__ __forceinline__ void init_regs(Reg* regs, int k) {
  for (int j = threadIdx.x; j < k; j += BLOCK) {
    regs[j].y = INF_BITS;
    regs[j].id = UNFILLED_ID;
  }
}

__device__ __forceinline__ void write_row(const SketchArgs& a, int row, const Reg* regs) {
  const int k = a.k;
  int32_t* s = a.s_out + (int64_t)row * k;
  double* y = a.y_out + (int64_t)row * k;
  for (int j = threadIdx.x; j < k; j += BLOCK) {
    const Reg r = regs[j];
    s[j] = (r.id == UNFILLED_ID) ? -1 : (int32_t)r.id;
    y[j] = __longlong_as_double((long long)r.y);
  }
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

// Sum of the positive weights (FP32, from bits) and the count of positives.
__device__ __forceinline__ void row_sum(const SketchArgs& a, int64_t lo, int n, SmemScalars& sh, float& sum,
                                        int& npos) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float s = 0.0f, comp = 0.0f;
  int c = 0;
  bool bad = false;
  for (int i = tid; i < n; i += BLOCK) {
    const double v = a.w[lo + i];
    if (positive_finite(v)) {
      const float y = f32_trunc(v) - comp;  // Kahan
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
    sh.red_f[warp] = s;
    sh.red_i[warp] = c;
  }
  __syncthreads();
  float ts = 0.0f;
  int tc = 0;
  for (int q = 0; q < WARPS; ++q) {
    ts += sh.red_f[q];
    tc += sh.red_i[q];
  }
  sum = ts;
  npos = tc;
  __syncthreads();
}

__device__ __forceinline__ void flush_counters(const SketchArgs& a, Counters& cnt, bool gave_up) {
  const int lane = threadIdx.x & 31;
  unsigned long long v[6] = {cnt.arrivals, cnt.elements, cnt.screened, cnt.heavy, cnt.escalated, cnt.cas};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v[q] += __shfl_xor_sync(FULL, v[q], d);
    if (lane == 0 && v[q]) atomicAdd(&a.hdr->counters[q], v[q]);
  }
  if (gave_up) atomicOr(&a.hdr->status, WS_ETIMEOUT);
}

template <bool PLAIN>
__global__ void __launch_bounds__(BLOCK) sketch_kernel(SketchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SmemScalars sh;
  const int k = a.k;
  Reg* regs = reinterpret_cast<Reg*>(smem);
  unsigned char* area = smem + (size_t)k * sizeof(Reg);
  const size_t area_bytes = area_size_bytes(k);
  int* scratch = reinterpret_cast<int*>(area + area_bytes);
  uint32_t* map = reinterpret_cast<uint32_t*>(area);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint16_t* pi = reinterpret_cast<uint16_t*>(area) + (size_t)warp * k;
  int* scr = scratch + warp * 32;
  Counters cnt;
  cnt.zero();
  bool gave_up = false;

  while (true) {
    if (tid == 0) sh.row = (int)atomicAdd(&a.hdr->row_counter, 1u);
    __syncthreads();
    const int row = sh.row;
    if (row >= a.n_rows) break;
    int64_t lo, hi;
    row_bounds(a, row, lo, hi);
    const int n = (int)(hi - lo);
    init_regs(regs, k);
    float sumv;
    int npos;
    row_sum(a, lo, n, sh, sumv, npos);  // contains __syncthreads

    if constexpr (PLAIN) {
      if (tid == 0) sh.pool = 0;
      __syncthreads();
      while (true) {
        int slot = 0;
        if (lane == 0) slot = atomicAdd(&sh.pool, 1);
        slot = __shfl_sync(FULL, slot, 0);
        if (slot >= n) break;
        const double v = a.w[lo + slot];
        if (!positive_finite(v)) continue;
        if (lane == 0) ++cnt.elements;
        heavy_element(a.ids[lo + slot], v, k, a.key0, a.key1, DBL_MAX_BITS, a.ctab, regs, pi, scr, lane, cnt,
                      gave_up);
      }
      __syncthreads();
      write_row(a, row, regs);
      __syncthreads();
    } else {
    // FastGM: passes with a growing bound until every register is filled
    for (int pass = 0;; ++pass) {
      float Tf;
      uint64_t Tbits;
      if (npos == 0) break;
      const float q = pass == 0 ? a.q1 : a.q2;
      Tf = q / sumv;
      double Td = 0.0;
      bool last = !(Tf < 3.0e38f) || pass >= 12;
      if (!last) {
        Td = f64_from_f32(Tf);
        for (int p = 1; p < pass; ++p) {  // passes >= 2 widen the bound by 16x each
          Td *= 16.0;
          Tf = fminf(Tf * 16.0f, 3.0e38f);
        }
        if (!(Td < 1.0e300)) last = true;
      }
      Tbits = last ? DBL_MAX_BITS : (uint64_t)__double_as_longlong(Td);
      if (last) Tf = 3.0e38f;
      if (tid == 0) {
        sh.pool = 0;
        sh.hcount = 0;
        sh.hnext = 0;
      }
      __syncthreads();
      light_phase(a, lo, n, Tbits, Tf, regs, map, sh, cnt, gave_up);
      __syncthreads();
      const int nh = sh.hcount;
      while (true) {
        int h = 0;
        if (lane == 0) h = atomicAdd(&sh.hnext, 1);
        h = __shfl_sync(FULL, h, 0);
        if (h >= nh) break;
        const int slot = (int)a.heavy[lo + h];
        if (lane == 0) ++cnt.heavy;
        heavy_element(a.ids[lo + slot], a.w[lo + slot], k, a.key0, a.key1, Tbits, a.ctab, regs, pi, scr, lane,
                      cnt, gave_up);
      }
      __syncthreads();
      int empty = 0;
      for (int j = tid; j < k; j += BLOCK) empty |= (regs[j].y == INF_BITS);
      const int any_empty = __syncthreads_or(empty);
      if (!any_empty || last) break;
      if (tid == 0) ++cnt.escalated;
    }
    write_row(a, row, regs);
    __syncthreads();
    }
  }
  flush_counters(a, cnt, gave_up);
}

// C_z = RN(1 / (k - z)); zero the header; check the row_ptr end points.
__global__ void init_kernel(WsHeader* hdr, double* ctab, int k, const int64_t* row_ptr, int n_rows, int64_t nnz,
                            uint32_t flags) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < k) ctab[z] = __drcp_rn((double)(k - z));
  if (z == 0) {
    hdr->status = 0u;
    hdr->row_counter = 0u;
    for (int q = 0; q < WS_NCOUNTERS; ++q) hdr->counters[q] = 0ull;
    if ((flags & GM_FLAG_VALIDATE) && (row_ptr[0] != 0 || row_ptr[n_rows] != nnz)) hdr->status |= WS_EDATA;
  }
}

size_t smem_bytes(int k) { return (size_t)k * sizeof(Reg) + area_size_bytes(k) + (size_t)WARPS * 32 * sizeof(int); }

static double quantile_bound(double p, int k) {
  // (1 - p) quantile of max of k iid Exp(1):  -ln(1 - (1 - p)^(1/k))
  return -std::log(-std::expm1(std::log1p(-p) / (double)k));
}

int launch_sketch(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                  int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
                  size_t workspace_bytes, cudaStream_t stream, bool plain) {
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K) return GM_EINVAL;
  if (nnz > 0x7FFFFFFFll) return GM_EINVAL;
  if (!workspace || !row_ptr || (n_rows > 0 && (!s_out || !y_out)) || (nnz > 0 && (!ids || !w)))
    return GM_EINVAL;
  const uint32_t bound = flags & GM_BOUND_MASK;
  if (!plain && bound == GM_BOUND_LEARNED) return GM_EINVAL;  // needs gm_sketch_bounds
  const size_t need = gm_sketch_workspace_bytes(n_rows, nnz, k, flags);
  if (need == 0) return GM_EINVAL;
  if (workspace_bytes < need) return GM_ENOMEM;
  WsLayout L = ws_layout(workspace, nnz, k);

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
  a.heavy = L.heavy;
  if (bound == GM_BOUND_NONE) {
    a.q1 = a.q2 = INFINITY;
  } else {
    a.q1 = (float)quantile_bound(0.05, k);
    a.q2 = (float)quantile_bound(1e-6, k);
  }
  const size_t sm = smem_bytes(k);
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GM_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GM_ECUDA;
  if (plain) {
    if (cudaFuncSetAttribute(sketch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return GM_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch_kernel<true>, BLOCK, sm) != cudaSuccess)
      return GM_ECUDA;
  } else {
    if (cudaFuncSetAttribute(sketch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return GM_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch_kernel<false>, BLOCK, sm) != cudaSuccess)
      return GM_ECUDA;
  }
  if (per_sm < 1) return GM_EINVAL;
  int grid = nsm * per_sm;
  if (grid > n_rows) grid = n_rows;
  if (plain)
    sketch_kernel<true><<<grid, BLOCK, sm, stream>>>(a);
  else
    sketch_kernel<false><<<grid, BLOCK, sm, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

}  // namespace gm

extern "C" size_t gm_sketch_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k, uint32_t flags) {
  (void)flags;
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K) return 0;
  return gm::ws_bytes(nnz, k);
}

extern "C" int gm_sketch(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                         int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
                         size_t workspace_bytes, void* stream) {
  return gm::launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, workspace, workspace_bytes,
                           (cudaStream_t)stream, false);
}

extern "C" int gm_sketch_plain(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                               int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out,
                               double* y_out, void* workspace, size_t workspace_bytes, void* stream) {
  return gm::launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, flags & GM_FLAG_VALIDATE, s_out, y_out,
                           workspace, workspace_bytes, (cudaStream_t)stream, true);
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
// cudaGetSymbolAddress once per device (with that device current) and cached.
// ---------------------------------------------------------------------------
#include <mutex>

namespace gm {

constexpr size_t NOALLOC_SCRATCH_BYTES =
    WS_HEADER_BYTES + ((size_t)GM_MAX_K * 8 + 255) / 256 * 256 + ((size_t)GM_NOALLOC_MAX_NNZ * 4 + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_noalloc_mutex;

// Device address of g_noalloc_scratch on the current device (looked up once).
static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return GM_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
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
  if (nnz > GM_NOALLOC_MAX_NNZ) return GM_ENOMEM;  // the fixed scratch is too small for this input
  if (flags & GM_FLAG_VALIDATE) return GM_EINVAL;  // no way to read a device status back
  const size_t need = gm_sketch_workspace_bytes(n_rows, nnz, k, flags);
  if (need == 0) return GM_EINVAL;
  if (need > gm::NOALLOC_SCRATCH_BYTES) return GM_ENOMEM;
  void* scratch = nullptr;
  const int rc = gm::noalloc_scratch(&scratch);
  if (rc != GM_OK) return rc;
  // The first kernel of every call zeroes the scratch header (status, row counter,
  // counters) and rewrites the 1/(k-z) table; the heavy list is written before it
  // is read.  No other state carries over from the previous call.
  return gm::launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, flags, s_out, y_out, scratch,
                           gm::NOALLOC_SCRATCH_BYTES, (cudaStream_t)stream, false);
}
