// gm_model.cu -- the learned first-pass bound: per-row features, an
// 8 -> 64 -> 64 -> 1 GELU MLP with its own forward, backward and Adam kernels,
// and gm_sketch_learned, which runs features and inference ahead of the sketch.
//
// The paper finds the release horizon of FastGM by FastSearch (Sec. 2.2): more
// arrivals are released until every register is filled.  Any horizon T gives
// the same registers as long as the rows whose registers are not all filled by
// T are redone with a wider one, so T only decides the work.  Here a network
// predicts ln y* (the largest register) of each row; exp(prediction + margin)
// is the row's first-pass bound.  y* Sum(v) has the law of the largest of k
// independent Exp(1) variables whatever the weights, so the best such network
// reproduces the closed-form quantile bound: it is an honest ablation of it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "gm.h"
#include "gm_device.cuh"
#include "gm_internal.h"
#include "gm_trace.h"

namespace gm {
namespace mlp {

constexpr int F = GM_MODEL_FEATURES;
constexpr int H = GM_MODEL_HIDDEN;
constexpr int P = GM_MODEL_PARAMS;
static_assert(H == 64, "a warp holds the hidden layers as two 32-wide halves");

// Parameter vector (global): W1[H][F] b1[H] W2[H][H] b2[H] w3[H] b3.
constexpr int G_W1 = 0, G_B1 = G_W1 + H * F, G_W2 = G_B1 + H, G_B2 = G_W2 + H * H, G_W3 = G_B2 + H,
              G_B3 = G_W3 + H;
static_assert(G_B3 + 1 == P, "parameter layout");

// Shared copy with padded rows: a lane reading row j of W1 (stride 9) or row i /
// column j of W2 (stride 65) hits 32 different banks.
constexpr int W1S = F + 1, W2S = H + 1;
constexpr int S_W1 = 0, S_B1 = S_W1 + H * W1S, S_W2 = S_B1 + H, S_B2 = S_W2 + H * W2S, S_W3 = S_B2 + H,
              S_B3 = S_W3 + H, S_TOTAL = S_B3 + 1;
constexpr size_t PARAM_SMEM = ((size_t)S_TOTAL * 4 + 15) / 16 * 16;

constexpr int NT = 256;  // threads of every model kernel
constexpr int NW = NT / 32;

__device__ __forceinline__ int shared_index(int p) {
  if (p < G_B1) return S_W1 + (p / F) * W1S + p % F;
  if (p < G_W2) return S_B1 + (p - G_B1);
  if (p < G_B2) return S_W2 + ((p - G_W2) / H) * W2S + (p - G_W2) % H;
  return S_B2 + (p - G_B2);  // b2, w3, b3 are contiguous in both layouts
}

__device__ __forceinline__ void load_params(const float* __restrict__ g, float* s) {
  for (int p = threadIdx.x; p < P; p += blockDim.x) s[shared_index(p)] = __ldg(&g[p]);
}

// GELU, erf form: x Phi(x); its derivative Phi(x) + x phi(x).
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  return cdf + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}

// Activations a warp keeps for one sample: lane l holds hidden units l and l+32.
struct Act {
  float a1[2], a2[2], h2[2];
  float out;  // network output (before the -ln Sum(v) skip)
};

// Forward pass of one sample by one warp.  x: the 8 features (every lane);
// h1: 64 floats of shared memory that receive the first hidden layer.
__device__ __forceinline__ void warp_forward(const float* sp, const float (&x)[F], float* h1, Act& A) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = lane + 32 * q;
    float a = sp[S_B1 + j];
#pragma unroll
    for (int f = 0; f < F; ++f) a = fmaf(sp[S_W1 + j * W1S + f], x[f], a);
    A.a1[q] = a;
    h1[j] = gelu(a);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int i = lane + 32 * q;
    const float* row = sp + S_W2 + i * W2S;
    float a = sp[S_B2 + i];
#pragma unroll 16
    for (int j = 0; j < H; ++j) a = fmaf(row[j], h1[j], a);
    A.a2[q] = a;
    A.h2[q] = gelu(a);
  }
  A.out = warp_sum(sp[S_W3 + lane] * A.h2[0] + sp[S_W3 + lane + 32] * A.h2[1]) + sp[S_B3];
}

// Backward pass of one sample from dL/dout = g.  Writes dL/da2 into da2 and
// dL/da1 into da1 (64 shared floats each).
__device__ __forceinline__ void warp_backward(const float* sp, const Act& A, float g, float* da2, float* da1) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int i = lane + 32 * q;
    da2[i] = g * sp[S_W3 + i] * gelu_grad(A.a2[q]);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = lane + 32 * q;
    float d = 0.0f;
#pragma unroll 16
    for (int i = 0; i < H; ++i) d = fmaf(sp[S_W2 + i * W2S + j], da2[i], d);
    da1[j] = d * gelu_grad(A.a1[q]);
  }
}

__device__ __forceinline__ void load_x(const float* feats, int64_t i, float (&x)[F]) {
#pragma unroll
  for (int f = 0; f < F; ++f) x[f] = __ldg(&feats[i * F + f]);
}

// ---------------------------------------------------------------------------
// Row features.  Weight bins: b = floor(4 log2 v) with the quarter-octave
// boundaries 2^(j/4) taken as their nearest doubles, i.e. 4e plus the number of
// those boundaries' significands that v's significand reaches; clamped to
// [-512, 511].  Quantile p: the bin of the ceil(p n+)-th smallest weight,
// reported as the bin's centre (b + 1/2) ln2 / 4.
// ---------------------------------------------------------------------------
constexpr int NBINS = 1024, BIN_MIN = -512;
constexpr uint64_t QTR_SIG1 = 0x306fe0a31b715ull;  // significand field of RN(2^(1/4))
constexpr uint64_t QTR_SIG2 = 0x6a09e667f3bcdull;  // RN(2^(1/2))
constexpr uint64_t QTR_SIG3 = 0xae89f995ad3adull;  // RN(2^(3/4))
__device__ __forceinline__ int quant_pct(int qi) { return qi == 0 ? 10 : qi == 1 ? 50 : qi == 2 ? 90 : 99; }

__device__ __forceinline__ int weight_bin(uint64_t bits) {
  const int e = (int)(bits >> 52) - 1023;
  const uint64_t m = bits & 0x000FFFFFFFFFFFFFull;
  int b = 4 * e + (m >= QTR_SIG1) + (m >= QTR_SIG2) + (m >= QTR_SIG3);
  if (e == -1023) b = BIN_MIN;  // subnormal
  return b < BIN_MIN ? BIN_MIN : (b > BIN_MIN + NBINS - 1 ? BIN_MIN + NBINS - 1 : b);
}

struct FeatSmem {
  int hist[NW][NBINS];  // one histogram per warp: a warp's own row, or a share of a long row
  float feat[NW][F];
  int red_i[NW];
  double red_s[NW];
  unsigned long long red_m[NW];
  int scan[NW];
  int qbin[4];
};

// Accumulate elements [lo, hi) with stride `stride` from `first` into (np, sum,
// max bits, histogram); eight loads in flight per thread (a warp streaming a row
// alone waits on HBM latency once per eight elements per lane).  The sum is in
// FP64: one add per element on the FP64 pipe, which nothing else here uses.
__device__ __forceinline__ void feat_scan(const double* __restrict__ w, int64_t first, int64_t hi, int stride,
                                          int* hist, int& np, double& acc, uint64_t& mxb) {
  constexpr int U = 8;
  for (int64_t base = first; base < hi; base += (int64_t)U * stride) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + (int64_t)u * stride;
      v[u] = i < hi ? __ldg(&w[i]) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t b = (uint64_t)__double_as_longlong(v[u]);
      if (b > 0ull && b < INF_BITS) {  // positive and finite
        ++np;
        acc += v[u];
        mxb = b > mxb ? b : mxb;
        atomicAdd(&hist[weight_bin(b) - BIN_MIN], 1);
      }
    }
  }
}

// The eight features from (np, sum, max, quantile bins), one per lane of a warp
// (lanes 0 .. 7; every lane passes the same np, sum, mxb, qbin): the four FP64
// logarithms run in one pass over the warp, as a warp's FP64 instruction costs
// the same with one active lane as with four.
__device__ __forceinline__ void warp_write_features(int np, double sum, uint64_t mxb, const int* qbin, int k,
                                                    float* feat) {
  const int lane = threadIdx.x & 31;
  if (lane >= F) return;
  float f = 0.0f;
  if (lane >= 3 && lane < 7) {
    const int qb = lane == 3 ? qbin[0] : (lane == 4 ? qbin[1] : (lane == 5 ? qbin[2] : qbin[3]));
    if (np > 0) f = (float)(((double)qb + 0.5) * (0.69314718055994531 / 4.0));
  } else if (np > 0 || lane == 7) {
    const double x = lane == 0 ? (double)np
                               : (lane == 1 ? sum : (lane == 2 ? __longlong_as_double((long long)mxb) : (double)k));
    f = (float)log(x);
  }
  feat[lane] = f;
}

__device__ __forceinline__ long long quant_rank(int np, int qi) {
  const long long r = ((long long)np * quant_pct(qi) + 99) / 100;
  return r < 1 ? 1 : r;
}

// The four quantile bins of a histogram by one warp (lane l owns bins
// [32 l, 32 l + 32)); every lane returns them.  hist: shared or global.
__device__ __forceinline__ void warp_quantiles(const int* hist, int np, int (&qbin)[4]) {
  const int lane = threadIdx.x & 31;
  constexpr int PER = NBINS / 32;
  int own = 0;
  for (int q = 0; q < PER; ++q) own += hist[PER * lane + q];
  int incl = own;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += y;
  }
#pragma unroll
  for (int qi = 0; qi < 4; ++qi) {
    const long long r = quant_rank(np, qi);
    int bin = 0, c = incl - own;
    bool found = false;  // (bins are signed: found is a flag of its own)
    if (np > 0 && c < r && incl >= r)
      for (int q = 0; q < PER; ++q) {
        c += hist[PER * lane + q];
        if (c >= r) {
          bin = BIN_MIN + PER * lane + q;
          found = true;
          break;
        }
      }
    const uint32_t who = __ballot_sync(FULL, found);
    qbin[qi] = who ? __shfl_sync(FULL, bin, __ffs(who) - 1) : 0;
  }
}

// Features of row [lo, hi) by one warp (rows of up to WARP_ROW_MAX elements):
// no block barrier.  hist: the warp's NBINS counters; feat: its 8 floats.
constexpr int64_t WARP_ROW_MAX = 2048;
// The statistics of row [lo, hi) by one warp: positive count, sum, max bits and
// the four quantile bins (every lane returns them).  hist: the warp's NBINS counters.
__device__ __forceinline__ void warp_row_stats(const double* __restrict__ w, int64_t lo, int64_t hi, int* hist,
                                               int& np, double& sum, uint64_t& mxb, int (&qbin)[4]) {
  const int lane = threadIdx.x & 31;
  for (int b = lane; b < NBINS; b += 32) hist[b] = 0;
  __syncwarp();
  np = 0;
  double acc = 0.0;
  mxb = 0ull;
  feat_scan(w, lo + lane, hi, 32, hist, np, acc, mxb);
  sum = acc;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    np += __shfl_xor_sync(FULL, np, d);
    sum += __shfl_xor_sync(FULL, sum, d);
    const uint64_t o = __shfl_xor_sync(FULL, mxb, d);
    mxb = o > mxb ? o : mxb;
  }
  __syncwarp();
  warp_quantiles(hist, np, qbin);
}

__device__ void warp_row_features(const double* __restrict__ w, int64_t lo, int64_t hi, int k, int* hist,
                                  float* feat) {
  int np, qbin[4];
  double sum;
  uint64_t mxb;
  warp_row_stats(w, lo, hi, hist, np, sum, mxb, qbin);
  warp_write_features(np, sum, mxb, qbin, k, feat);
  __syncwarp();
}

// Features of a long row by the whole block (per-warp histograms).
__device__ void block_row_features(const double* __restrict__ w, int64_t lo, int64_t hi, int k, FeatSmem& sm,
                                   float* feat) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int b = tid; b < NW * NBINS; b += NT) (&sm.hist[0][0])[b] = 0;
  __syncthreads();
  int np = 0;
  double acc = 0.0;
  uint64_t mxb = 0ull;
  feat_scan(w, lo + tid, hi, NT, sm.hist[warp], np, acc, mxb);
  double sum = acc;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    np += __shfl_xor_sync(FULL, np, d);
    sum += __shfl_xor_sync(FULL, sum, d);
    const uint64_t o = __shfl_xor_sync(FULL, mxb, d);
    mxb = o > mxb ? o : mxb;
  }
  if (lane == 0) {
    sm.red_i[warp] = np;
    sm.red_s[warp] = sum;
    sm.red_m[warp] = mxb;
  }
  __syncthreads();
  np = 0;
  sum = 0.0;
  mxb = 0ull;
  for (int q = 0; q < NW; ++q) {
    np += sm.red_i[q];
    sum += sm.red_s[q];
    mxb = sm.red_m[q] > mxb ? sm.red_m[q] : mxb;
  }
  // exclusive scan of the merged histogram: thread t owns bins 4t .. 4t+3
  static_assert(NBINS == 4 * NT, "four bins per thread");
  int cnt4[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int c = 0;
#pragma unroll
    for (int w8 = 0; w8 < NW; ++w8) c += sm.hist[w8][4 * tid + q];
    cnt4[q] = c;
  }
  const int own = cnt4[0] + cnt4[1] + cnt4[2] + cnt4[3];
  int incl = own;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) sm.scan[warp] = incl;
  __syncthreads();
  int run = incl - own;
  for (int q = 0; q < warp; ++q) run += sm.scan[q];
#pragma unroll
  for (int qi = 0; qi < 4; ++qi) {
    const long long r = quant_rank(np, qi);
    int c = run;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int before = c;
      c += cnt4[q];
      if (np > 0 && before < r && c >= r) sm.qbin[qi] = BIN_MIN + 4 * tid + q;
    }
  }
  __syncthreads();
  if (tid < 32) warp_write_features(np, sum, mxb, sm.qbin, k, feat);
  __syncthreads();
}

__device__ __forceinline__ void clamp_row(const int64_t* row_ptr, int r, int64_t nnz, int64_t& lo, int64_t& hi) {
  int64_t l = row_ptr[r], h = row_ptr[r + 1];
  l = l < 0 ? 0 : (l > nnz ? nnz : l);
  h = h < l ? l : (h > nnz ? nnz : h);
  lo = l;
  hi = h;
}

// Rows of up to WARP_ROW_MAX elements go to warps (global warp index, strided),
// longer rows to whole blocks; `emit(row, feat)` runs in the warp (or warp 0 of
// the block) that computed them.
template <class EMIT>
__device__ __forceinline__ void for_each_row_features(const int64_t* row_ptr, const double* w, int n_rows,
                                                      int64_t nnz, int k, FeatSmem& sm, EMIT emit) {
  const int warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * NW + warp, nw = (int64_t)gridDim.x * NW;
  for (int64_t r = gw; r < n_rows; r += nw) {
    int64_t lo, hi;
    clamp_row(row_ptr, (int)r, nnz, lo, hi);
    if (hi - lo > WARP_ROW_MAX) continue;
    warp_row_features(w, lo, hi, k, sm.hist[warp], sm.feat[warp]);
    emit((int)r, sm.feat[warp]);
  }
  __syncthreads();
  for (int r = blockIdx.x; r < n_rows; r += gridDim.x) {
    int64_t lo, hi;
    clamp_row(row_ptr, r, nnz, lo, hi);
    if (hi - lo <= WARP_ROW_MAX) continue;  // uniform over the block
    block_row_features(w, lo, hi, k, sm, sm.feat[0]);
    if (warp == 0) emit(r, sm.feat[0]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(NT) features_kernel(const int64_t* row_ptr, const double* w, int n_rows,
                                                      int64_t nnz, int k, float* feats) {
  __shared__ FeatSmem sm;
  for_each_row_features(row_ptr, w, n_rows, nnz, k, sm, [&](int r, const float* feat) {
    const int lane = threadIdx.x & 31;
    if (lane < F) feats[(int64_t)r * F + lane] = feat[lane];
  });
}

// ---------------------------------------------------------------------------
// The learned bound of a batch.  Rows of up to WARP_ROW_MAX elements are done by
// one warp each (features, network, bound: learned_short_kernel).  Longer rows
// are listed and cut into PIECE-element pieces, one warp's task each, spread over
// the whole grid (learned_piece_kernel: per-piece counts, sums and maxima,
// histograms added with integer atomics); then one warp per long row adds its
// pieces' partials in a fixed order and finishes it (learned_long_kernel).  The
// result is the same bits every run.
// ---------------------------------------------------------------------------
constexpr int64_t PIECE = 2048;  // elements per piece of a long row: one warp's task

struct LongHdr {
  unsigned long long n_long, n_pieces;  // 64-bit: no wrap even for overlapping (invalid) rows
};
struct LongEnt {
  int row, piece_off, n_pieces, pad;
};
struct PiecePart {
  int np, pad;
  double sum;
  unsigned long long mxb;
};
struct RowStats {  // a row's feature statistics, before the logarithms
  int np;         // positive weights; -1: the row has no learned bound (overlapping rows)
  int qbin[4];    // quantile bins
  int pad;
  double sum;
  unsigned long long mxb;  // bits of the largest weight
};
struct LearnedWs {
  LongHdr* hdr;
  LongEnt* longs;
  int* piece_row;
  int* hist;  // NBINS per long row
  PiecePart* parts;
  RowStats* stats;  // per row
  long long max_long, max_pieces;  // capacities (never reached by valid row offsets)
};

static int64_t learned_max_long(int64_t nnz) { return nnz / (WARP_ROW_MAX + 1) + 1; }
static int64_t learned_max_pieces(int64_t nnz) { return nnz / PIECE + learned_max_long(nnz); }
static size_t learned_ws_bytes(int32_t n_rows, int64_t nnz) {
  const int64_t ml = learned_max_long(nnz), mp = learned_max_pieces(nnz);
  return 256 + round_up((size_t)ml * sizeof(LongEnt), 256) + round_up((size_t)mp * 4, 256) +
         round_up((size_t)ml * NBINS * 4, 256) + round_up((size_t)mp * sizeof(PiecePart), 256) +
         round_up((size_t)n_rows * sizeof(RowStats), 256);
}
static LearnedWs learned_ws(unsigned char* p, int32_t n_rows, int64_t nnz) {
  const int64_t ml = learned_max_long(nnz), mp = learned_max_pieces(nnz);
  LearnedWs L;
  L.hdr = reinterpret_cast<LongHdr*>(p);
  p += 256;
  L.longs = reinterpret_cast<LongEnt*>(p);
  p += round_up((size_t)ml * sizeof(LongEnt), 256);
  L.piece_row = reinterpret_cast<int*>(p);
  p += round_up((size_t)mp * 4, 256);
  L.hist = reinterpret_cast<int*>(p);
  p += round_up((size_t)ml * NBINS * 4, 256);
  L.parts = reinterpret_cast<PiecePart*>(p);
  p += round_up((size_t)mp * sizeof(PiecePart), 256);
  L.stats = reinterpret_cast<RowStats*>(p);
  L.max_long = ml;
  L.max_pieces = mp;
  return L;
}

// The network on a warp's features, then the row's first-pass bound
// T = exp(ln y* prediction + margin), made a positive normal float (or +inf).
__device__ __forceinline__ void warp_emit_bound(const float* sp, const float* feat, float* h1w, float margin,
                                                float* t_row, int r) {
  float x[F];
#pragma unroll
  for (int f = 0; f < F; ++f) x[f] = feat[f];
  Act A;
  warp_forward(sp, x, h1w, A);
  if ((threadIdx.x & 31) == 0) {
    float T = expf(A.out - x[1] + margin);
    if (!(T >= 1.0e-37f)) T = 1.0e-37f;  // tiny or NaN: the first pass fails, later passes are closed-form
    if (!(T < 3.0e38f)) T = __int_as_float(0x7F800000);
    t_row[r] = T;
  }
  __syncwarp();
}

__device__ __forceinline__ void put_stats(RowStats* st, int np, double sum, uint64_t mxb, const int (&qbin)[4]) {
  RowStats x;
  x.np = np;
  x.qbin[0] = qbin[0];
  x.qbin[1] = qbin[1];
  x.qbin[2] = qbin[2];
  x.qbin[3] = qbin[3];
  x.pad = 0;
  x.sum = sum;
  x.mxb = mxb;
  *st = x;
}

__global__ void __launch_bounds__(NT) learned_short_kernel(const int64_t* row_ptr, const double* w, int n_rows,
                                                           int64_t nnz, LearnedWs L) {
  __shared__ int hist[NW][NBINS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * NW + warp, nw = (int64_t)gridDim.x * NW;
  for (int64_t r = gw; r < n_rows; r += nw) {
    int64_t lo, hi;
    clamp_row(row_ptr, (int)r, nnz, lo, hi);
    if (hi - lo <= WARP_ROW_MAX) {
      int np, qbin[4];
      double sum;
      uint64_t mxb;
      warp_row_stats(w, lo, hi, hist[warp], np, sum, mxb, qbin);
      if (lane == 0) put_stats(L.stats + r, np, sum, mxb, qbin);
      continue;
    }
    // a long row: list it, with its range of pieces, and clear its histogram.
    // Rows that overlap (row offsets not ascending) can overrun the lists: such
    // a row gets no learned bound (a negative T: the closed form).
    const long long np = (hi - lo + PIECE - 1) / PIECE;
    long long i = 0, off = 0;
    if (lane == 0) {
      i = (long long)atomicAdd(&L.hdr->n_long, 1ull);
      off = (long long)atomicAdd(&L.hdr->n_pieces, (unsigned long long)np);
    }
    i = __shfl_sync(FULL, i, 0);
    off = __shfl_sync(FULL, off, 0);
    const bool ok = i < L.max_long && off + np <= L.max_pieces;
    if (lane == 0) {
      if (i < L.max_long) L.longs[i] = LongEnt{ok ? (int)r : -1, (int)off, (int)np, 0};
      if (!ok) L.stats[r].np = -1;
    }
    const long long pend = min(off + np, L.max_pieces);
    for (long long g = off + lane; g < pend; g += 32) L.piece_row[g] = ok ? (int)i : -1;
    if (ok)
      for (int b = lane; b < NBINS; b += 32) L.hist[i * NBINS + b] = 0;
  }
}

__global__ void __launch_bounds__(NT) learned_piece_kernel(const int64_t* row_ptr, const double* w, int64_t nnz,
                                                           LearnedWs L) {
  __shared__ int hist[NW][NBINS];  // one histogram per warp: the warp's current piece
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long n_pieces = min((long long)L.hdr->n_pieces, L.max_pieces);
  int* h = hist[warp];
  for (long long g = (long long)blockIdx.x * NW + warp; g < n_pieces; g += (long long)gridDim.x * NW) {
    const int i = L.piece_row[g];
    if (i < 0) continue;  // uniform over the warp
    const LongEnt e = L.longs[i];
    int64_t lo, hi;
    clamp_row(row_ptr, e.row, nnz, lo, hi);
    const int64_t plo = lo + (g - e.piece_off) * PIECE;
    const int64_t phi = min(hi, plo + PIECE);
    for (int b = lane; b < NBINS; b += 32) h[b] = 0;
    __syncwarp();
    int np = 0;
    double acc = 0.0;
    uint64_t mxb = 0ull;
    feat_scan(w, plo + lane, phi, 32, h, np, acc, mxb);
    double sum = acc;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      np += __shfl_xor_sync(FULL, np, d);
      sum += __shfl_xor_sync(FULL, sum, d);
      const uint64_t o = __shfl_xor_sync(FULL, mxb, d);
      mxb = o > mxb ? o : mxb;
    }
    __syncwarp();
    for (int b = lane; b < NBINS; b += 32) {
      const int c = h[b];
      if (c) atomicAdd(&L.hist[(int64_t)i * NBINS + b], c);
    }
    if (lane == 0) {
      PiecePart pp;
      pp.np = np;
      pp.pad = 0;
      pp.sum = sum;
      pp.mxb = mxb;
      L.parts[g] = pp;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(NT) learned_long_kernel(LearnedWs L) {
  __shared__ int hist[NW][NBINS];  // the row's histogram, staged for the quantile search
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long n_long = min((long long)L.hdr->n_long, L.max_long);
  for (long long i = (long long)blockIdx.x * NW + warp; i < n_long; i += (long long)gridDim.x * NW) {
    const LongEnt e = L.longs[i];
    if (e.row < 0) continue;  // uniform over the warp
    // the pieces' partials: lane l adds pieces l, l + 32, ... in order, then a
    // butterfly; a fixed order, so the same sum every run
    int np = 0;
    double sum = 0.0;
    unsigned long long mxb = 0ull;
    for (int q = lane; q < e.n_pieces; q += 32) {
      const PiecePart pp = L.parts[e.piece_off + q];
      np += pp.np;
      sum += pp.sum;
      mxb = pp.mxb > mxb ? pp.mxb : mxb;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      np += __shfl_xor_sync(FULL, np, d);
      sum += __shfl_xor_sync(FULL, sum, d);
      const unsigned long long o = __shfl_xor_sync(FULL, mxb, d);
      mxb = o > mxb ? o : mxb;
    }
    const int4* g4 = reinterpret_cast<const int4*>(L.hist + i * NBINS);
    int4* s4 = reinterpret_cast<int4*>(hist[warp]);
    for (int b = lane; b < NBINS / 4; b += 32) s4[b] = __ldcg(g4 + b);
    __syncwarp();
    int qbin[4];
    warp_quantiles(hist[warp], np, qbin);
    if (lane == 0) put_stats(L.stats + e.row, np, sum, mxb, qbin);
    __syncwarp();
  }
}

// Features, network and bound of every row from its statistics, NW rows per CTA
// step: warp 0 takes the four logarithms of all NW rows in one pass (lane 4 q + j:
// row q, value j of ln n+, ln sum v, ln max v, ln k; then the quantile features),
// as a warp's FP64 instruction costs the same with one active lane as with 32;
// then each warp runs the network on its row.
__global__ void __launch_bounds__(NT) learned_finish_kernel(int n_rows, int k, const float* params, float margin,
                                                            float* t_row, LearnedWs L) {
  extern __shared__ __align__(16) float sp[];
  __shared__ float feat[NW][F];
  __shared__ float h1[NW][H];
  __shared__ int npq[NW];
  static_assert(NW * 4 == 32, "four values per row in one warp pass");
  load_params(params, sp);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = (int64_t)blockIdx.x * NW; base < n_rows; base += (int64_t)gridDim.x * NW) {
    if (warp == 0) {
      const int q = lane >> 2, j = lane & 3;
      const int64_t r = base + q;
      if (r < n_rows) {
        const RowStats st = L.stats[r];
        if (j == 0) npq[q] = st.np;
        if (st.np >= 0) {
          float f = 0.0f;
          if (st.np > 0 || j == 3) {
            const double x = j == 0 ? (double)st.np
                                    : (j == 1 ? st.sum : (j == 2 ? __longlong_as_double((long long)st.mxb) : (double)k));
            f = (float)log(x);
          }
          feat[q][j == 3 ? 7 : j] = f;
          const int qb = j == 0 ? st.qbin[0] : (j == 1 ? st.qbin[1] : (j == 2 ? st.qbin[2] : st.qbin[3]));
          feat[q][3 + j] = st.np > 0 ? (float)(((double)qb + 0.5) * (0.69314718055994531 / 4.0)) : 0.0f;
        }
      }
    }
    __syncthreads();
    const int64_t r = base + warp;
    if (r < n_rows) {
      if (npq[warp] >= 0)
        warp_emit_bound(sp, feat[warp], h1[warp], margin, t_row, (int)r);
      else if (lane == 0)
        t_row[r] = -1.0f;  // no learned bound: the closed form
    }
    __syncthreads();
  }
}

// ln of each row's largest register (+inf if a register is unfilled).
__global__ void ln_ystar_kernel(const double* y, int n_rows, int k, float* out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= n_rows) return;
  uint64_t m = 0ull;
  for (int j = lane; j < k; j += 32) {
    const uint64_t b = (uint64_t)__double_as_longlong(y[r * k + j]);
    m = b > m ? b : m;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const uint64_t o = __shfl_xor_sync(FULL, m, d);
    m = o > m ? o : m;
  }
  if (lane == 0) out[r] = m >= INF_BITS ? __int_as_float(0x7F800000) : (float)log(__longlong_as_double((long long)m));
}

// Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from Philox (counter = index,
// tag), biases zero.
__global__ void init_kernel(float* params, uint32_t k0, uint32_t k1) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float bound = 0.0f;
  if (p < G_B1)
    bound = 0.35355339059327376f;  // 1/sqrt(8)
  else if ((p >= G_W2 && p < G_B2) || (p >= G_W3 && p < G_B3))
    bound = 0.125f;  // 1/sqrt(64)
  const Words r = philox((uint32_t)p, 0x4D4C5031u, k0, k1);
  const float u = (float)(r.w0 >> 8) * 5.9604644775390625e-8f;  // [0, 1), 24 bits
  params[p] = bound * (2.0f * u - 1.0f);
}

__global__ void __launch_bounds__(NT) forward_kernel(const float* params, const float* feats, int n, float* out) {
  extern __shared__ __align__(16) float sp[];
  __shared__ float h1[NW][H];
  load_params(params, sp);
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * NW + warp; i < n; i += (int64_t)gridDim.x * NW) {
    float x[F];
    load_x(feats, i, x);
    Act A;
    warp_forward(sp, x, h1[warp], A);
    if ((threadIdx.x & 31) == 0) out[i] = A.out - x[1];
    __syncwarp();
  }
}

// Gradient of the mean pinball loss.  Every CTA takes a fixed contiguous range
// of samples in tiles of 32; its warps run forward and backward passes into the
// tile, then thread t sums the tile's contributions to parameters t, t+256, ...
// in sample order.  Per-CTA partials go to the workspace and a second kernel adds
// them in CTA order, so the gradient is the same bits on every run.
constexpr int TILE = 32;
constexpr int GRAD_CTAS = 304;
constexpr int PER_T = (P + NT - 1) / NT;  // 19 parameters per thread

struct Tile {
  float h1[TILE][H], h2[TILE][H], da1[TILE][H], da2[TILE][H];
  float x[TILE][F];
  float g[TILE], loss[TILE];
};
constexpr size_t GRAD_SMEM = PARAM_SMEM + sizeof(Tile);

__device__ __forceinline__ float tile_term(const Tile& t, int p, int ns) {
  float s = 0.0f;
  if (p < G_B1) {
    const int j = p / F, f = p % F;
    for (int i = 0; i < ns; ++i) s = fmaf(t.da1[i][j], t.x[i][f], s);
  } else if (p < G_W2) {
    const int j = p - G_B1;
    for (int i = 0; i < ns; ++i) s += t.da1[i][j];
  } else if (p < G_B2) {
    const int r = (p - G_W2) / H, c = (p - G_W2) % H;
    for (int i = 0; i < ns; ++i) s = fmaf(t.da2[i][r], t.h1[i][c], s);
  } else if (p < G_W3) {
    const int r = p - G_B2;
    for (int i = 0; i < ns; ++i) s += t.da2[i][r];
  } else if (p < G_B3) {
    const int r = p - G_W3;
    for (int i = 0; i < ns; ++i) s = fmaf(t.g[i], t.h2[i][r], s);
  } else {
    for (int i = 0; i < ns; ++i) s += t.g[i];
  }
  return s;
}

__global__ void __launch_bounds__(NT) grad_kernel(const float* params, const float* feats, const float* target, int n,
                                                  float tau, float* part) {
  extern __shared__ __align__(16) float sp[];
  Tile& t = *reinterpret_cast<Tile*>(reinterpret_cast<unsigned char*>(sp) + PARAM_SMEM);
  load_params(params, sp);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t per = ((int64_t)n + gridDim.x - 1) / gridDim.x;
  const int64_t s0 = (int64_t)blockIdx.x * per, s1 = min((int64_t)n, s0 + per);
  const float inv_n = 1.0f / (float)n;
  float acc[PER_T];
#pragma unroll
  for (int m = 0; m < PER_T; ++m) acc[m] = 0.0f;
  float lacc = 0.0f;
  __syncthreads();
  for (int64_t base = s0; base < s1; base += TILE) {
    const int ns = (int)min((int64_t)TILE, s1 - base);
    for (int slot = warp; slot < ns; slot += NW) {
      float x[F];
      load_x(feats, base + slot, x);
      Act A;
      warp_forward(sp, x, t.h1[slot], A);
      const float pred = A.out - x[1];
      const float r = __ldg(&target[base + slot]) - pred;
      const float gp = r > 0.0f ? -tau : 1.0f - tau;  // d loss / d pred
      const float g = gp * inv_n;
#pragma unroll
      for (int q = 0; q < 2; ++q) t.h2[slot][lane + 32 * q] = A.h2[q];
      if (lane < F) t.x[slot][lane] = __ldg(&feats[(base + slot) * F + lane]);
      if (lane == 0) {
        t.g[slot] = g;
        t.loss[slot] = r > 0.0f ? tau * r : (tau - 1.0f) * r;
      }
      warp_backward(sp, A, g, t.da2[slot], t.da1[slot]);
      __syncwarp();
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PER_T; ++m) {
      const int p = tid + NT * m;
      if (p < P) acc[m] += tile_term(t, p, ns);
    }
    if (tid == 0)
      for (int i = 0; i < ns; ++i) lacc += t.loss[i];
    __syncthreads();
  }
  float* mine = part + (int64_t)blockIdx.x * (P + 1);
#pragma unroll
  for (int m = 0; m < PER_T; ++m) {
    const int p = tid + NT * m;
    if (p < P) mine[p] = acc[m];
  }
  if (tid == 0) mine[P] = lacc;
}

__global__ void reduce_kernel(const float* part, int nparts, int n, float* grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > P) return;
  float s = 0.0f;
  for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * (P + 1) + p];
  if (p < P)
    grad[p] = s;
  else
    loss[0] = s / (float)n;
}

__global__ void adam_kernel(float* params, float* mom, const float* grad, float lr, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float g = grad[p];
  const float m = 0.9f * mom[p] + 0.1f * g;
  const float v = 0.999f * mom[P + p] + 0.001f * g * g;
  mom[p] = m;
  mom[P + p] = v;
  params[p] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
}

}  // namespace mlp
}  // namespace gm

using namespace gm;
using namespace gm::mlp;

static int finish(cudaError_t e) { return e == cudaSuccess ? GM_OK : GM_ECUDA; }

// Raise a kernel's dynamic shared memory limit to `bytes`, once per (kernel,
// device): concurrent calls never see a half-set attribute.
static int allow_smem(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GM_ECUDA;
  std::lock_guard<std::mutex> g(mu);
  if (done.count({kern, dev})) return GM_OK;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return GM_ECUDA;
  done.insert({kern, dev});
  return GM_OK;
}

static int model_grid(int n_units, int per_sm) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int g = nsm * per_sm;
  return n_units < g ? (n_units < 1 ? 1 : n_units) : g;
}

extern "C" int gm_features(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                           int32_t k, float* feats, void* stream) {
  (void)ids;
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K || !row_ptr || (n_rows > 0 && !feats) || (nnz > 0 && !w))
    return GM_EINVAL;
  if (n_rows == 0) return GM_OK;
  const int grid = model_grid(n_rows, 8);
  if (grid < 1) return GM_ECUDA;
  features_kernel<<<grid, NT, 0, (cudaStream_t)stream>>>(row_ptr, w, n_rows, nnz, k, feats);
  return finish(cudaGetLastError());
}

extern "C" int gm_row_ln_ystar(const double* y, int32_t n_rows, int32_t k, float* ln_ystar, void* stream) {
  if (n_rows < 0 || k < 1 || (n_rows > 0 && (!y || !ln_ystar))) return GM_EINVAL;
  if (n_rows == 0) return GM_OK;
  const int64_t threads = (int64_t)n_rows * 32;
  ln_ystar_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(y, n_rows, k, ln_ystar);
  return finish(cudaGetLastError());
}

extern "C" int gm_model_init(float* params, uint64_t seed, void* stream) {
  if (!params) return GM_EINVAL;
  init_kernel<<<(P + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, (uint32_t)seed, (uint32_t)(seed >> 32));
  return finish(cudaGetLastError());
}

extern "C" int gm_model_forward(const float* params, const float* feats, int32_t n, float* out, void* stream) {
  if (n < 0 || !params || (n > 0 && (!feats || !out))) return GM_EINVAL;
  if (n == 0) return GM_OK;
  const int grid = model_grid((n + NW - 1) / NW, 4);
  if (grid < 1) return GM_ECUDA;
  forward_kernel<<<grid, NT, PARAM_SMEM, (cudaStream_t)stream>>>(params, feats, n, out);
  return finish(cudaGetLastError());
}

extern "C" size_t gm_model_grad_workspace_bytes(void) { return (size_t)GRAD_CTAS * (P + 1) * sizeof(float); }

extern "C" int gm_model_grad(const float* params, const float* feats, const float* target, int32_t n, float tau,
                             float* grad, float* loss, void* workspace, size_t workspace_bytes, void* stream) {
  if (n < 1 || !params || !feats || !target || !grad || !loss || !workspace || !ws_aligned(workspace)) return GM_EINVAL;
  if (!(tau > 0.0f && tau < 1.0f)) return GM_EINVAL;
  if (workspace_bytes < gm_model_grad_workspace_bytes()) return GM_ENOMEM;
  const gm::TraceRange trace("gm_model_grad");
  if (allow_smem((const void*)grad_kernel, GRAD_SMEM) != GM_OK)
    return GM_ECUDA;
  float* part = static_cast<float*>(workspace);
  const cudaStream_t st = (cudaStream_t)stream;
  grad_kernel<<<GRAD_CTAS, NT, GRAD_SMEM, st>>>(params, feats, target, n, tau, part);
  reduce_kernel<<<(P + 1 + 255) / 256, 256, 0, st>>>(part, GRAD_CTAS, n, grad, loss);
  return finish(cudaGetLastError());
}

extern "C" int gm_model_adam(float* params, float* adam, const float* grad, float lr, int32_t step, void* stream) {
  if (!params || !adam || !grad || step < 1 || !(lr > 0.0f)) return GM_EINVAL;
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)step));
  const float bc2 = (float)(1.0 - std::pow(0.999, (double)step));
  adam_kernel<<<(P + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, adam, grad, lr, bc1, bc2);
  return finish(cudaGetLastError());
}

static const char MODEL_MAGIC[8] = {'G', 'M', 'M', 'L', 'P', '0', '0', '1'};

extern "C" int gm_model_save(const float* params, const char* path, void* stream) {
  if (!params || !path) return GM_EINVAL;
  std::vector<float> host(P);
  const cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(host.data(), params, P * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return GM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GM_ECUDA;
  FILE* f = std::fopen(path, "wb");
  if (!f) return GM_EINVAL;
  const int32_t dims[2] = {F, H};
  const bool ok = std::fwrite(MODEL_MAGIC, 1, 8, f) == 8 && std::fwrite(dims, 4, 2, f) == 2 &&
                  std::fwrite(host.data(), sizeof(float), P, f) == (size_t)P;
  return (std::fclose(f) == 0 && ok) ? GM_OK : GM_EINVAL;
}

extern "C" int gm_model_load(float* params, const char* path, void* stream) {
  if (!params || !path) return GM_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return GM_EINVAL;
  char magic[8];
  int32_t dims[2];
  std::vector<float> host(P);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, MODEL_MAGIC, 8) == 0 &&
            std::fread(dims, 4, 2, f) == 2 && dims[0] == F && dims[1] == H &&
            std::fread(host.data(), sizeof(float), P, f) == (size_t)P;
  std::fclose(f);
  if (!ok) return GM_EDATA;
  const cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(params, host.data(), P * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return GM_ECUDA;
  return finish(cudaStreamSynchronize(st));  // the host copy dies with this call
}

extern "C" size_t gm_learned_bound_workspace_bytes(int32_t n_rows, int64_t nnz) {
  return (nnz < 0 || n_rows < 0) ? 0 : learned_ws_bytes(n_rows, nnz);
}

static int learned_bound_launch(const int64_t* row_ptr, const double* w, int32_t n_rows, int64_t nnz, int32_t k,
                                const float* params, float margin, float* t_row, void* workspace,
                                cudaStream_t st) {
  if (n_rows == 0) return GM_OK;
  const LearnedWs L = learned_ws(static_cast<unsigned char*>(workspace), n_rows, nnz);
  const int grid = model_grid(1 << 30, 4);  // a full wave: the kernels stride over their work
  if (grid < 1) return GM_ECUDA;
  if (allow_smem((const void*)learned_finish_kernel, PARAM_SMEM) != GM_OK) return GM_ECUDA;
  if (cudaMemsetAsync(L.hdr, 0, sizeof(LongHdr), st) != cudaSuccess) return GM_ECUDA;
  learned_short_kernel<<<grid, NT, 0, st>>>(row_ptr, w, n_rows, nnz, L);
  learned_piece_kernel<<<grid, NT, 0, st>>>(row_ptr, w, nnz, L);
  learned_long_kernel<<<grid, NT, 0, st>>>(L);
  const int fgrid = model_grid((n_rows + NW - 1) / NW, 4);
  if (fgrid < 1) return GM_ECUDA;
  learned_finish_kernel<<<fgrid, NT, PARAM_SMEM, st>>>(n_rows, k, params, margin, t_row, L);
  return finish(cudaGetLastError());
}

extern "C" int gm_learned_bound(const int64_t* row_ptr, const double* w, int32_t n_rows, int64_t nnz, int32_t k,
                                const float* params, float margin, float* t_out, void* workspace,
                                size_t workspace_bytes, void* stream) {
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K || nnz > 0x7FFFFFFFll) return GM_EINVAL;
  if (!params || !std::isfinite(margin) || !row_ptr || (n_rows > 0 && !t_out) || (nnz > 0 && !w) || !workspace ||
      !ws_aligned(workspace))
    return GM_EINVAL;
  if (workspace_bytes < learned_ws_bytes(n_rows, nnz)) return GM_ENOMEM;
  const gm::TraceRange trace("gm_learned_bound");
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  aux_events(&ev0, &ev1);
  if (ev0) cudaEventRecord(ev0, (cudaStream_t)stream);
  const int rc =
      learned_bound_launch(row_ptr, w, n_rows, nnz, k, params, margin, t_out, workspace, (cudaStream_t)stream);
  if (ev1) cudaEventRecord(ev1, (cudaStream_t)stream);
  return rc;
}

extern "C" size_t gm_sketch_learned_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k) {
  const size_t base = gm_sketch_workspace_bytes(n_rows, nnz, k, 0u);
  if (base == 0) return 0;
  return base + round_up((size_t)n_rows * 4, 256) + learned_ws_bytes(n_rows, nnz);
}

extern "C" int gm_sketch_learned(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                                 int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, const float* params,
                                 float margin, int32_t* s_out, double* y_out, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K || nnz > 0x7FFFFFFFll) return GM_EINVAL;
  if (!params || !std::isfinite(margin) || !workspace || !ws_aligned(workspace) || !row_ptr) return GM_EINVAL;
  const gm::TraceRange trace("gm_sketch_learned");
  const size_t base = gm_sketch_workspace_bytes(n_rows, nnz, k, 0u);
  const size_t need = gm_sketch_learned_workspace_bytes(n_rows, nnz, k);
  if (need == 0) return GM_EINVAL;
  if (workspace_bytes < need) return GM_ENOMEM;
  unsigned char* extra = static_cast<unsigned char*>(workspace) + base;
  float* t_row = reinterpret_cast<float*>(extra);
  const cudaStream_t st = (cudaStream_t)stream;
  if (n_rows > 0 && nnz > 0 && w) {
    const int rc = learned_bound_launch(row_ptr, w, n_rows, nnz, k, params, margin, t_row,
                                        extra + round_up((size_t)n_rows * 4, 256), st);
    if (rc != GM_OK) return rc;
  }
  const uint32_t f = (flags & ~(uint32_t)GM_BOUND_MASK) | GM_BOUND_CLOSED;  // later passes: closed form
  return launch_sketch(row_ptr, ids, w, n_rows, nnz, k, seed, f, s_out, y_out, workspace, base, st, false,
                       nnz > 0 ? t_row : nullptr);
}
