// gm_diag.cu -- diagnostic kernels: the per-arrival device arithmetic, exposed
// value by value for tests (see include/gm_diag.h).
#include <cuda_runtime.h>

#include "gm.h"
#include "gm_diag.h"
#include "gm_stream.cuh"

namespace gm {

template <int ARITH>
__global__ void diag_neglog_kernel(const uint64_t* __restrict__ x, int64_t n, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t v = x[i];
    Words wd{(uint32_t)v, (uint32_t)(v >> 32), 0u, 0u};
    out[i] = arr_neglog<ARITH>(wd);
  }
}

template <int ARITH>
__global__ void diag_dmul_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                 double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = arr_mul<ARITH>(a[i], b[i]);
}

template <int ARITH>
__global__ void diag_drcp_kernel(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = arr_rcp<ARITH>(v[i]);
}

__global__ void diag_ctab_kernel(double* ctab, int k) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < k) ctab[z] = __drcp_rn((double)(k - z));
}

// One warp: the warp path of the sketch kernels, writing arrivals instead of
// updating registers.
template <int ARITH, class PI>
__global__ void diag_arrivals_kernel(int32_t id, double v, int k, uint32_t key0, uint32_t key1, int n_steps,
                                     const double* __restrict__ ctab, double* b_out, int32_t* c_out) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const PI pi{reinterpret_cast<decltype(PI::member_type())>(dsm)};
  const int lane = threadIdx.x;
  const double R = arr_rcp<ARITH>(v);
  pi.reset(k, lane);
  Fix carry = fix_zero();
  for (int z0 = 0; z0 < n_steps; z0 += 32) {
    int J;
    const uint64_t bb = warp_batch<ARITH>(id, R, z0, k, key0, key1, ctab, carry, lane, J);
    const int cnt = min(32, n_steps - z0);
    int c;
    warp_fy_steps(pi, z0, J, cnt, lane, c);
    if (lane < cnt) {
      b_out[z0 + lane] = __longlong_as_double((long long)bb);
      c_out[z0 + lane] = c;
    }
  }
}

__global__ void diag_first_kernel(const int32_t* __restrict__ ids, const double* __restrict__ v, int64_t n, int k,
                                  uint32_t key0, uint32_t key1, float T, uint8_t* __restrict__ screened,
                                  double* __restrict__ b0) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Words wd = philox((uint32_t)ids[i], 0u, key0, key1);
    screened[i] = screen_out(wd.w1, f32_trunc(v[i]), T, (float)k) ? 1 : 0;
    const double C0 = drcp_pos((double)k);
    const double t = dmul_pos(neglog_u(wd.w0, wd.w1), C0);
    // a single term: the exact sum is the term itself
    b0[i] = dmul_pos(t, drcp_pos(v[i]));
  }
}

// Eight independent FMA chains per thread, `iters` steps each: the FP64 (or FP32)
// FMA rate of the device, for the arithmetic comparison in bench.py --arith.
template <typename T>
__global__ void diag_fma_kernel(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3, x4 = x0 + (T)4,
    x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// One arrival's value chain per thread, each independent: Philox, -ln u, the
// product by C_z, the exact sum (a single term), its rounding, the product by R
// and RandInt -- the algorithmic work of one arrival, for instruction counting.
template <int ARITH>
__global__ void diag_arrival_cost_kernel(const int32_t* __restrict__ ids, const double* __restrict__ R, int64_t n,
                                         int k, uint32_t key0, uint32_t key1, const double* __restrict__ ctab,
                                         double* __restrict__ out, int32_t* __restrict__ jout) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int z = (int)(i % k);
    const Words wd = philox((uint32_t)ids[i], (uint32_t)z, key0, key1);
    Fix acc = fix_zero();
    fix_add(acc, fix_from(arr_mul_t<ARITH>(arr_neglog<ARITH>(wd), __ldg(ctab + z))));
    out[i] = arr_mul<ARITH>(fix_round(acc), R[i]);
    jout[i] = randint(wd.w2, wd.w3, z, k);
  }
}

// The first-arrival screen alone: Philox and the FP32 test, per element.
__global__ void diag_screen_cost_kernel(const int32_t* __restrict__ ids, const double* __restrict__ v, int64_t n, int k,
                                        uint32_t key0, uint32_t key1, float T, uint8_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Words wd = philox((uint32_t)ids[i], 0u, key0, key1);
    out[i] = screen_out(wd.w1, f32_trunc(v[i]), T, (float)k) ? 1 : 0;
  }
}

static size_t round16(size_t x) { return (x + 15) / 16 * 16; }

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace gm

extern "C" int gm_diag_neglog(const uint64_t* x, int64_t n, int32_t fp64_unit, double* out, void* stream) {
  if (n < 0) return GM_EINVAL;
  if (n == 0) return GM_OK;
  if (!x || !out) return GM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (fp64_unit)
    gm::diag_neglog_kernel<gm::ARITH_FP64><<<gm::grid_for(n), 256, 0, st>>>(x, n, out);
  else
    gm::diag_neglog_kernel<gm::ARITH_INT><<<gm::grid_for(n), 256, 0, st>>>(x, n, out);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_diag_dmul(const double* a, const double* b, int64_t n, int32_t fp64_unit, double* out,
                            void* stream) {
  if (n < 0) return GM_EINVAL;
  if (n == 0) return GM_OK;
  if (!a || !b || !out) return GM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (fp64_unit)
    gm::diag_dmul_kernel<gm::ARITH_FP64><<<gm::grid_for(n), 256, 0, st>>>(a, b, n, out);
  else
    gm::diag_dmul_kernel<gm::ARITH_INT><<<gm::grid_for(n), 256, 0, st>>>(a, b, n, out);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_diag_drcp(const double* v, int64_t n, int32_t fp64_unit, double* out, void* stream) {
  if (n < 0) return GM_EINVAL;
  if (n == 0) return GM_OK;
  if (!v || !out) return GM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (fp64_unit)
    gm::diag_drcp_kernel<gm::ARITH_FP64><<<gm::grid_for(n), 256, 0, st>>>(v, n, out);
  else
    gm::diag_drcp_kernel<gm::ARITH_INT><<<gm::grid_for(n), 256, 0, st>>>(v, n, out);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_diag_arrivals(int32_t id, double v, int32_t k, uint64_t seed, int32_t n_steps, int32_t variant,
                                double* b_out, int32_t* c_out, double* ctab_scratch, void* stream) {
  const bool fp64_unit = (variant & 1) != 0, hashed = (variant & 2) != 0;
  if (k < 1 || k > GM_MAX_K || n_steps < 0 || n_steps > k || id < 0 || !(v > 0.0) || !(v < 1.0 / 0.0))
    return GM_EINVAL;
  if (hashed && n_steps > gm::HASH_MAX_FILL - 32) return GM_EINVAL;
  if (!ctab_scratch || (n_steps > 0 && (!b_out || !c_out))) return GM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  gm::diag_ctab_kernel<<<(k + 255) / 256, 256, 0, st>>>(ctab_scratch, k);
  if (n_steps == 0) return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
  const size_t sm = hashed ? (size_t)gm::HASH_SLOTS * 4 : gm::round16((size_t)k * sizeof(uint16_t));
  if (hashed) {
    if (fp64_unit)
      gm::diag_arrivals_kernel<gm::ARITH_FP64, gm::HashPi><<<1, 32, sm, st>>>(id, v, k, k0, k1, n_steps, ctab_scratch, b_out, c_out);
    else
      gm::diag_arrivals_kernel<gm::ARITH_INT, gm::HashPi><<<1, 32, sm, st>>>(id, v, k, k0, k1, n_steps, ctab_scratch, b_out, c_out);
  } else {
    if (fp64_unit)
      gm::diag_arrivals_kernel<gm::ARITH_FP64, gm::DensePi><<<1, 32, sm, st>>>(id, v, k, k0, k1, n_steps, ctab_scratch, b_out, c_out);
    else
      gm::diag_arrivals_kernel<gm::ARITH_INT, gm::DensePi><<<1, 32, sm, st>>>(id, v, k, k0, k1, n_steps, ctab_scratch, b_out, c_out);
  }
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_diag_first_arrival(const int32_t* ids, const double* v, int64_t n, int32_t k, uint64_t seed,
                                     float T, uint8_t* screened, double* b0, void* stream) {
  if (n < 0 || k < 1) return GM_EINVAL;
  if (n == 0) return GM_OK;
  if (!ids || !v || !screened || !b0) return GM_EINVAL;
  gm::diag_first_kernel<<<gm::grid_for(n), 256, 0, (cudaStream_t)stream>>>(
      ids, v, n, k, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32), T, screened, b0);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_diag_fma(int32_t fp64, int32_t blocks, int32_t iters, void* out, void* stream) {
  if (blocks < 1 || iters < 1 || !out) return GM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (fp64)
    gm::diag_fma_kernel<double><<<blocks, 256, 0, st>>>((double*)out, iters, 0.999, 1e-3);
  else
    gm::diag_fma_kernel<float><<<blocks, 256, 0, st>>>((float*)out, iters, 0.999f, 1e-3f);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}

extern "C" int gm_diag_arrival_cost(const int32_t* ids, const double* R, int64_t n, int32_t k, uint64_t seed,
                                    double* ctab_scratch, double* out, int32_t* jout, uint8_t* screened,
                                    float T, void* stream) {
  if (n < 0 || k < 1 || k > GM_MAX_K) return GM_EINVAL;
  if (n == 0) return GM_OK;
  if (!ids || !R || !ctab_scratch || !out || !jout || !screened) return GM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
  gm::diag_ctab_kernel<<<(k + 255) / 256, 256, 0, st>>>(ctab_scratch, k);
  gm::diag_arrival_cost_kernel<gm::ARITH_MIX><<<gm::grid_for(n), 256, 0, st>>>(ids, R, n, k, k0, k1, ctab_scratch,
                                                                               out, jout);
  gm::diag_arrival_cost_kernel<gm::ARITH_INT><<<gm::grid_for(n), 256, 0, st>>>(ids, R, n, k, k0, k1, ctab_scratch,
                                                                               out, jout);
  gm::diag_screen_cost_kernel<<<gm::grid_for(n), 256, 0, st>>>(ids, R, n, k, k0, k1, T, screened);
  return cudaGetLastError() == cudaSuccess ? GM_OK : GM_ECUDA;
}
