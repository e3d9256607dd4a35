/*
 * gm_diag.h -- diagnostic entry points of libgm.
 *
 * They expose, one value at a time, the device arithmetic that every arrival of
 * the sketch goes through (Sec. 2.2, Eq. biz_dis / Eq. biz_biz-1, with the
 * rounding reading stated in gm.h), so that tests can compare it with independent
 * references: high-precision logarithms, IEEE products and reciprocals, and the
 * CPU oracle's arrival streams.  All arrays are device pointers owned by the
 * caller; calls are asynchronous on `stream` and return GM_OK, GM_EINVAL or
 * GM_ECUDA (codes of gm.h).  `fp64_unit` = 0 selects the default integer-pipe
 * arithmetic, 1 the FP64-unit arithmetic (GM_FLAG_FP64_UNIT).
 */
#ifndef GM_DIAG_H
#define GM_DIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* out[i] = RN(-ln u_i), u_i = (2 (x[i] >> 12) + 1) 2^-53: the E of an arrival whose
 * Philox words 0,1 form x[i] = (w1:w0).  n >= 0. */
int gm_diag_neglog(const uint64_t* x, int64_t n, int32_t fp64_unit, double* out, void* stream);

/* out[i] = RN(a[i] * b[i]) for positive finite a[i], b[i].  n >= 0. */
int gm_diag_dmul(const double* a, const double* b, int64_t n, int32_t fp64_unit, double* out, void* stream);

/* out[i] = RN(1 / v[i]) for positive finite v[i].  n >= 0. */
int gm_diag_drcp(const double* v, int64_t n, int32_t fp64_unit, double* out, void* stream);

/* The first n_steps arrivals (time b_out[z], server c_out[z]) of element (id, v)
 * for k registers and `seed`, produced by the warp path of the sketch kernels
 * (32 arrivals per step, exact shuffle scan, parallel Fisher-Yates).
 * variant: bit 0 = FP64-unit arithmetic, bit 1 = the hashed permutation of the
 * FastGM warp path (then n_steps <= 352) instead of the dense one.
 * 0 <= n_steps <= k <= GM_MAX_K (gm.h), v positive finite, id >= 0.
 * ctab_scratch: device scratch of at least k doubles (overwritten). */
int gm_diag_arrivals(int32_t id, double v, int32_t k, uint64_t seed, int32_t n_steps, int32_t variant,
                     double* b_out, int32_t* c_out, double* ctab_scratch, void* stream);

/* The FastGM first-arrival screen and the exact first arrival, per element:
 * screened[i] = 1 when the conservative FP32 screen skips element (ids[i], v[i])
 * for bound T (it must then hold b0[i] > T), b0[i] = its exact first arrival
 * time for k registers and `seed` (integer-pipe arithmetic).  k >= 1, n >= 0. */
int gm_diag_first_arrival(const int32_t* ids, const double* v, int64_t n, int32_t k, uint64_t seed, float T,
                          uint8_t* screened, double* b0, void* stream);

/* The algorithmic work of one arrival and of one first-arrival screen, each
 * computed independently per element (for instruction counting): out[i] = the
 * arrival time of step z = i mod k of element ids[i] with R = R[i] (a
 * single-term sum), jout[i] its RandInt target, screened[i] the screen decision
 * for weight R[i] and bound T.  Three kernels: the arrival in the default
 * arithmetic, the arrival with GM_FLAG_INT_PRODUCTS' arithmetic (same outputs,
 * written last), the screen.  ctab_scratch: >= k doubles.  1 <= k <= GM_MAX_K. */
int gm_diag_arrival_cost(const int32_t* ids, const double* R, int64_t n, int32_t k, uint64_t seed,
                         double* ctab_scratch, double* out, int32_t* jout, uint8_t* screened, float T,
                         void* stream);

/* blocks x 256 threads, each running 8 independent FMA chains of `iters` steps
 * in FP64 (fp64 = 1) or FP32 (fp64 = 0); out: device array of blocks*256
 * doubles (or floats).  Timed by the caller, it gives the device's FMA rate:
 * 8 * iters * blocks * 256 FMAs per launch. */
int gm_diag_fma(int32_t fp64, int32_t blocks, int32_t iters, void* out, void* stream);

/* Register two CUDA events (cudaEvent_t, created by the caller) that every later
 * gm_sketch / gm_sketch_plain / gm_sketch_learned call records on its stream
 * immediately before and after its main sketch kernel, so that kernel can be
 * timed alone; (NULL, NULL) stops it.  Process-wide setting, not thread-safe:
 * for timing only.  GM_EINVAL if exactly one of the two is NULL. */
int gm_diag_time_main_kernel(void* before, void* after);

/* The same for the kernels of gm_jaccard, gm_cardinality, gm_merge and
 * gm_learned_bound: every later call of one of them records `before` on its
 * stream immediately before its first kernel and `after` immediately after its
 * last, so that its device time excludes the host's launch overhead.
 * Process-wide, not thread-safe: for timing only. */
int gm_diag_time_aux_kernels(void* before, void* after);

#ifdef __cplusplus
}
#endif

#endif /* GM_DIAG_H */
