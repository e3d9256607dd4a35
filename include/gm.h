/*
 * gm.h -- C-ABI of libgm, the GB300 (sm_103a) k-register Gumbel-Max sketch.
 *
 * Paper: Y. Zhang, P. Wang, Y. Qi, K. Cheng, J. Zhao, G. Tian, X. Guan,
 * "Fast Gumbel-Max Sketch and its Applications", arXiv 2302.05176.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, unless a
 *     parameter says "host".  The library never frees them and never keeps
 *     them after the call returns.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  The return value only reports
 *     errors found on the host before launch (bad sizes, null pointers, a
 *     workspace that is too small, a failed launch).  Errors found on the
 *     device are recorded in the workspace and read back by gm_status().
 *   - The library allocates no memory.  Scratch space comes from a caller
 *     workspace whose size gm_sketch_workspace_bytes() reports.  Calls that
 *     share a workspace must be ordered (same stream, or synchronised).  A
 *     workspace must start on a 256-byte boundary (as cudaMalloc returns; the
 *     kernels use 16-byte atomics and loads inside it): GM_EINVAL otherwise.
 *   - All functions are thread-safe as long as concurrent calls use distinct
 *     workspaces.
 *
 * The sketch (Sec. 1, Eq. sjv and Eq. yjpi): for a non-negative vector v and
 * k registers, register j holds
 *     y_j = min_{i : v_i > 0} b_{i,j},   s_j = the i attaining it,
 * where b_{i,1..k} are element i's k arrival times, generated in ascending order
 * as exponential order statistics (Sec. 2.2, Eq. biz_dis / biz_biz-1) and
 * spread over the k registers by a Fisher-Yates shuffle (same section).
 * Arrival z (0-based) of element id with weight v, for a given (k, seed):
 *     (w0,w1,w2,w3) = Philox4x32-10(key = (seed_lo, seed_hi), ctr = (id, z, 0, 0))
 *     u   = (2 * ((w1:w0) >> 12) + 1) * 2^-53            exact, in (0, 1)
 *     E   = RN(-ln u)
 *     t_z = RN(E * RN(1 / (k - z)))
 *     S_z = RN(t_0 + ... + t_z)        (the sum formed exactly, rounded once)
 *     b_z = RN(S_z * RN(1 / v))
 *     J   = z + floor((w3:w2) * (k - z) / 2^64);  swap(pi[z], pi[J]);  server = pi[z]
 * Ties in a register go to the smaller id.  An unfilled register reads
 * y = +inf, s = -1.  Zero weights take no part (N^+ of Sec. 1).
 * Results do not depend on the pruning bound, the launch shape or the
 * algorithm variant: gm_sketch (FastGM) and gm_sketch_plain (all k n+
 * arrivals) return the same registers.
 */
#ifndef GM_H
#define GM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GM_OK 0
#define GM_EINVAL 1   /* an argument is out of range (see each function)           */
#define GM_ENOMEM 2   /* the workspace is smaller than gm_*_workspace_bytes() says  */
#define GM_ECUDA 3    /* a CUDA launch or query failed                              */
#define GM_ETIMEOUT 4 /* a bounded device-side retry loop gave up (device status)   */
#define GM_EDATA 5    /* invalid input data found on the device (device status)     */

/* ---- flags for gm_sketch ------------------------------------------------ */
/* Validate the CSR on the device: row_ptr[0] == 0, non-decreasing, row_ptr[n_rows]
 * == nnz, ids >= 0, weights finite and >= 0.  A violation sets GM_EDATA in the
 * device status (gm_status); the registers of an invalid row are unspecified. */
#define GM_FLAG_VALIDATE (1u << 0)
/* Arithmetic of an arrival.  Default: -ln(u) exactly on the integer pipes (a
 * table-driven logarithm in 128-bit fixed point), the two products of each
 * arrival and 1/v on the FP64 unit (IEEE multiply and reciprocal), which is
 * otherwise idle.  GM_FLAG_INT_PRODUCTS computes the products and 1/v on the
 * integer pipes too (the same bits; slower on GB300).  GM_FLAG_FP64_UNIT also
 * takes -ln(u) from the FP64 unit (CUDA's log: within one ulp of the default;
 * much slower on GB300).  All three are kept for comparison and tested. */
#define GM_FLAG_INT_PRODUCTS (1u << 1)
#define GM_FLAG_FP64_UNIT (1u << 2)
/* Testing aid: divide the closed-form bounds of the first pass (and of long-row
 * chunks) by 8, so that most rows find a register unfilled and take the
 * escalation paths.  The registers are the same; only the work grows. */
#define GM_FLAG_TIGHT_BOUND (1u << 3)
/* Initial pruning bound per row (Sec. 2.2 FastSearch / FastPrune).  Any bound
 * gives the same registers; it only changes how many arrivals are generated.
 *   GM_BOUND_CLOSED: the (1 - p) quantile of y* given sum v (the law of y* sum v
 *     is that of the largest of k Exp(1), Sec. 2.3), then wider passes.
 *   GM_BOUND_NONE: FastGM without prior knowledge of y*: FastSearch's release
 *     horizon starts at R = k arrivals per row (T = 1 / sum v) and doubles until
 *     every register is filled (each pass regenerates the arrivals below its T;
 *     register updates are idempotent minima).  A row cut into chunks runs the
 *     same ladder per chunk on the chunk's own registers, and once the row's
 *     merged registers are all filled a chunk stops every stream at their largest
 *     value y* (FastPrune).
 *   GM_BOUND_LEARNED: per-row bound from a trained model (gm_model_*). */
#define GM_BOUND_CLOSED (0u << 4)
#define GM_BOUND_NONE (1u << 4)
#define GM_BOUND_LEARNED (2u << 4)
#define GM_BOUND_MASK (3u << 4)
/* Long rows with a fixed bound (closed form, learned or a caller's) are compacted
 * -- every element's first arrival screened by the whole GPU first, the sketch
 * then formed from the elements left -- when the batch is large and made of long
 * rows (more than 2^23 elements, an average row above 32,768).  This flag
 * compacts them in any batch (not Stream-FastGM chunks, not GM_BOUND_NONE).  The
 * registers are the same either way. */
#define GM_FLAG_COMPACT_LONG (1u << 6)

/* ---- device-side counters, read back by gm_status ------------------------- */
typedef struct gm_stats {
  uint64_t arrivals;        /* arrivals generated (light lanes and warp segments)      */
  uint64_t elements;        /* positive elements visited                               */
  uint64_t screened_out;    /* elements whose first arrival exceeded the row bound      */
  uint64_t heavy_elements;  /* elements streamed by 8- or 32-lane segments             */
  uint64_t rows_escalated;  /* row passes repeated with a larger bound (unfilled rows) */
  uint64_t cas_retries;     /* register compare-and-swap retries                        */
  /* per-warp clock cycles summed over the warps of the sketch kernel: light lanes,
   * 8-lane segments, 32-lane warps, dense permutations, waiting at barriers, row
   * setup (sums, bounds), row finish (filled check, output), total */
  uint64_t cycles_light, cycles_medium, cycles_heavy, cycles_dense, cycles_wait, cycles_setup, cycles_finish,
      cycles_total;
  uint64_t kept;            /* arrivals within the bound (each updates a register)      */
  uint64_t rows_fallback;   /* rows whose first-pass bound was below y* (redone wider)  */
  uint32_t status;          /* GM_OK, GM_EDATA or GM_ETIMEOUT                           */
  uint32_t reserved;
} gm_stats;

/* Bytes of workspace gm_sketch / gm_sketch_plain need for this problem.
 * Returns 0 if the arguments are out of range. */
size_t gm_sketch_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k, uint32_t flags);

/*
 * gm_sketch -- FastGM (Algorithm 1, Sec. 2.2) over a batch of CSR rows.
 *
 *   row_ptr  int64[n_rows + 1]   row r owns elements [row_ptr[r], row_ptr[r+1])
 *   ids      int32[nnz]          element ids (>= 0); ids within a row should be distinct
 *   w        float64[nnz]        weights (finite, >= 0; zero weights are skipped)
 *   n_rows   >= 0
 *   nnz      == row_ptr[n_rows] (row bounds are clamped to [0, nnz] on the device)
 *   k        number of registers, 1 <= k <= GM_MAX_K
 *   seed     64-bit key of the arrival streams (sketches compare only under one seed)
 *   flags    GM_FLAG_* | GM_BOUND_*
 *   s_out    int32[n_rows * k]   row-major: register j of row r at r * k + j
 *   y_out    float64[n_rows * k]
 *   workspace / workspace_bytes  device scratch, >= gm_sketch_workspace_bytes(...)
 *   stream   cudaStream_t
 * Returns GM_OK, GM_EINVAL (bad sizes / null pointers / k out of range),
 * GM_ENOMEM (workspace too small) or GM_ECUDA.
 */
#define GM_MAX_K 4096
int gm_sketch(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
              int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
              size_t workspace_bytes, void* stream);

/*
 * gm_sketch_plain -- the straightforward O(k n+) sketch (Sec. 1, "the
 * straightforward method"): every positive element generates all k arrivals.
 * Same arguments, same output as gm_sketch; it exists as the baseline FastGM
 * is measured against.  `flags` accepts GM_FLAG_VALIDATE and GM_FLAG_FP64_UNIT.
 */
int gm_sketch_plain(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                    int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out,
                    void* workspace, size_t workspace_bytes, void* stream);

/*
 * gm_sketch_noalloc -- gm_sketch without a workspace argument: it allocates
 * nothing and takes no scratch from the caller.  (The paper has no counterpart;
 * this is a library convenience.)
 *
 * For callers that cannot allocate device memory or hand the library a
 * workspace: hosts whose device memory belongs to a framework or plugin
 * allocator that forbids foreign allocations, serving loops that must never
 * stall on cudaMalloc (which can synchronise the device and can fail under
 * memory pressure), and thin foreign-function bindings that can only pass the
 * input and output buffers.
 *
 * The scratch is one fixed device array inside libgm, sized for
 * nnz <= GM_NOALLOC_MAX_NNZ, n_rows <= GM_NOALLOC_MAX_ROWS and k <= GM_MAX_K:
 * 10,788,096 bytes (about 10.8 MB) that every GPU which loads the library holds
 * until the process exits.  Arguments and output are those of gm_sketch (same
 * kernels, same registers), minus the workspace.
 *   - Returns GM_ENOMEM if nnz > GM_NOALLOC_MAX_NNZ or n_rows >
 *     GM_NOALLOC_MAX_ROWS (checked on the host, nothing is launched), GM_EINVAL
 *     for the argument errors of gm_sketch, GM_ECUDA on a CUDA error.
 *   - Errors found on the device (GM_FLAG_VALIDATE's GM_EDATA, GM_ETIMEOUT) are
 *     recorded in the array's header: read them with gm_sketch_noalloc_status
 *     after the call, before the next call on that device overwrites them.
 *   - Each call made outside stream capture looks up the array's device address
 *     (cudaGetSymbolAddress, with the calling device current) and caches it per
 *     device; a call made during capture uses that cache, so make one call on the
 *     device before capturing one.
 *   - All calls share the one array, which keeps the last call's contents (each
 *     call first resets what must start at zero).  Calls whose work overlaps on
 *     the GPU -- on different streams, or from different host threads without
 *     ordering -- race on it and give undefined registers: order them.
 */
#define GM_NOALLOC_MAX_NNZ (1 << 20)
#define GM_NOALLOC_MAX_ROWS (1 << 16)
int gm_sketch_noalloc(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                      int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* stream);

/* gm_sketch_noalloc_status -- gm_status for the fixed array of gm_sketch_noalloc:
 * waits for the work queued on `stream`, copies the device status and counters
 * of the last gm_sketch_noalloc call on the current device into *stats (host,
 * may be NULL) and returns GM_OK, GM_EDATA, GM_ETIMEOUT or GM_ECUDA.  Allocates
 * nothing.  (No counterpart in the paper.) */
int gm_sketch_noalloc_status(gm_stats* stats, void* stream);

/*
 * gm_status -- wait for the work queued on `stream`, then copy the device
 * status and counters of the last call that used `workspace` into *stats
 * (host pointer, may be NULL) and return the device status (GM_OK, GM_EDATA
 * or GM_ETIMEOUT), or GM_ECUDA if the copy fails.  Blocks the calling thread.
 */
int gm_status(const void* workspace, gm_stats* stats, void* stream);

/*
 * gm_jaccard -- probability-Jaccard estimates (Sec. 1; unbiased, variance
 * J(1-J)/k, Sec. 2.4):  out[p] = (1/k) * #{ j : s_a[p k + j] == s_b[p k + j] >= 0 }.
 *   s_a, s_b int32[n_pairs * k]  (the caller gathers the two sketches of each pair
 *                                 into row p of s_a and s_b; both under one (k, seed))
 *   out      float64[n_pairs]
 * Unfilled registers (s = -1) never match.  Returns GM_EINVAL if k < 1 or
 * n_pairs < 0.
 */
int gm_jaccard(const int32_t* s_a, const int32_t* s_b, int64_t n_pairs, int32_t k, double* out, void* stream);

/*
 * gm_cardinality -- weighted-cardinality estimates (Lemiesz's estimator,
 * Sec. 1 and the Sec. 2.4 theorem):  out[r] = (k - 1) / sum_j y[r k + j].
 *   y   float64[n_rows * k],  out float64[n_rows]
 * A row with an unfilled register (y = +inf) estimates 0.  The sum is formed in
 * FP64 in an order of the library's choosing (relative difference to any other
 * order <= k * 2^-53).  Returns GM_EINVAL if k < 2 or n_rows < 0.
 */
int gm_cardinality(const double* y, int32_t n_rows, int32_t k, double* out, void* stream);

/*
 * gm_merge -- union of sketches (Sec. 2.3 Mergeability): register-wise minimum
 * of (y, s), ties to the smaller id, unfilled (+inf, -1) losing to anything.
 *   s_a, y_a, s_b, y_b  [n_regs] inputs;  s_out, y_out [n_regs] outputs (may alias
 *   either input).  Returns GM_EINVAL if n_regs < 0.
 */
int gm_merge(const int32_t* s_a, const double* y_a, const int32_t* s_b, const double* y_b, int64_t n_regs,
             int32_t* s_out, double* y_out, void* stream);

/* ---- learned pruning bound ---------------------------------------------------
 * Not in the paper: a small MLP predicts, per row, the bound below which FastGM
 * generates arrivals (the role of FastSearch's release horizon, Sec. 2.2).  Any
 * bound gives the same registers; an unfilled row is redone with the closed-form
 * bound and then wider ones, so the result stays exact.
 *
 * Model: 8 -> 64 -> 64 -> 1, GELU (erf form), FP32.  Parameters, one contiguous
 * device float array of GM_MODEL_PARAMS: W1[64][8], b1[64], W2[64][64], b2[64],
 * w3[64], b3.  The output is ln(bound) = net(x) - x[1]: the network sees the
 * scale-free quantity ln(y* sum v) (scaling v by c scales y* by 1/c exactly).
 * Features per row (float[8]): ln n+, ln sum v, ln max v, ln of the weights'
 * 10/50/90/99 % quantiles (from a log2 histogram, 1/4-octave bins), ln k.
 */
#define GM_MODEL_FEATURES 8
#define GM_MODEL_HIDDEN 64
#define GM_MODEL_PARAMS (GM_MODEL_HIDDEN * GM_MODEL_FEATURES + GM_MODEL_HIDDEN + \
                         GM_MODEL_HIDDEN * GM_MODEL_HIDDEN + GM_MODEL_HIDDEN + GM_MODEL_HIDDEN + 1)

/* Features of every row into feats[n_rows * 8] (device).  Rows without positive
 * weights get ln n+ = ln sum v = ... = -inf replaced by 0.  GM_EINVAL on bad sizes. */
int gm_features(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz, int32_t k,
                float* feats, void* stream);

/* Per row, ln max_j y_j of a finished sketch (the training target), into
 * ln_ystar[n_rows]; +inf when a register is unfilled.  k >= 1. */
int gm_row_ln_ystar(const double* y, int32_t n_rows, int32_t k, float* ln_ystar, void* stream);

/* Initialise params (device, GM_MODEL_PARAMS floats): uniform(-1/sqrt(fan_in),
 * 1/sqrt(fan_in)) from a Philox stream keyed by `seed`, biases 0. */
int gm_model_init(float* params, uint64_t seed, void* stream);

/* out[i] = predicted ln bound of sample i (feats: float[n * 8]). */
int gm_model_forward(const float* params, const float* feats, int32_t n, float* out, void* stream);

/* Mean pinball loss at level tau (0 < tau < 1), L = mean_i rho_tau(t_i - pred_i)
 * with rho_tau(r) = tau r for r > 0 and (tau - 1) r otherwise, of the prediction
 * against target[n] (ln y*); its gradient into grad[GM_MODEL_PARAMS] (overwritten)
 * and L into loss[1] (device).  At r = 0 the subgradient of the r <= 0 branch is
 * taken.  The loss is minimised by the tau-quantile of ln y* given the features,
 * so the bound exceeds y* in a fraction tau of rows.  n >= 1.  The result is the
 * same bits on every run (fixed partition, fixed summation order).  Workspace:
 * gm_model_grad_workspace_bytes() bytes of device scratch. */
size_t gm_model_grad_workspace_bytes(void);
int gm_model_grad(const float* params, const float* feats, const float* target, int32_t n, float tau, float* grad,
                  float* loss, void* workspace, size_t workspace_bytes, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) of params with grad; adam holds
 * 2 * GM_MODEL_PARAMS floats of moments (zero them before step 1); step >= 1. */
int gm_model_adam(float* params, float* adam, const float* grad, float lr, int32_t step, void* stream);

/* Save / load params to / from a file (host path; blocks on `stream`).  The file
 * holds a 16-byte header ("GMMLP001", feature and hidden sizes) and the floats. */
int gm_model_save(const float* params, const char* path, void* stream);
int gm_model_load(float* params, const char* path, void* stream);

/* The learned first-pass bound of every row of a CSR batch (device arrays):
 * t_out[r] = exp(prediction_r + margin) as a positive FP32 value (clamped to
 * [1e-37, +inf]), prediction_r = gm_model_forward of the row's gm_features.
 * Rows of up to 2,048 elements take one warp each; longer rows are cut into
 * 2,048-element pieces, one warp each over the whole grid, combined in a fixed
 * order, so t_out is the same bits on every call (the sum of a long row may differ
 * from gm_features' in the last FP32 place).  A row with no positive weight
 * gets the features of gm_features (zeros).  params: GM_MODEL_PARAMS floats;
 * margin finite.  Workspace: gm_learned_bound_workspace_bytes(n_rows, nnz) bytes
 * of device memory.  Rows that overlap (row_ptr not ascending) may get t_out = -1
 * (no learned bound) instead. */
size_t gm_learned_bound_workspace_bytes(int32_t n_rows, int64_t nnz);
int gm_learned_bound(const int64_t* row_ptr, const double* w, int32_t n_rows, int64_t nnz, int32_t k,
                     const float* params, float margin, float* t_out, void* workspace, size_t workspace_bytes,
                     void* stream);

/* gm_sketch with the first-pass bound of each row predicted by the model
 * (gm_learned_bound, run on `stream` ahead of the sketch kernels):
 * T_r = exp(prediction_r + margin).  Same registers as gm_sketch.  Workspace:
 * gm_sketch_learned_workspace_bytes(). */
size_t gm_sketch_learned_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k);
int gm_sketch_learned(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                      int32_t k, uint64_t seed, uint32_t flags, const float* params, float margin, int32_t* s_out,
                      double* y_out, void* workspace, size_t workspace_bytes, void* stream);

/* ---- autotuning ---------------------------------------------------------------
 * Not in the paper.  Four runtime parameters shape gm_sketch's work without
 * changing its output: the quantile of the first-pass bound (p_first: the bound
 * is the (1 - p_first) quantile of y* given sum v) and the routing of elements by
 * their expected number of arrivals below the bound -- one lane each up to
 * light_max, 8-lane segments up to medium_max, 32-lane warps up to heavy_max,
 * a dense permutation beyond.  gm_sketch takes them from a process-wide table
 * keyed by (k, floor(log2(mean row length))), else the defaults (0.05, 4, 64,
 * 256).  gm_tune times candidate values on the caller's batch (coordinate
 * descent, up to two sweeps, each candidate the fastest of three timed calls
 * after one warm-up and adopted when 1 % faster; it synchronises `stream`),
 * installs the fastest for that key and returns it.
 * Requires 0 < p_first < 1 and 0 < light_max <= medium_max <= heavy_max. */
typedef struct gm_tuning {
  float p_first;
  float light_max;
  float medium_max;
  float heavy_max;
} gm_tuning;
void gm_tuning_default(gm_tuning* t);
int gm_tune(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz, int32_t k,
            uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace, size_t workspace_bytes,
            gm_tuning* best, double* best_ms, void* stream);
/* Install / read / forget table entries (mean_row_len = nnz / n_rows of the
 * batches the entry serves); save and load the table as text. */
int gm_tuning_set(int32_t k, int64_t mean_row_len, const gm_tuning* t);
int gm_tuning_get(int32_t k, int64_t mean_row_len, gm_tuning* out);
int gm_tuning_clear(void);
int gm_tuning_save(const char* path);
int gm_tuning_load(const char* path);

/* ---- FastSearch's schedule and caller-given bounds --------------------------------
 * gm_sketch_budget: the release step of FastSearch (Algorithm 1, Sec. 2.2): in
 * row r, element i releases the first min(k, ceil(R_row[r] * (v_i / sum v)))
 * arrivals of its stream (sum over the row's positive weights; the ratio and the
 * product in FP64, round to nearest, then the ceiling), and the registers keep the
 * minima of those arrivals.  R_row: device doubles [n_rows].  Registers that no
 * released arrival reached read (+inf, -1).  Same workspace as gm_sketch.
 *
 * gm_sketch_bounded: FastGM with the first-pass bound of each row given by the
 * caller, bound_row[r] (device doubles): > 0 and finite -- that bound (rounded
 * up to FP32); +inf -- no bound; <= 0 or NaN -- the closed form.  Any bound gives
 * gm_sketch's registers.  With bound_row = y* of the FastSearch registers this is
 * FastPrune.  Workspace: gm_sketch_bounded_workspace_bytes().
 *
 * gm_row_ystar: out[r] = max_j y[r, j] (+inf when a register is unfilled). */
int gm_sketch_budget(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                     int32_t k, uint64_t seed, uint32_t flags, const double* R_row, int32_t* s_out, double* y_out,
                     void* workspace, size_t workspace_bytes, void* stream);
size_t gm_sketch_bounded_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k);
int gm_sketch_bounded(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                      int32_t k, uint64_t seed, uint32_t flags, const double* bound_row, int32_t* s_out,
                      double* y_out, void* workspace, size_t workspace_bytes, void* stream);
int gm_row_ystar(const double* y, int32_t n_rows, int32_t k, double* out, void* stream);

/*
 * gm_sketch_fastsearch -- FastGM under the paper's own FastSearch schedule
 * (Algorithm 1, Sec. 2.2), all on the device: each row is taken by one CTA,
 * which runs the rounds R = delta, 2 delta, ... -- element i releases the first
 * min(k, ceil(R (v_i / sum v))) arrivals of its stream (sum v in FP64 in a fixed
 * order; the ratio and the product in FP64, then the ceiling) -- until every
 * register holds an arrival, then FastPrune: every element streams until its
 * arrival exceeds the row's y* = max_j y_j.  An element whose budget did not grow
 * in a round releases nothing in it; one whose budget grew releases its stream
 * again from the first arrival (register updates are idempotent).  After 4,096
 * rounds a last round releases every arrival.  Same registers as gm_sketch.
 *   delta       >= 1 (Algorithm 1 takes delta = k)
 *   rounds_out  device int32[n_rows] (nullable): the rounds each row took, so the
 *               budget at which FastSearch found every register filled is
 *               rounds_out[r] * delta (0 for a row without positive weights)
 * flags: GM_FLAG_VALIDATE and the arithmetic flags.  Workspace: as gm_sketch.
 * gm_status's rows_escalated counts the rounds beyond the first, summed over rows.
 */
int gm_sketch_fastsearch(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                         int32_t k, uint64_t seed, uint32_t flags, int32_t delta, int32_t* rounds_out,
                         int32_t* s_out, double* y_out, void* workspace, size_t workspace_bytes, void* stream);

/* ---- Stream-FastGM (Algorithm 2, Sec. 3 of the paper: the extension to streams) --
 * A stream of elements, each occurring any number of times with a fixed weight,
 * folded chunk by chunk into one running sketch (s int32[k], y double[k] on the
 * device, owned by the caller).  The result after any sequence of chunks is the
 * sketch of the set of distinct elements seen: an element's arrivals depend only
 * on (seed, id, v), so a repeated occurrence changes nothing.  Each chunk is
 * sketched as one row whose registers start from the running sketch; once every
 * register is filled, the chunk's bound is the running y* (FastPrune), so most
 * elements of a long stream fail the first-arrival screen.  Duplicates inside a
 * chunk are allowed; an id must always come with the same weight.
 *
 * gm_stream_reset: s = -1, y = +inf (an empty sketch).  gm_stream_ingest: fold
 * ids/w[0..n) into (s, y); workspace of gm_stream_workspace_bytes(n, k) bytes;
 * flags as gm_sketch except GM_BOUND_LEARNED (GM_EINVAL).  Asynchronous. */
size_t gm_stream_workspace_bytes(int64_t n, int32_t k);
int gm_stream_reset(int32_t* s, double* y, int32_t k, void* stream);
int gm_stream_ingest(int32_t* s, double* y, int32_t k, const int32_t* ids, const double* w, int64_t n, uint64_t seed,
                     uint32_t flags, void* workspace, size_t workspace_bytes, void* stream);

/* ---- host-memory batches ---------------------------------------------------------
 * gm_sketch over a CSR batch in HOST memory (row_ptr, ids, w, s_out, y_out all
 * host arrays; page-locked ones are copied asynchronously, pageable ones through
 * the CUDA runtime's staging buffers).  The batch is cut into chunks of rows (at
 * least 128 rows, about a sixteenth of the batch) that are copied to the device,
 * sketched and copied back on eight streams, so the copies of some chunks overlap
 * the sketches of others.  Blocks until every register is in s_out / y_out.  The
 * same registers as gm_sketch on the whole batch.  row_ptr is checked on the host
 * (GM_EINVAL: row_ptr[0] != 0, decreasing, row_ptr[n_rows] != nnz).  workspace:
 * device memory of gm_sketch_host_workspace_bytes_csr(row_ptr, n_rows, k) bytes
 * (sized by the largest chunk; 0 for invalid row offsets), at most
 * gm_sketch_host_workspace_bytes(n_rows, nnz, k) (any row offsets); GM_ENOMEM when
 * smaller.  Concurrent calls in one process are serialised. */
size_t gm_sketch_host_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k);
size_t gm_sketch_host_workspace_bytes_csr(const int64_t* row_ptr, int32_t n_rows, int32_t k);
int gm_sketch_host(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                   int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
                   size_t workspace_bytes);

/* ---- CUDA graphs --------------------------------------------------------------
 * Not in the paper.  A gm_sketch call is five kernel launches plus host-side
 * setup; for a workload repeated over the same buffers (a fixed-shape batch
 * refilled in place, a benchmark loop) the whole call can be captured once into
 * a CUDA graph and replayed with one launch.  gm_graph_create captures
 * gm_sketch(row_ptr, ..., workspace_bytes) on a private stream (nothing runs);
 * gm_graph_launch replays it on `stream`, reading whatever the buffers hold at
 * that time (the sizes, k, seed and flags are fixed; row_ptr's values may change
 * as long as they stay a valid CSR of nnz elements).  Errors as gm_sketch;
 * GM_ECUDA if capture or instantiation fails. */
typedef struct gm_graph gm_graph;
int gm_graph_create(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                    int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
                    size_t workspace_bytes, gm_graph** out);
int gm_graph_launch(gm_graph* graph, void* stream);
int gm_graph_destroy(gm_graph* graph);

/* Human-readable text of a status code (static storage, never NULL). */
const char* gm_strerror(int code);

/* Library version string, e.g. "libgm 0.1 sm_103a" (static storage). */
const char* gm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GM_H */
