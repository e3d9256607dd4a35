/*
 * gm_server.h -- a continuous-batching serving engine for Gumbel-Max sketches.
 *
 * Not in the paper (Zhang et al., arXiv 2302.05176, has no serving system): the
 * engine turns the batch entry point gm_sketch (FastGM, Algorithm 1, Sec. 2.2)
 * into a request loop.  Clients submit single-vector sketch requests and
 * weighted-Jaccard / cardinality queries (Sec. 1, Sec. 2.4) over sketches the
 * engine keeps resident in device memory.  A scheduler thread owned by the
 * engine
 *   - groups queued sketch requests of equal k, in arrival order, into one CSR
 *     batch per launch (continuous batching: a batch is formed whenever a
 *     stream slot is free, from whatever has arrived by then);
 *   - admits a request only when its inputs, its share of the batch workspace
 *     and its resident output fit in the engine's device arena (memory-based
 *     admission); requests larger than the whole arena are refused at submit;
 *   - runs up to n_streams batches at once on separate CUDA streams, so
 *     later batches overlap with earlier ones and with host-side packing;
 *   - runs every query whose sketches are finished in one batched launch.
 * A sketch in a batch gets exactly the registers gm_sketch gives for that vector
 * alone (rows are independent and every arrival is a function of (seed, id)),
 * and a query the value gm_jaccard / gm_cardinality give for those sketches.
 *
 * Ownership: the caller's input arrays (ids, w) must stay valid and unchanged
 * until the request is finished (poll / wait report a final status).  Pinned
 * (page-locked) inputs are copied to the device asynchronously; pageable ones
 * are copied through a pinned staging area when small, else synchronously by
 * the CUDA driver.  All calls are thread-safe.  Tickets are never reused.
 *
 * Errors: GM_EINVAL (bad argument or unknown ticket), GM_ENOMEM (a request that
 * can never fit in the arena, or the arena could not be allocated), GM_ECUDA,
 * GM_EAGAIN (not finished yet), GM_ECANCELED (the request was cancelled).
 */
#ifndef GM_SERVER_H
#define GM_SERVER_H

#include <stddef.h>
#include <stdint.h>

#include "gm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GM_EAGAIN 6
#define GM_ECANCELED 7

#define GM_REQ_SKETCH 0
#define GM_REQ_JACCARD 1
#define GM_REQ_CARDINALITY 2

typedef struct gm_server gm_server;

typedef struct gm_server_config {
  size_t device_bytes;    /* device arena: batch inputs, workspaces and resident sketches */
  size_t staging_bytes;   /* pinned host staging per stream slot, for pageable inputs     */
  int64_t max_batch_nnz;  /* elements per sketch launch (a larger request runs alone)    */
  int32_t max_batch_rows; /* vectors per sketch launch                                   */
  int32_t n_streams;      /* batches in flight at once (1 .. 8)                          */
  uint64_t seed;          /* the sketch seed of every request (queries need a common seed) */
  uint32_t flags;         /* gm_sketch flags (bound mode, arithmetic)                     */
  const float* params;    /* optional: bound network (device, GM_MODEL_PARAMS floats);
                             when set, sketches run gm_sketch_learned with margin below  */
  float margin;
  int32_t stage_pinned;   /* 1: copy page-locked inputs through the staging area too
                             (one DMA per batch instead of two per request)             */
  int32_t fake_device;    /* 1: no CUDA call at all; launches finish at once, sketches
                             read back empty (-1, +inf) and queries give NaN.  Tests the
                             host logic (admission, batching, cancellation) on machines
                             without a GPU.                                            */
} gm_server_config;

typedef struct gm_server_result {
  int32_t status;       /* GM_OK, GM_EAGAIN (pending), GM_ECANCELED or a failure code     */
  int32_t kind;         /* GM_REQ_*                                                       */
  int32_t k;
  int32_t batch_size;   /* vectors (or queries) in the launch that served the request    */
  double value;         /* query result; NaN for a sketch                                */
  int64_t t_submit_ns;  /* gm_server_now_ns() at submit, launch and completion           */
  int64_t t_launch_ns;
  int64_t t_done_ns;
} gm_server_result;

typedef struct gm_server_stats {
  uint64_t submitted, finished, cancelled, refused, failed;
  uint64_t sketch_batches, query_batches, sketch_rows, sketch_elements, queries;
  uint64_t arena_bytes, arena_peak_bytes, arena_resident_bytes;
  uint64_t queued, in_flight_batches;
  uint64_t staged_requests, direct_requests;  /* inputs copied via staging / by their own DMA */
  uint64_t pack_ns;     /* scheduler time spent packing and launching sketch batches        */
  uint64_t launch_ns;   /* of which inside gm_sketch / gm_sketch_learned                    */
} gm_server_stats;

/* Defaults: 8 GB arena, 64 MB staging, 2^23 elements and 4096 vectors per launch,
 * 4 streams, seed 1, closed-form bound, no model.  Batches of about 100 MB of
 * input keep host-to-device copies and kernels of successive batches
 * overlapping; much larger ones make later requests wait behind one long copy. */
void gm_server_config_default(gm_server_config* cfg);

/* Create an engine on the current CUDA device and start its scheduler thread. */
int gm_server_create(const gm_server_config* cfg, gm_server** out);

/* Cancel queued requests, wait for launches in flight, free everything. */
int gm_server_destroy(gm_server* srv);

/* The engine's clock (steady, nanoseconds). */
int64_t gm_server_now_ns(void);

/* Queue a sketch of one vector: ids int32[nnz] (distinct), w double[nnz] (host
 * memory), 1 <= k <= GM_MAX_K.  nnz >= 0.  On success *ticket names it. */
int gm_server_submit_sketch(gm_server* srv, const int32_t* ids, const double* w, int64_t nnz, int32_t k,
                            uint64_t* ticket);

/* Queue queries over earlier sketch tickets (finished or not): the Jaccard
 * estimate of two sketches of equal k, or the cardinality estimate (k >= 2). */
int gm_server_submit_jaccard(gm_server* srv, uint64_t sketch_a, uint64_t sketch_b, uint64_t* ticket);
int gm_server_submit_cardinality(gm_server* srv, uint64_t sketch, uint64_t* ticket);

/* Status of a ticket without blocking (GM_EAGAIN while pending), or after
 * waiting up to timeout_s seconds.  out may be NULL. */
int gm_server_poll(gm_server* srv, uint64_t ticket, gm_server_result* out);
int gm_server_wait(gm_server* srv, uint64_t ticket, double timeout_s, gm_server_result* out);

/* Copy a finished, resident sketch to host arrays s int32[k], y double[k]. */
int gm_server_read_sketch(gm_server* srv, uint64_t ticket, int32_t* s, double* y);

/* Drop a resident sketch (its device memory is reused once no query needs it). */
int gm_server_release(gm_server* srv, uint64_t ticket);

/* Cancel a request that has not been launched; a launched one finishes on the
 * device but reports GM_ECANCELED and keeps nothing resident. */
int gm_server_cancel(gm_server* srv, uint64_t ticket);

int gm_server_stats_get(gm_server* srv, gm_server_stats* out);

/* Hold (paused = 1) or resume (0) the launch of new batches.  Launches in flight
 * finish; submissions are still accepted and queue up.  For maintenance drains
 * and for tests that need requests to stay queued. */
int gm_server_pause(gm_server* srv, int32_t paused);

#ifdef __cplusplus
}
#endif

#endif /* GM_SERVER_H */
