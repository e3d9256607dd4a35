// gm_server.cu -- continuous-batching serving engine (include/gm_server.h).
//
// One scheduler thread per engine.  Under the engine mutex it (1) retires
// launches whose completion event has fired, (2) forms a sketch batch from the
// queue when a stream slot is free and the device arena admits it, and (3)
// forms a query batch from the queries whose sketches are finished.  Packing
// the batch (host copies, H2D copies, the launch) happens outside the mutex,
// so clients can keep submitting meanwhile.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gm.h"
#include "gm_estim.cuh"
#include "gm_internal.h"
#include "gm_server.h"
#include "gm_trace.h"

namespace gm {
namespace srv {

struct QDesc {
  const int32_t* sa;
  const int32_t* sb;
  const double* y;
  int32_t k;
  int32_t kind;
};

// One warp per query (the same reductions as gm_jaccard / gm_cardinality).
__global__ void __launch_bounds__(EST_BLOCK) query_kernel(const QDesc* __restrict__ q, int n, double* out) {
  const int warps = gridDim.x * (EST_BLOCK / 32);
  for (int i = blockIdx.x * (EST_BLOCK / 32) + (threadIdx.x >> 5); i < n; i += warps) {
    const QDesc d = q[i];
    const double v = d.kind == GM_REQ_JACCARD ? warp_jaccard(d.sa, d.sb, d.k) : warp_cardinality(d.y, d.k);
    if ((threadIdx.x & 31) == 0) out[i] = v;
  }
}

constexpr size_t ALIGN = 256;
constexpr int MAX_QUERIES = 65536;  // per query launch
constexpr size_t SCAN_CAP = 1 << 16;

static int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over [0, cap): offsets into one device allocation.
class Arena {
 public:
  void init(size_t cap) {
    cap_ = cap / ALIGN * ALIGN;
    free_.clear();
    if (cap_) free_[0] = cap_;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(bytes ? bytes : 1, ALIGN);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(bytes ? bytes : 1, ALIGN);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t cap() const { return cap_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

enum State { QUEUED, RUNNING, DONE, CANCELLED, FAILED };

struct Req {
  int kind = GM_REQ_SKETCH;
  int k = 0;
  int64_t nnz = 0;
  const int32_t* ids = nullptr;
  const double* w = nullptr;
  bool pinned = false;    // ids and w are page-locked: copied by DMA, never staged
  uint64_t a = 0, b = 0;  // query operands
  State state = QUEUED;
  int status = GM_EAGAIN;
  double value = NAN;
  int64_t t_submit = 0, t_launch = 0, t_done = 0;
  int batch_size = 0;
  bool cancel_requested = false;
  bool released = false;
  // a finished sketch: its registers are row `row` of output block `block`
  int block = -1;
  int row = 0;
  int refs = 0;  // sketches: 1 until released (or failed / cancelled) + queries that need it
};

struct OutBlock {
  size_t off = 0, bytes = 0;
  int rows = 0, k = 0;
  int live = 0;  // sketches of the block still referenced
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  unsigned char* staging = nullptr;  // pinned: ids region, then w region
  int64_t staging_elems = 0;
  int64_t* h_rowptr = nullptr;       // pinned
  uint32_t* h_status = nullptr;      // pinned: the batch workspace's status word
  QDesc* h_q = nullptr;              // pinned
  double* h_qout = nullptr;          // pinned
  bool busy = false;
  // the batch in flight
  bool is_query = false;
  std::vector<uint64_t> tickets;
  size_t in_off = 0, in_bytes = 0, ws_off = 0, ws_bytes = 0;
  int block = -1;
  int launch_rc = GM_OK;
};

struct Server {
  gm_server_config cfg{};
  int device = 0;
  bool fake = false;
  unsigned char* dev_base = nullptr;
  Arena arena;
  std::vector<Slot> slots;
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> sketch_q;
  std::vector<uint64_t> query_q;
  std::map<int, OutBlock> blocks;
  int next_block = 0;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread thread;
  bool stop = false;
  bool paused = false;
  int in_flight = 0;
  std::atomic<uint64_t> launch_ns_acc{0};  // written by the scheduler outside the mutex
  std::atomic<uint64_t> pack_ns_acc{0};
  gm_server_stats st{};

  size_t resident_bytes() const {
    size_t s = 0;
    for (const auto& kv : blocks) s += round_up(kv.second.bytes, ALIGN);
    return s;
  }
};

static size_t ws_need(const Server& S, int64_t rows, int64_t nnz, int k) {
  return S.cfg.params ? gm_sketch_learned_workspace_bytes((int32_t)rows, nnz, k)
                      : gm_sketch_workspace_bytes((int32_t)rows, nnz, k, S.cfg.flags);
}
static size_t in_need(int64_t rows, int64_t nnz) {
  return round_up((size_t)(rows + 1) * 8, ALIGN) + round_up((size_t)nnz * 4, ALIGN) + round_up((size_t)nnz * 8, ALIGN);
}
static size_t out_need(int64_t rows, int k) {
  return round_up((size_t)rows * k * 4, ALIGN) + round_up((size_t)rows * k * 8, ALIGN);
}

static void finish_req(Server& S, Req& r, State s, int status) {
  r.state = s;
  r.status = status;
  r.t_done = now_ns();
  ++S.st.finished;
  if (s == CANCELLED) ++S.st.cancelled;
  if (s == FAILED) ++S.st.failed;
}

// Drop one reference of a resident sketch; free its block when nothing needs it.
static void unref_sketch(Server& S, Req& r) {
  if (r.refs <= 0) return;
  if (--r.refs > 0 || r.block < 0) return;
  auto it = S.blocks.find(r.block);
  r.block = -1;
  if (it == S.blocks.end()) return;
  if (--it->second.live == 0) {
    S.arena.release(it->second.off, it->second.bytes);
    S.blocks.erase(it);
  }
}

// ---------------------------------------------------------------------------
// Retire finished launches (mutex held).
// ---------------------------------------------------------------------------
static bool retire(Server& S) {
  bool any = false;
  for (auto& sl : S.slots) {
    if (!sl.busy) continue;
    int rc = sl.launch_rc;
    if (rc == GM_OK && !S.fake) {
      const cudaError_t e = cudaEventQuery(sl.ev);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) rc = GM_ECUDA;
    }
    any = true;
    if (!sl.is_query) {
      if (rc == GM_OK && !S.fake && *sl.h_status != 0u)
        rc = (*sl.h_status & WS_EDATA) ? GM_EDATA : GM_ETIMEOUT;
      for (size_t i = 0; i < sl.tickets.size(); ++i) {
        Req& r = S.reqs[sl.tickets[i]];
        if (rc != GM_OK || r.cancel_requested) {
          finish_req(S, r, rc != GM_OK ? FAILED : CANCELLED, rc != GM_OK ? rc : GM_ECANCELED);
          r.released = true;  // nothing stays resident
          unref_sketch(S, r);
        } else {
          finish_req(S, r, DONE, GM_OK);
        }
      }
      S.arena.release(sl.in_off, sl.in_bytes);
      S.arena.release(sl.ws_off, sl.ws_bytes);
    } else {
      for (size_t i = 0; i < sl.tickets.size(); ++i) {
        Req& q = S.reqs[sl.tickets[i]];
        if (rc != GM_OK) {
          finish_req(S, q, FAILED, rc);
        } else {
          q.value = S.fake ? NAN : sl.h_qout[i];
          finish_req(S, q, q.cancel_requested ? CANCELLED : DONE, q.cancel_requested ? GM_ECANCELED : GM_OK);
        }
        unref_sketch(S, S.reqs[q.a]);
        if (q.kind == GM_REQ_JACCARD) unref_sketch(S, S.reqs[q.b]);
      }
      S.arena.release(sl.in_off, sl.in_bytes);
    }
    sl.busy = false;
    sl.tickets.clear();
    --S.in_flight;
  }
  if (any) S.cv_done.notify_all();
  return any;
}

static Slot* free_slot(Server& S) {
  for (auto& sl : S.slots)
    if (!sl.busy) return &sl;
  return nullptr;
}

// ---------------------------------------------------------------------------
// Sketch batches.
// ---------------------------------------------------------------------------
struct SketchPlan {
  Slot* slot = nullptr;
  std::vector<uint64_t> tickets;  // staged requests first, then the directly copied ones
  int64_t staged = 0;             // requests copied through the staging area
  int64_t nnz = 0;
  int k = 0;
  unsigned char* in = nullptr;
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  int32_t* s_out = nullptr;
  double* y_out = nullptr;
};

// Choose and admit the next sketch batch (mutex held).  Returns false if none.
static bool plan_sketch_batch(Server& S, SketchPlan& P) {
  while (!S.sketch_q.empty() && S.reqs[S.sketch_q.front()].state != QUEUED) S.sketch_q.pop_front();
  if (S.sketch_q.empty()) return false;
  Slot* sl = free_slot(S);
  if (!sl) return false;
  const int k = S.reqs[S.sketch_q.front()].k;
  std::vector<uint64_t> pick;
  int64_t nnz = 0;
  size_t scanned = 0;
  for (auto it = S.sketch_q.begin(); it != S.sketch_q.end() && scanned < SCAN_CAP; ++it, ++scanned) {
    const Req& r = S.reqs[*it];
    if (r.state != QUEUED || r.k != k) continue;
    if ((int64_t)pick.size() >= S.cfg.max_batch_rows) break;
    if (!pick.empty() && nnz + r.nnz > S.cfg.max_batch_nnz) break;
    pick.push_back(*it);
    nnz += r.nnz;
  }
  // admission: shrink the batch until its inputs, workspace and outputs fit
  while (!pick.empty()) {
    const int64_t m = (int64_t)pick.size();
    const size_t a = in_need(m, nnz), b = ws_need(S, m, nnz, k), c = out_need(m, k);
    size_t oa, ob, oc;
    if (S.arena.alloc(a, &oa)) {
      if (S.arena.alloc(b, &ob)) {
        if (S.arena.alloc(c, &oc)) {
          sl->in_off = oa;
          sl->in_bytes = a;
          sl->ws_off = ob;
          sl->ws_bytes = b;
          OutBlock blk;
          blk.off = oc;
          blk.bytes = c;
          blk.rows = (int)m;
          blk.k = k;
          blk.live = (int)m;
          const int id = S.next_block++;
          S.blocks[id] = blk;
          sl->block = id;
          break;
        }
        S.arena.release(ob, b);
      }
      S.arena.release(oa, a);
    }
    nnz -= S.reqs[pick.back()].nnz;
    pick.pop_back();
  }
  if (pick.empty()) {
    // the oldest request does not fit now; with nothing in flight only resident
    // sketches hold the arena, so it can never fit: refuse it
    if (S.in_flight == 0) {
      Req& r = S.reqs[S.sketch_q.front()];
      finish_req(S, r, FAILED, GM_ENOMEM);
      r.released = true;
      --r.refs;  // never launched: no block to free
      S.sketch_q.pop_front();
      S.cv_done.notify_all();
      return true;  // progress
    }
    return false;
  }
  // staged requests first (they fill the staging area in queue order)
  std::vector<uint64_t> staged, direct;
  int64_t used = 0;
  for (uint64_t t : pick) {
    const Req& r = S.reqs[t];
    if (!S.fake && (!r.pinned || S.cfg.stage_pinned) && used + r.nnz <= sl->staging_elems) {
      staged.push_back(t);
      used += r.nnz;
    } else {
      direct.push_back(t);
    }
  }
  P.tickets = staged;
  P.tickets.insert(P.tickets.end(), direct.begin(), direct.end());
  S.st.staged_requests += staged.size();
  S.st.direct_requests += direct.size();
  P.staged = (int64_t)staged.size();
  P.nnz = nnz;
  P.k = k;
  P.slot = sl;
  const int64_t now = now_ns();
  for (size_t i = 0; i < P.tickets.size(); ++i) {
    Req& r = S.reqs[P.tickets[i]];
    r.state = RUNNING;
    r.t_launch = now;
    r.batch_size = (int)P.tickets.size();
    r.block = sl->block;
    r.row = (int)i;
  }
  sl->busy = true;
  sl->is_query = false;
  sl->tickets = P.tickets;
  sl->launch_rc = GM_OK;
  ++S.in_flight;
  ++S.st.sketch_batches;
  S.st.sketch_rows += P.tickets.size();
  S.st.sketch_elements += (uint64_t)nnz;
  if (!S.fake) {
    P.in = S.dev_base + sl->in_off;
    P.ws = S.dev_base + sl->ws_off;
    P.ws_bytes = sl->ws_bytes;
    unsigned char* out = S.dev_base + S.blocks[sl->block].off;
    P.s_out = reinterpret_cast<int32_t*>(out);
    P.y_out = reinterpret_cast<double*>(out + round_up((size_t)P.tickets.size() * k * 4, ALIGN));
  }
  return true;
}

// Copy the batch to the device and launch it (mutex NOT held: the requests are
// RUNNING, so nothing else touches them or the slot).
static int launch_sketch_batch(Server& S, SketchPlan& P, const std::vector<Req*>& rq) {
  const TraceRange trace("gm_server sketch batch");
  Slot& sl = *P.slot;
  const int64_t m = (int64_t)rq.size();
  int64_t* rp_d = reinterpret_cast<int64_t*>(P.in);
  int32_t* ids_d = reinterpret_cast<int32_t*>(P.in + round_up((size_t)(m + 1) * 8, ALIGN));
  double* w_d = reinterpret_cast<double*>(P.in + round_up((size_t)(m + 1) * 8, ALIGN) +
                                          round_up((size_t)P.nnz * 4, ALIGN));
  int32_t* st_ids = reinterpret_cast<int32_t*>(sl.staging);
  double* st_w = reinterpret_cast<double*>(sl.staging + round_up((size_t)sl.staging_elems * 4, ALIGN));
  int64_t e = 0;
  sl.h_rowptr[0] = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (i < P.staged && rq[i]->nnz > 0) {
      std::memcpy(st_ids + e, rq[i]->ids, (size_t)rq[i]->nnz * 4);
      std::memcpy(st_w + e, rq[i]->w, (size_t)rq[i]->nnz * 8);
    }
    e += rq[i]->nnz;
    sl.h_rowptr[i + 1] = e;
  }
  const cudaStream_t st = sl.stream;
  const int64_t staged_nnz = P.staged > 0 ? sl.h_rowptr[P.staged] : 0;
  if (cudaMemcpyAsync(rp_d, sl.h_rowptr, (size_t)(m + 1) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return GM_ECUDA;
  if (staged_nnz > 0) {
    if (cudaMemcpyAsync(ids_d, st_ids, (size_t)staged_nnz * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return GM_ECUDA;
    if (cudaMemcpyAsync(w_d, st_w, (size_t)staged_nnz * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return GM_ECUDA;
  }
  for (int64_t i = P.staged; i < m; ++i) {
    const int64_t o = sl.h_rowptr[i], n = rq[i]->nnz;
    if (n == 0) continue;
    if (cudaMemcpyAsync(ids_d + o, rq[i]->ids, (size_t)n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return GM_ECUDA;
    if (cudaMemcpyAsync(w_d + o, rq[i]->w, (size_t)n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return GM_ECUDA;
  }
  int rc;
  const int64_t t_launch = now_ns();
  if (S.cfg.params)
    rc = gm_sketch_learned(rp_d, ids_d, w_d, (int32_t)m, P.nnz, P.k, S.cfg.seed, S.cfg.flags, S.cfg.params,
                           S.cfg.margin, P.s_out, P.y_out, P.ws, P.ws_bytes, st);
  else
    rc = gm_sketch(rp_d, ids_d, w_d, (int32_t)m, P.nnz, P.k, S.cfg.seed, S.cfg.flags, P.s_out, P.y_out, P.ws,
                   P.ws_bytes, st);
  S.launch_ns_acc += (uint64_t)(now_ns() - t_launch);
  if (rc != GM_OK) return rc;
  // the workspace header's status word (written by the sketch kernels)
  if (cudaMemcpyAsync(sl.h_status, P.ws, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return GM_ECUDA;
  if (cudaEventRecord(sl.ev, st) != cudaSuccess) return GM_ECUDA;
  return GM_OK;
}

// ---------------------------------------------------------------------------
// Query batches (mutex held throughout: they are small).
// ---------------------------------------------------------------------------
static bool run_query_batch(Server& S) {
  if (S.query_q.empty()) return false;
  std::vector<uint64_t> ready, keep;
  bool progress = false;
  for (uint64_t t : S.query_q) {
    Req& q = S.reqs[t];
    if (q.state != QUEUED) continue;  // cancelled
    const Req& a = S.reqs[q.a];
    const Req* b = q.kind == GM_REQ_JACCARD ? &S.reqs[q.b] : nullptr;
    const bool bad = a.state == CANCELLED || a.state == FAILED || (b && (b->state == CANCELLED || b->state == FAILED));
    if (bad) {
      finish_req(S, q, FAILED, GM_EINVAL);
      unref_sketch(S, S.reqs[q.a]);
      if (b) unref_sketch(S, S.reqs[q.b]);
      progress = true;
      continue;
    }
    if (a.state == DONE && (!b || b->state == DONE) && (int)ready.size() < MAX_QUERIES)
      ready.push_back(t);
    else
      keep.push_back(t);
  }
  if (ready.empty()) {
    S.query_q.swap(keep);
    if (progress) S.cv_done.notify_all();
    return progress;
  }
  Slot* sl = free_slot(S);
  size_t off = 0;
  const int n = (int)ready.size();
  const size_t bytes = round_up((size_t)n * sizeof(QDesc), ALIGN) + (size_t)n * 8;
  if (!sl || !S.arena.alloc(bytes, &off)) {
    // no slot or no memory now: try again later
    keep.insert(keep.end(), ready.begin(), ready.end());
    S.query_q.swap(keep);
    if (progress) S.cv_done.notify_all();
    return progress;
  }
  S.query_q.swap(keep);
  const int64_t now = now_ns();
  for (int i = 0; i < n; ++i) {
    Req& q = S.reqs[ready[i]];
    q.state = RUNNING;
    q.t_launch = now;
    q.batch_size = n;
    if (!S.fake) {
      const Req& a = S.reqs[q.a];
      const OutBlock& ba = S.blocks[a.block];
      const unsigned char* base_a = S.dev_base + ba.off;
      QDesc d{};
      d.k = q.k;
      d.kind = q.kind;
      d.sa = reinterpret_cast<const int32_t*>(base_a) + (size_t)a.row * a.k;
      d.y = reinterpret_cast<const double*>(base_a + round_up((size_t)ba.rows * ba.k * 4, ALIGN)) +
            (size_t)a.row * a.k;
      if (q.kind == GM_REQ_JACCARD) {
        const Req& b = S.reqs[q.b];
        const OutBlock& bb = S.blocks[b.block];
        d.sb = reinterpret_cast<const int32_t*>(S.dev_base + bb.off) + (size_t)b.row * b.k;
      }
      sl->h_q[i] = d;
    }
  }
  sl->busy = true;
  sl->is_query = true;
  sl->tickets = ready;
  sl->in_off = off;
  sl->in_bytes = bytes;
  sl->launch_rc = GM_OK;
  ++S.in_flight;
  ++S.st.query_batches;
  S.st.queries += (uint64_t)n;
  if (!S.fake) {
    QDesc* qd = reinterpret_cast<QDesc*>(S.dev_base + off);
    double* out = reinterpret_cast<double*>(S.dev_base + off + round_up((size_t)n * sizeof(QDesc), ALIGN));
    const cudaStream_t st = sl->stream;
    int rc = GM_OK;
    if (cudaMemcpyAsync(qd, sl->h_q, (size_t)n * sizeof(QDesc), cudaMemcpyHostToDevice, st) != cudaSuccess)
      rc = GM_ECUDA;
    if (rc == GM_OK) {
      query_kernel<<<std::min((n + EST_BLOCK / 32 - 1) / (EST_BLOCK / 32), 152 * 8), EST_BLOCK, 0, st>>>(qd, n,
                                                                                                         out);
      if (cudaGetLastError() != cudaSuccess) rc = GM_ECUDA;
    }
    if (rc == GM_OK && cudaMemcpyAsync(sl->h_qout, out, (size_t)n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = GM_ECUDA;
    if (rc == GM_OK && cudaEventRecord(sl->ev, st) != cudaSuccess) rc = GM_ECUDA;
    sl->launch_rc = rc;
  }
  return true;
}

// ---------------------------------------------------------------------------
// The scheduler thread.
// ---------------------------------------------------------------------------
static void scheduler(Server* Sp) {
  Server& S = *Sp;
  if (!S.fake) cudaSetDevice(S.device);
  std::unique_lock<std::mutex> lk(S.mu);
  while (true) {
    bool progress = retire(S);
    if (S.stop && S.in_flight == 0) break;
    if (!S.stop && !S.paused) {
      progress |= run_query_batch(S);
      SketchPlan P;
      if (plan_sketch_batch(S, P)) {
        progress = true;
        if (P.slot) {
          std::vector<Req*> rq;
          rq.reserve(P.tickets.size());
          for (uint64_t t : P.tickets) rq.push_back(&S.reqs[t]);  // node addresses are stable
          int rc = GM_OK;
          if (!S.fake) {
            lk.unlock();
            const int64_t t0 = now_ns();
            rc = launch_sketch_batch(S, P, rq);
            S.pack_ns_acc += (uint64_t)(now_ns() - t0);
            if (rc != GM_OK) cudaStreamSynchronize(P.slot->stream);  // no copy may land after the free
            lk.lock();
          }
          P.slot->launch_rc = rc;
        }
      }
    }
    if (!progress) {
      if (S.in_flight > 0)
        S.cv_work.wait_for(lk, std::chrono::microseconds(20));
      else
        S.cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

static int validate_cfg(const gm_server_config& c) {
  if (c.n_streams < 1 || c.n_streams > 8 || c.max_batch_rows < 1 || c.max_batch_nnz < 1) return GM_EINVAL;
  if (c.max_batch_nnz > 0x7FFFFFFFll || c.device_bytes < (1u << 20)) return GM_EINVAL;
  if (c.params && !std::isfinite(c.margin)) return GM_EINVAL;
  return GM_OK;
}

static void free_all(Server* S) {
  if (!S->fake) {
    for (auto& sl : S->slots) {
      if (sl.ev) cudaEventDestroy(sl.ev);
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.staging) cudaFreeHost(sl.staging);
      if (sl.h_rowptr) cudaFreeHost(sl.h_rowptr);
      if (sl.h_status) cudaFreeHost(sl.h_status);
      if (sl.h_q) cudaFreeHost(sl.h_q);
      if (sl.h_qout) cudaFreeHost(sl.h_qout);
    }
    if (S->dev_base) cudaFree(S->dev_base);
  }
  delete S;
}

}  // namespace srv
}  // namespace gm

using gm::srv::Req;
using gm::srv::Server;

struct gm_server {
  Server* s;
};

extern "C" void gm_server_config_default(gm_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->device_bytes = (size_t)8 << 30;
  c->staging_bytes = (size_t)64 << 20;
  c->max_batch_nnz = (int64_t)1 << 23;
  c->max_batch_rows = 4096;
  c->n_streams = 4;
  c->seed = 1;
  c->flags = 0;
  c->params = nullptr;
  c->margin = 0.0f;
  c->fake_device = 0;
}

extern "C" int64_t gm_server_now_ns(void) { return gm::srv::now_ns(); }

extern "C" int gm_server_create(const gm_server_config* cfg, gm_server** out) {
  if (!cfg || !out) return GM_EINVAL;
  *out = nullptr;
  const int v = gm::srv::validate_cfg(*cfg);
  if (v != GM_OK) return v;
  Server* S = new (std::nothrow) Server();
  if (!S) return GM_ENOMEM;
  S->cfg = *cfg;
  S->fake = cfg->fake_device != 0;
  S->arena.init(cfg->device_bytes);
  S->slots.resize(cfg->n_streams);
  if (!S->fake) {
    int rc = GM_OK;
    if (cudaGetDevice(&S->device) != cudaSuccess) rc = GM_ECUDA;
    if (rc == GM_OK && cudaMalloc(&S->dev_base, S->arena.cap()) != cudaSuccess) {
      S->dev_base = nullptr;
      cudaGetLastError();
      rc = GM_ENOMEM;
    }
    const int64_t elems = (int64_t)(cfg->staging_bytes / 12);
    for (auto& sl : S->slots) {
      if (rc != GM_OK) break;
      sl.staging_elems = elems;
      const size_t stb = gm::round_up((size_t)elems * 4, gm::srv::ALIGN) + (size_t)elems * 8;
      if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
          cudaHostAlloc(reinterpret_cast<void**>(&sl.staging), stb ? stb : 16, cudaHostAllocDefault) != cudaSuccess ||
          cudaHostAlloc(reinterpret_cast<void**>(&sl.h_rowptr), ((size_t)cfg->max_batch_rows + 1) * 8,
                        cudaHostAllocDefault) != cudaSuccess ||
          cudaHostAlloc(reinterpret_cast<void**>(&sl.h_status), 16, cudaHostAllocDefault) != cudaSuccess ||
          cudaHostAlloc(reinterpret_cast<void**>(&sl.h_q), (size_t)gm::srv::MAX_QUERIES * sizeof(gm::srv::QDesc),
                        cudaHostAllocDefault) != cudaSuccess ||
          cudaHostAlloc(reinterpret_cast<void**>(&sl.h_qout), (size_t)gm::srv::MAX_QUERIES * 8,
                        cudaHostAllocDefault) != cudaSuccess)
        rc = GM_ECUDA;
    }
    if (rc != GM_OK) {
      gm::srv::free_all(S);
      return rc;
    }
  }
  S->st.arena_bytes = S->arena.cap();
  S->thread = std::thread(gm::srv::scheduler, S);
  gm_server* h = new (std::nothrow) gm_server{S};
  if (!h) {
    {
      std::lock_guard<std::mutex> g(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    S->thread.join();
    gm::srv::free_all(S);
    return GM_ENOMEM;
  }
  *out = h;
  return GM_OK;
}

extern "C" int gm_server_destroy(gm_server* h) {
  if (!h || !h->s) return GM_EINVAL;
  Server* S = h->s;
  {
    std::lock_guard<std::mutex> g(S->mu);
    for (auto& kv : S->reqs)
      if (kv.second.state == gm::srv::QUEUED) gm::srv::finish_req(*S, kv.second, gm::srv::CANCELLED, GM_ECANCELED);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->thread.join();
  gm::srv::free_all(S);
  delete h;
  return GM_OK;
}

static size_t alone_footprint(const Server& S, int64_t nnz, int k) {
  return gm::srv::in_need(1, nnz) + gm::round_up(gm::srv::ws_need(S, 1, nnz, k), gm::srv::ALIGN) +
         gm::srv::out_need(1, k);
}

extern "C" int gm_server_submit_sketch(gm_server* h, const int32_t* ids, const double* w, int64_t nnz, int32_t k,
                                       uint64_t* ticket) {
  if (!h || !h->s || !ticket || nnz < 0 || k < 1 || k > GM_MAX_K) return GM_EINVAL;
  if (nnz > 0 && (!ids || !w)) return GM_EINVAL;
  Server& S = *h->s;
  if (nnz > 0x7FFFFFFFll) return GM_EINVAL;  // one launch holds at most 2^31 - 1 elements (a larger
                                             // request runs alone in its batch)
  bool pinned = false;
  if (!S.fake && nnz > 0) {
    cudaPointerAttributes pa, pb;
    if (cudaPointerGetAttributes(&pa, ids) == cudaSuccess && cudaPointerGetAttributes(&pb, w) == cudaSuccess)
      pinned = pa.type == cudaMemoryTypeHost && pb.type == cudaMemoryTypeHost;
    cudaGetLastError();  // pageable memory may leave an error behind on old drivers
  }
  std::lock_guard<std::mutex> g(S.mu);
  if (S.stop) return GM_EINVAL;
  if (alone_footprint(S, nnz, k) > S.arena.cap()) {
    ++S.st.refused;
    return GM_ENOMEM;
  }
  const uint64_t t = S.next_ticket++;
  Req& r = S.reqs[t];
  r.kind = GM_REQ_SKETCH;
  r.k = k;
  r.nnz = nnz;
  r.ids = ids;
  r.w = w;
  r.pinned = pinned;
  r.refs = 1;
  r.t_submit = gm::srv::now_ns();
  S.sketch_q.push_back(t);
  ++S.st.submitted;
  *ticket = t;
  S.cv_work.notify_one();
  return GM_OK;
}

static int submit_query(gm_server* h, int kind, uint64_t a, uint64_t b, uint64_t* ticket) {
  if (!h || !h->s || !ticket) return GM_EINVAL;
  Server& S = *h->s;
  std::lock_guard<std::mutex> g(S.mu);
  if (S.stop) return GM_EINVAL;
  auto ia = S.reqs.find(a);
  if (ia == S.reqs.end() || ia->second.kind != GM_REQ_SKETCH || ia->second.released) return GM_EINVAL;
  Req* rb = nullptr;
  if (kind == GM_REQ_JACCARD) {
    auto ib = S.reqs.find(b);
    if (ib == S.reqs.end() || ib->second.kind != GM_REQ_SKETCH || ib->second.released) return GM_EINVAL;
    if (ib->second.k != ia->second.k) return GM_EINVAL;
    rb = &ib->second;
  } else if (ia->second.k < 2) {
    return GM_EINVAL;
  }
  const auto st_a = ia->second.state;
  if (st_a == gm::srv::CANCELLED || st_a == gm::srv::FAILED) return GM_EINVAL;
  if (rb && (rb->state == gm::srv::CANCELLED || rb->state == gm::srv::FAILED)) return GM_EINVAL;
  // the query holds a reference on each operand until it finishes
  ++ia->second.refs;
  if (rb) ++rb->refs;
  const uint64_t t = S.next_ticket++;
  Req& q = S.reqs[t];
  q.kind = kind;
  q.k = ia->second.k;
  q.a = a;
  q.b = rb ? b : 0;
  q.t_submit = gm::srv::now_ns();
  S.query_q.push_back(t);
  ++S.st.submitted;
  *ticket = t;
  S.cv_work.notify_one();
  return GM_OK;
}

extern "C" int gm_server_submit_jaccard(gm_server* h, uint64_t a, uint64_t b, uint64_t* ticket) {
  return submit_query(h, GM_REQ_JACCARD, a, b, ticket);
}

extern "C" int gm_server_submit_cardinality(gm_server* h, uint64_t a, uint64_t* ticket) {
  return submit_query(h, GM_REQ_CARDINALITY, a, 0, ticket);
}

static void fill_result(const Req& r, gm_server_result* out) {
  if (!out) return;
  out->status = r.status;
  out->kind = r.kind;
  out->k = r.k;
  out->batch_size = r.batch_size;
  out->value = r.value;
  out->t_submit_ns = r.t_submit;
  out->t_launch_ns = r.t_launch;
  out->t_done_ns = r.t_done;
}

static bool final_state(const Req& r) {
  return r.state == gm::srv::DONE || r.state == gm::srv::CANCELLED || r.state == gm::srv::FAILED;
}

extern "C" int gm_server_poll(gm_server* h, uint64_t ticket, gm_server_result* out) {
  if (!h || !h->s) return GM_EINVAL;
  Server& S = *h->s;
  std::lock_guard<std::mutex> g(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return GM_EINVAL;
  fill_result(it->second, out);
  return final_state(it->second) ? it->second.status : GM_EAGAIN;
}

extern "C" int gm_server_wait(gm_server* h, uint64_t ticket, double timeout_s, gm_server_result* out) {
  if (!h || !h->s || !(timeout_s >= 0.0)) return GM_EINVAL;
  Server& S = *h->s;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return GM_EINVAL;
  const Req& r = it->second;
  const auto until = std::chrono::steady_clock::now() +
                     std::chrono::nanoseconds((int64_t)(std::min(timeout_s, 1.0e6) * 1e9));
  while (!final_state(r))
    if (S.cv_done.wait_until(lk, until) == std::cv_status::timeout) break;
  fill_result(r, out);
  return final_state(r) ? r.status : GM_EAGAIN;
}

extern "C" int gm_server_read_sketch(gm_server* h, uint64_t ticket, int32_t* s, double* y) {
  if (!h || !h->s || !s || !y) return GM_EINVAL;
  Server& S = *h->s;
  std::lock_guard<std::mutex> g(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end() || it->second.kind != GM_REQ_SKETCH) return GM_EINVAL;
  const Req& r = it->second;
  if (r.state == gm::srv::QUEUED || r.state == gm::srv::RUNNING) return GM_EAGAIN;
  if (r.state != gm::srv::DONE || r.block < 0) return r.state == gm::srv::DONE ? GM_EINVAL : r.status;
  if (S.fake) {
    for (int j = 0; j < r.k; ++j) {
      s[j] = -1;
      y[j] = INFINITY;
    }
    return GM_OK;
  }
  const gm::srv::OutBlock& b = S.blocks[r.block];
  const unsigned char* base = S.dev_base + b.off;
  const int32_t* sd = reinterpret_cast<const int32_t*>(base) + (size_t)r.row * r.k;
  const double* yd =
      reinterpret_cast<const double*>(base + gm::round_up((size_t)b.rows * b.k * 4, gm::srv::ALIGN)) +
      (size_t)r.row * r.k;
  cudaSetDevice(S.device);
  if (cudaMemcpy(s, sd, (size_t)r.k * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GM_ECUDA;
  if (cudaMemcpy(y, yd, (size_t)r.k * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return GM_ECUDA;
  return GM_OK;
}

extern "C" int gm_server_release(gm_server* h, uint64_t ticket) {
  if (!h || !h->s) return GM_EINVAL;
  Server& S = *h->s;
  std::lock_guard<std::mutex> g(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return GM_EINVAL;
  Req& r = it->second;
  if (r.kind != GM_REQ_SKETCH) {
    if (!final_state(r)) return GM_EAGAIN;
    S.reqs.erase(it);
    return GM_OK;
  }
  if (!final_state(r)) return GM_EAGAIN;
  if (r.state != gm::srv::DONE) return GM_OK;  // failed / cancelled: already released
  if (r.released) return GM_EINVAL;
  r.released = true;
  gm::srv::unref_sketch(S, r);
  S.cv_work.notify_one();
  return GM_OK;
}

extern "C" int gm_server_cancel(gm_server* h, uint64_t ticket) {
  if (!h || !h->s) return GM_EINVAL;
  Server& S = *h->s;
  std::lock_guard<std::mutex> g(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return GM_EINVAL;
  Req& r = it->second;
  if (r.state == gm::srv::QUEUED) {
    gm::srv::finish_req(S, r, gm::srv::CANCELLED, GM_ECANCELED);
    if (r.kind == GM_REQ_SKETCH) {
      r.released = true;
      --r.refs;  // never launched: no block to free
    } else {  // drop the references the query took
      gm::srv::unref_sketch(S, S.reqs[r.a]);
      if (r.kind == GM_REQ_JACCARD) gm::srv::unref_sketch(S, S.reqs[r.b]);
    }
    S.cv_done.notify_all();
    return GM_OK;
  }
  if (r.state == gm::srv::RUNNING) {
    r.cancel_requested = true;
    return GM_OK;
  }
  return GM_EINVAL;  // already final
}

extern "C" int gm_server_stats_get(gm_server* h, gm_server_stats* out) {
  if (!h || !h->s || !out) return GM_EINVAL;
  Server& S = *h->s;
  std::lock_guard<std::mutex> g(S.mu);
  *out = S.st;
  out->arena_bytes = S.arena.cap();
  out->arena_peak_bytes = S.arena.peak();
  out->arena_resident_bytes = S.resident_bytes();
  uint64_t q = 0;
  for (const auto& kv : S.reqs) q += kv.second.state == gm::srv::QUEUED;
  out->queued = q;
  out->in_flight_batches = (uint64_t)S.in_flight;
  out->pack_ns = S.pack_ns_acc.load();
  out->launch_ns = S.launch_ns_acc.load();
  return GM_OK;
}

extern "C" int gm_server_pause(gm_server* h, int32_t paused) {
  if (!h || !h->s) return GM_EINVAL;
  Server& S = *h->s;
  {
    std::lock_guard<std::mutex> g(S.mu);
    S.paused = paused != 0;
  }
  S.cv_work.notify_one();
  return GM_OK;
}
