// gm_host.cu -- gm_sketch over a CSR batch in host memory, pipelined: chunks of
// rows are copied in, sketched and copied out on two streams, so the transfers
// of one chunk overlap the sketch of the next.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "gm.h"
#include "gm_internal.h"
#include "gm_trace.h"

namespace gm {
namespace host {

// Measured on the 4,096-row lognormal batch at k = 1024 (pinned host buffers,
// 207 GB/s host-to-device): 2 slots x 4 chunks 3.72 ms per batch, 4 x 8 3.27 ms,
// 8 x 16 3.14 ms (the device-resident sketch: 2.89 ms).  With as many slots as
// the copies need, the copy of one chunk, the kernels of several and the copy
// back of another all overlap, and a chunk's kernel fills the SMs that the tail
// of the previous chunk's kernel leaves idle.
#ifndef GM_HOST_SLOTS
#define GM_HOST_SLOTS 8
#endif
#ifndef GM_HOST_CHUNKS
#define GM_HOST_CHUNKS 16
#endif
#ifndef GM_HOST_CHUNK_ROWS
#define GM_HOST_CHUNK_ROWS 128
#endif
constexpr int SLOTS = GM_HOST_SLOTS;  // chunks in flight (each its own stream and device buffers)
constexpr int CHUNKS_MIN = GM_HOST_CHUNKS;            // a batch is cut into at least this many chunks ...
constexpr int32_t CHUNK_ROWS_MIN = GM_HOST_CHUNK_ROWS;  // ... of at least this many rows
constexpr size_t ALIGN = 256;

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int64_t* h_rowptr = nullptr;  // pinned, rebased row offsets of the chunk
  uint32_t* h_status = nullptr;  // pinned, the chunk's workspace status word
  int32_t cap_rows = 0;
};

struct State {
  std::mutex mu;  // one pipelined call at a time per process
  int device = -1;
  Slot slots[SLOTS];
};
static State g_state;

static void free_slots(State& S) {
  for (Slot& s : S.slots) {
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.h_rowptr) cudaFreeHost(s.h_rowptr);
    if (s.h_status) cudaFreeHost(s.h_status);
    s = Slot();
  }
}

static int ensure_slots(State& S, int32_t rows) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GM_ECUDA;
  if (S.device != dev) {
    free_slots(S);
    S.device = dev;
  }
  for (Slot& s : S.slots) {
    if (!s.stream && (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
                      cudaHostAlloc(reinterpret_cast<void**>(&s.h_status), 16, cudaHostAllocDefault) != cudaSuccess))
      return GM_ECUDA;
    if (s.cap_rows < rows) {
      if (s.h_rowptr) cudaFreeHost(s.h_rowptr);
      s.h_rowptr = nullptr;
      if (cudaHostAlloc(reinterpret_cast<void**>(&s.h_rowptr), ((size_t)rows + 1) * 8, cudaHostAllocDefault) !=
          cudaSuccess)
        return GM_ECUDA;
      s.cap_rows = rows;
    }
  }
  return GM_OK;
}

// Device layout of one slot: row_ptr | ids | w | s | y | sketch workspace.
struct SlotMem {
  int64_t* row_ptr;
  int32_t* ids;
  double* w;
  int32_t* s;
  double* y;
  void* ws;
  size_t ws_bytes;
};
static size_t slot_bytes(int32_t rows, int64_t nnz, int32_t k) {
  return round_up(((size_t)rows + 1) * 8, ALIGN) + round_up((size_t)nnz * 4, ALIGN) +
         round_up((size_t)nnz * 8, ALIGN) + round_up((size_t)rows * k * 4, ALIGN) +
         round_up((size_t)rows * k * 8, ALIGN) + round_up(ws_bytes(rows, nnz, k), ALIGN);
}
static SlotMem slot_mem(unsigned char* base, int32_t rows, int64_t nnz, int32_t k) {
  SlotMem m;
  size_t o = 0;
  m.row_ptr = reinterpret_cast<int64_t*>(base + o);
  o += round_up(((size_t)rows + 1) * 8, ALIGN);
  m.ids = reinterpret_cast<int32_t*>(base + o);
  o += round_up((size_t)nnz * 4, ALIGN);
  m.w = reinterpret_cast<double*>(base + o);
  o += round_up((size_t)nnz * 8, ALIGN);
  m.s = reinterpret_cast<int32_t*>(base + o);
  o += round_up((size_t)rows * k * 4, ALIGN);
  m.y = reinterpret_cast<double*>(base + o);
  o += round_up((size_t)rows * k * 8, ALIGN);
  m.ws = base + o;
  m.ws_bytes = round_up(ws_bytes(rows, nnz, k), ALIGN);
  return m;
}

static int32_t chunk_rows(int32_t n_rows) {
  int32_t c = (n_rows + CHUNKS_MIN - 1) / CHUNKS_MIN;
  if (c < CHUNK_ROWS_MIN) c = CHUNK_ROWS_MIN;
  return c < n_rows ? c : n_rows;
}

// The most elements any chunk of `rows` rows holds (row_ptr ascending).
static int64_t max_chunk_nnz(const int64_t* row_ptr, int32_t n_rows, int32_t rows) {
  int64_t m = 0;
  for (int32_t r0 = 0; r0 < n_rows; r0 += rows) {
    const int32_t r1 = r0 + rows < n_rows ? r0 + rows : n_rows;
    const int64_t c = row_ptr[r1] - row_ptr[r0];
    m = c > m ? c : m;
  }
  return m;
}

// Valid host row offsets: start at 0, end at nnz, never decrease.
static bool rows_valid(const int64_t* row_ptr, int32_t n_rows, int64_t nnz) {
  if (row_ptr[0] != 0 || row_ptr[n_rows] != nnz) return false;
  for (int32_t r = 0; r < n_rows; ++r)
    if (row_ptr[r + 1] < row_ptr[r]) return false;
  return true;
}

}  // namespace host
}  // namespace gm

using namespace gm::host;

extern "C" size_t gm_sketch_host_workspace_bytes(int32_t n_rows, int64_t nnz, int32_t k) {
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K) return 0;
  const int32_t rows = chunk_rows(n_rows > 0 ? n_rows : 1);
  return (size_t)SLOTS * slot_bytes(rows, nnz, k);  // a chunk may hold every element
}

extern "C" size_t gm_sketch_host_workspace_bytes_csr(const int64_t* row_ptr, int32_t n_rows, int32_t k) {
  if (!row_ptr || n_rows < 0 || k < 1 || k > GM_MAX_K) return 0;
  const int64_t nnz = row_ptr[n_rows];
  if (nnz < 0 || !rows_valid(row_ptr, n_rows, nnz)) return 0;
  const int32_t rows = chunk_rows(n_rows > 0 ? n_rows : 1);
  return (size_t)SLOTS * slot_bytes(rows, n_rows > 0 ? max_chunk_nnz(row_ptr, n_rows, rows) : 0, k);
}

extern "C" int gm_sketch_host(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows,
                              int64_t nnz, int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out,
                              void* workspace, size_t workspace_bytes) {
  if (n_rows < 0 || nnz < 0 || k < 1 || k > GM_MAX_K || nnz > 0x7FFFFFFFll) return GM_EINVAL;
  if (!row_ptr || !workspace || !gm::ws_aligned(workspace) || (n_rows > 0 && (!s_out || !y_out)) ||
      (nnz > 0 && (!ids || !w)))
    return GM_EINVAL;
  if (!rows_valid(row_ptr, n_rows, nnz)) return GM_EINVAL;
  const int32_t rows = chunk_rows(n_rows > 0 ? n_rows : 1);
  const int64_t cap = n_rows > 0 ? max_chunk_nnz(row_ptr, n_rows, rows) : 0;  // elements per slot
  if (workspace_bytes < (size_t)SLOTS * slot_bytes(rows, cap, k)) return GM_ENOMEM;
  if (n_rows == 0) return GM_OK;
  const gm::TraceRange trace("gm_sketch_host");
  State& S = g_state;
  std::lock_guard<std::mutex> lock(S.mu);
  int rc = ensure_slots(S, rows);
  if (rc != GM_OK) return rc;
  const size_t per_slot = slot_bytes(rows, cap, k);
  unsigned char* base = static_cast<unsigned char*>(workspace);
  bool used[SLOTS] = {};
  int first_err = GM_OK;
  // on an error, let the work already queued finish before returning (it writes
  // into the caller's buffers)
  auto drain = [&](int code) {
    for (int i = 0; i < SLOTS; ++i)
      if (used[i]) cudaStreamSynchronize(S.slots[i].stream);
    return code;
  };
  int c = 0;
  for (int32_t r0 = 0; r0 < n_rows && first_err == GM_OK; r0 += rows, ++c) {
    const int32_t r1 = r0 + rows < n_rows ? r0 + rows : n_rows;
    const int32_t m = r1 - r0;
    Slot& sl = S.slots[c % SLOTS];
    if (used[c % SLOTS]) {  // the slot's previous chunk must be out before its buffers are reused
      if (cudaEventSynchronize(sl.done) != cudaSuccess) return drain(GM_ECUDA);
      if (*sl.h_status) first_err = (*sl.h_status & gm::WS_EDATA) ? GM_EDATA : GM_ETIMEOUT;
    }
    used[c % SLOTS] = true;
    const int64_t lo = row_ptr[r0], n = row_ptr[r1] - lo;
    for (int32_t i = 0; i <= m; ++i) sl.h_rowptr[i] = row_ptr[r0 + i] - lo;
    const SlotMem dm = slot_mem(base + (size_t)(c % SLOTS) * per_slot, rows, cap, k);
    const cudaStream_t st = sl.stream;
    if (cudaMemcpyAsync(dm.row_ptr, sl.h_rowptr, ((size_t)m + 1) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (n > 0 && cudaMemcpyAsync(dm.ids, ids + lo, (size_t)n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        (n > 0 && cudaMemcpyAsync(dm.w, w + lo, (size_t)n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess))
      return drain(GM_ECUDA);
    rc = gm::launch_sketch(dm.row_ptr, dm.ids, dm.w, m, n, k, seed, flags, dm.s, dm.y, dm.ws, dm.ws_bytes, st, false,
                           nullptr);
    if (rc != GM_OK) return drain(rc);
    if (cudaMemcpyAsync(sl.h_status, dm.ws, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(s_out + (size_t)r0 * k, dm.s, (size_t)m * k * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(y_out + (size_t)r0 * k, dm.y, (size_t)m * k * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(sl.done, st) != cudaSuccess)
      return drain(GM_ECUDA);
  }
  if (first_err != GM_OK) return drain(first_err);
  for (int i = 0; i < SLOTS; ++i)
    if (used[i]) {
      if (cudaEventSynchronize(S.slots[i].done) != cudaSuccess) return GM_ECUDA;
      if (*S.slots[i].h_status && first_err == GM_OK)
        first_err = (*S.slots[i].h_status & gm::WS_EDATA) ? GM_EDATA : GM_ETIMEOUT;
    }
  return first_err;
}
