// gm_internal.h -- workspace layout shared by the libgm translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace gm {

// arrivals, elements, screened, warp-path elements, escalated passes, CAS retries, then the
// summed per-warp clocks of the light, 8-lane, 32-lane, dense phases, barrier waits, row setup,
// row finish and the total, then the kept arrivals (those within the bound) and the short rows
// whose first-pass bound was below y*
constexpr int WS_NCOUNTERS = 16;
constexpr uint32_t WS_EDATA = 1u;
constexpr uint32_t WS_ETIMEOUT = 2u;
constexpr int SPLIT_LEN = 32768;  // rows longer than this are long rows, cut into chunks
constexpr int PIECE_LEN = 4096;   // long rows' pre-pass pieces (one warp each); chunks are whole pieces

// Start of every workspace; zeroed by the first kernel of each call.
struct WsHeader {
  uint32_t status;        // WS_* bits
  uint32_t unit_counter;  // next work unit of the persistent grid
  uint32_t n_long;        // rows longer than SPLIT_LEN
  uint32_t n_extra;       // chunk units of long rows beyond their first chunk
  uint32_t esc_count;     // long rows to redo with a larger bound
  uint32_t esc_counter;   // next entry of that list
  uint32_t n_pieces;      // pre-pass pieces of all long rows
  uint32_t n_hunits;      // compacted long rows: units of heavy and super-heavy elements (dispatched first)
  uint32_t cunit;         // compacted long rows: entries of a compact list per chunk unit
  uint32_t pad;
  unsigned long long counters[WS_NCOUNTERS];
};

// Per long row: its row index, chunk count, first extra unit, sum of weights.
// The sums are added from the row's pre-pass pieces in piece order, so they are
// the same bits on every call.
struct LongRow {
  uint32_t row;
  uint32_t nchunks;
  uint32_t chunk_off;    // index of its first extra unit (chunks 1 .. nchunks-1)
  uint32_t done;         // chunks finished
  float sum;             // sum of positive weights (FP32, places the bound only)
  int npos;              // positive weights
  double dsum;           // FP64 sum of the positive weights (budget passes only)
  uint32_t piece_off;    // index of its first pre-pass piece
  uint32_t npieces;      // pieces of PIECE_LEN elements
  uint32_t pieces_done;  // pieces summed so far
  uint32_t ncomp;        // compacted mode: light and medium elements left after the first-arrival screen
  uint32_t nsuper;       // compacted mode: super-heavy elements, listed at the back of the row's plist range
  uint32_t nheavy;       // compacted mode: heavy elements, listed at the back of the row's work list
  uint32_t heavy_off;    // compacted mode: index of its first heavy unit
  uint32_t nhunits;      // compacted mode: its units of heavy elements, then one per super-heavy element
};

// Sums of one pre-pass piece of a long row.
struct LongPiece {
  float sum;
  int npos;
  double dsum;
};

constexpr size_t WS_HEADER_BYTES = 256;

constexpr size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int64_t max_long_rows(int64_t nnz) { return nnz / (SPLIT_LEN + 1) + 1; }
constexpr int64_t max_pieces(int64_t nnz) { return nnz / PIECE_LEN + max_long_rows(nnz) + 1; }

// Workspace: header | C table (k doubles) | work list (nnz u32) | promotion list
// (nnz u32) | long index per row (n_rows i32) | long rows (max_long) | long
// registers (max_long * k * 16 B) | escalation list (max_long u32) | piece sums
// (max_pieces)
struct WsLayout {
  WsHeader* hdr;
  double* ctab;
  uint32_t* list;
  uint32_t* plist;
  int32_t* long_idx;
  LongRow* longs;
  void* long_regs;
  uint32_t* esc;
  LongPiece* parts;
  int64_t max_long;
};

inline WsLayout ws_layout(void* ws, int32_t n_rows, int64_t nnz, int k) {
  unsigned char* p = static_cast<unsigned char*>(ws);
  WsLayout L;
  const int64_t ml = max_long_rows(nnz);
  size_t off = 0;
  L.hdr = reinterpret_cast<WsHeader*>(p + off);
  off += WS_HEADER_BYTES;
  L.ctab = reinterpret_cast<double*>(p + off);
  off += round_up((size_t)k * 8, 256);
  L.list = reinterpret_cast<uint32_t*>(p + off);
  off += round_up((size_t)nnz * 4, 256);
  L.plist = reinterpret_cast<uint32_t*>(p + off);
  off += round_up((size_t)nnz * 4, 256);
  L.long_idx = reinterpret_cast<int32_t*>(p + off);
  off += round_up((size_t)n_rows * 4, 256);
  L.longs = reinterpret_cast<LongRow*>(p + off);
  off += round_up((size_t)ml * sizeof(LongRow), 256);
  L.long_regs = p + off;
  off += round_up((size_t)ml * (size_t)k * 16, 256);
  L.esc = reinterpret_cast<uint32_t*>(p + off);
  off += round_up((size_t)ml * 4, 256);
  L.parts = reinterpret_cast<LongPiece*>(p + off);
  L.max_long = ml;
  return L;
}

constexpr size_t ws_bytes(int32_t n_rows, int64_t nnz, int k) {
  return WS_HEADER_BYTES + round_up((size_t)k * 8, 256) + 2 * round_up((size_t)nnz * 4, 256) +
         round_up((size_t)n_rows * 4, 256) + round_up((size_t)max_long_rows(nnz) * sizeof(LongRow), 256) +
         round_up((size_t)max_long_rows(nnz) * (size_t)k * 16, 256) + round_up((size_t)max_long_rows(nnz) * 4, 256) +
         round_up((size_t)max_pieces(nnz) * sizeof(LongPiece), 256);
}

// Caller workspaces start on a 256-byte boundary (every region inside is laid
// out at 256-byte offsets; 16-byte atomics and vector loads rely on it).
inline bool ws_aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

// The sketch launcher behind gm_sketch, gm_sketch_plain, gm_sketch_noalloc and
// gm_sketch_learned.  t_row: per-row first-pass bounds (device floats) or null
// for the closed-form bound.
int launch_sketch(const int64_t* row_ptr, const int32_t* ids, const double* w, int32_t n_rows, int64_t nnz,
                  int32_t k, uint64_t seed, uint32_t flags, int32_t* s_out, double* y_out, void* workspace,
                  size_t workspace_bytes, cudaStream_t stream, bool plain, const float* t_row);

// Events that gm_diag_time_aux_kernels registered (null when unset): the estimator
// and learned pre-pass entry points record them before their first and after their
// last kernel.
void aux_events(cudaEvent_t* before, cudaEvent_t* after);

// Entries per dense permutation: k rounded up to a multiple of 8, so that each
// array starts on a 16-byte boundary (16-byte stores).
__host__ __device__ inline size_t pi_stride(int k) { return ((size_t)k + 7) / 8 * 8; }

}  // namespace gm
