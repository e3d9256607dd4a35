// gm_internal.h -- workspace layout shared by the libgm translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace gm {

constexpr int WS_NCOUNTERS = 6;  // arrivals, elements, screened, heavy, escalated, cas retries
constexpr uint32_t WS_EDATA = 1u;
constexpr uint32_t WS_ETIMEOUT = 2u;

// Start of every workspace; zeroed by the first kernel of each call.
struct WsHeader {
  uint32_t status;       // WS_* bits
  uint32_t row_counter;  // next row for the persistent grid
  uint32_t pad[2];
  unsigned long long counters[WS_NCOUNTERS];
};

constexpr size_t WS_HEADER_BYTES = 256;

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Workspace: header | C table (k doubles) | heavy list (nnz u32)
struct WsLayout {
  WsHeader* hdr;
  double* ctab;
  uint32_t* heavy;
};

inline size_t ws_bytes(int64_t nnz, int k) {
  return WS_HEADER_BYTES + round_up((size_t)k * 8, 256) + round_up((size_t)nnz * 4, 256);
}

inline WsLayout ws_layout(void* ws, int64_t nnz, int k) {
  (void)nnz;
  unsigned char* p = static_cast<unsigned char*>(ws);
  WsLayout L;
  L.hdr = reinterpret_cast<WsHeader*>(p);
  L.ctab = reinterpret_cast<double*>(p + WS_HEADER_BYTES);
  L.heavy = reinterpret_cast<uint32_t*>(p + WS_HEADER_BYTES + round_up((size_t)k * 8, 256));
  return L;
}

// Shared memory of the sketch kernel besides the registers: the light lanes'
// sparse maps (32 entries x 256 lanes x 4 B) or, reusing the same bytes, the
// warps' dense permutations (8 warps x k x 2 B).
__host__ __device__ inline size_t area_size_bytes(int k) {
  size_t a = (size_t)32 * 256 * 4, b = (size_t)8 * (size_t)k * 2;
  size_t m = a > b ? a : b;
  return (m + 15) / 16 * 16;
}

}  // namespace gm
