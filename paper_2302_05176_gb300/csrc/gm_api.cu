// gm_api.cu -- status read-back, error strings and version of libgm.
#include <cuda_runtime.h>

#include <cstring>

#include "gm.h"
#include "gm_internal.h"
#include "gm_server.h"

extern "C" int gm_status(const void* workspace, gm_stats* stats, void* stream) {
  if (!workspace) return GM_EINVAL;
  gm::WsHeader h;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GM_ECUDA;
  const int code = (h.status & gm::WS_EDATA) ? GM_EDATA : (h.status & gm::WS_ETIMEOUT) ? GM_ETIMEOUT : GM_OK;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->arrivals = h.counters[0];
    stats->elements = h.counters[1];
    stats->screened_out = h.counters[2];
    stats->heavy_elements = h.counters[3];
    stats->rows_escalated = h.counters[4];
    stats->cas_retries = h.counters[5];
    stats->cycles_light = h.counters[6];
    stats->cycles_medium = h.counters[7];
    stats->cycles_heavy = h.counters[8];
    stats->cycles_dense = h.counters[9];
    stats->cycles_wait = h.counters[10];
    stats->cycles_setup = h.counters[11];
    stats->cycles_finish = h.counters[12];
    stats->cycles_total = h.counters[13];
    stats->kept = h.counters[14];
    stats->rows_fallback = h.counters[15] + h.esc_count;
    stats->status = (uint32_t)code;
  }
  return code;
}

extern "C" const char* gm_strerror(int code) {
  switch (code) {
    case GM_OK: return "ok";
    case GM_EINVAL: return "invalid argument";
    case GM_ENOMEM: return "workspace too small";
    case GM_ECUDA: return "CUDA error";
    case GM_ETIMEOUT: return "device retry limit reached";
    case GM_EDATA: return "invalid input data";
    case GM_EAGAIN: return "not finished yet";
    case GM_ECANCELED: return "cancelled";
    default: return "unknown status";
  }
}

extern "C" const char* gm_version(void) { return "libgm 0.1 sm_103a"; }
