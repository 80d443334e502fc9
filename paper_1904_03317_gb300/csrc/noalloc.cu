// Level smoothing whose recurrence vector lives in a static device array, for
// callers that must not allocate device memory while they run: processes
// whose device memory is owned by another allocator (a framework's caching
// allocator, or a fixed memory budget), and latency-critical loops that cannot
// afford the device-wide synchronisation cudaMalloc and cudaFree imply.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gmg_internal.h"

#define GMG_NOALLOC_SCRATCH_BYTES (8u << 20)

namespace gmg {

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GMG_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[128] = {};

// Device address of the array on `device` (which must be current).  In host
// code the array's name is only a host-side stand-in, so the address comes
// from cudaGetSymbolAddress, once per device.
static gmg_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= 128) {
    set_error("gmg_level_smooth_noalloc: device index out of range");
    return GMG_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("gmg_level_smooth_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return GMG_ECUDA;
    }
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return GMG_OK;
}

}  // namespace gmg

using namespace gmg;

extern "C" gmg_status gmg_level_smooth_noalloc(gmg_hier* hh, int level, const void* d_g, void* d_u,
                                               int from_zero) {
  if (!hh || !d_g || !d_u) {
    set_error("gmg_level_smooth_noalloc: null argument");
    return GMG_EINVAL;
  }
  Hier& h = hh->h;
  if (!h.ctx || h.ctx->c.device < 0 || !h.dev) {
    set_error("gmg_level_smooth_noalloc: needs a hierarchy built on a device context");
    return GMG_EINVAL;
  }
  if (level < 1 || level > h.L) {
    set_error("gmg_level_smooth_noalloc: level out of range");
    return GMG_EINVAL;
  }
  const size_t esz = h.params.vcycle_prec == GMG_PREC_FP32 ? sizeof(float) : sizeof(double);
  const size_t need = h.levels[level].slot_class.size() * esz;
  if (need > GMG_NOALLOC_SCRATCH_BYTES) {
    set_error("gmg_level_smooth_noalloc: level " + std::to_string(level) + " needs " + std::to_string(need) +
              " bytes of scratch; the static scratch holds " + std::to_string(GMG_NOALLOC_SCRATCH_BYTES) +
              " (use gmg_level_smooth with a caller buffer)");
    return GMG_EINVAL;
  }
  cudaError_t e = cudaSetDevice(h.ctx->c.device);
  if (e != cudaSuccess) {
    set_error(std::string("gmg_level_smooth_noalloc: cudaSetDevice: ") + cudaGetErrorString(e));
    return GMG_ECUDA;
  }
  void* tmp = nullptr;
  gmg_status st = noalloc_scratch(h.ctx->c.device, &tmp);
  if (st != GMG_OK) return st;
  // the smoothing driver clears (from zero) or fills (from a start value) the
  // part of the array it uses before reading it
  return device_level_smooth(h, level, d_g, d_u, tmp, from_zero);
}
