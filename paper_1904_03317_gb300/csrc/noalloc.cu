// Level smoothing whose recurrence vector lives in a static device array, for
// callers that must not allocate device memory while they run: processes
// whose device memory is owned by another allocator (a framework's caching
// allocator, or a fixed memory budget), and latency-critical loops that cannot
// afford the device-wide synchronisation cudaMalloc and cudaFree imply.
#include <cuda_runtime.h>

#include <string>

#include "gmg_internal.h"

#define GMG_NOALLOC_SCRATCH_BYTES (8u << 20)

namespace gmg {

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GMG_NOALLOC_SCRATCH_BYTES];

// In host code the array's name is only a host-side stand-in, so its device
// address comes from cudaGetSymbolAddress, with the hierarchy's device
// current.  The lookup loads the module that holds the array (its 8 MiB are
// allocated then, if this process has not loaded it on this device yet), so
// it runs while the hierarchy is built, where allocating is expected; the
// no-allocation entry point only uses the address kept here.  The address
// belongs to the context current during the build, the same context that owns
// the hierarchy's other device memory.
gmg_status noalloc_prepare(Hier& h) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("static smoothing scratch: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return GMG_ECUDA;
  }
  h.noalloc_scratch = p;
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
  if (d_g == d_u) {
    set_error("gmg_level_smooth_noalloc: g and u must not alias");
    return GMG_EINVAL;
  }
  Hier& h = hh->h;
  if (!h.ctx || h.ctx->c.device < 0 || !h.dev || !h.noalloc_scratch) {
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
  // the smoothing driver clears (from zero) or fills (from a start value) the
  // part of the array it uses before reading it
  return device_level_smooth(h, level, d_g, d_u, h.noalloc_scratch, from_zero);
}
