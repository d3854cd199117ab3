// pvsc_cheb_step_noalloc: the fused Chebyshev step for callers that cannot
// allocate device memory.
//
// pvsc_cheb_step needs a caller-provided work buffer for the per-block dot
// product partials and the arrival counter of its last-block reduction.  Some
// callers have no way to provide one: code that runs after start-up under a
// fixed device-memory budget (a framework whose pool already owns the free
// memory), callbacks and plugins that must not call cudaMalloc because it can
// synchronise the whole device, and hosts that forbid allocation once they are
// initialised.  This entry point instead uses a fixed-size scratch array that
// lives in the library image as a file-scope __device__ variable, so nothing
// is allocated by the library or by the caller.
//
// The array is kNoAllocScratchBytes = 2 MiB.  In host code its name is only a
// host-side stand-in, never a device address: every call looks the device
// address up with cudaGetSymbolAddress, with the lattice's device current (a
// cheap host call once the module is loaded; nothing is cached, so the address
// stays right after cudaDeviceReset reloads the module).  The first call on a
// device loads the module there: make it before any stream capture.  Every
// call on a device shares the one array and it keeps
// the contents the previous call left; the arrival counter at its start is
// cleared (cudaMemsetAsync on the caller's stream) before each sweep.  Calls
// whose kernels overlap on the GPU (different streams, no ordering) race on
// the array: order them on one stream or synchronise between them.
#include "internal.h"

namespace pvsc {

constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device.
static int noalloc_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return set_error(PVSC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                     cudaGetErrorString(e));
  *out = p;
  return PVSC_OK;
}

}  // namespace pvsc

using namespace pvsc;

extern "C" int pvsc_cheb_step_noalloc(const pvsc_lattice* lat, int R, int prec, const void* x,
                                      void* y, void* z, const double* alpha, const double* beta,
                                      const double* gamma, const double* delta, int dot_flags,
                                      double* dots, void* stream) {
  if (int rc = check_lattice(lat)) return rc;
  if (!valid_R(R)) return set_error(PVSC_ERR_ARG, "R = %d: must be 1, 2, 4, 8, 16, 32 or 64", R);
  int device = -1;
  PVSC_CUDA_TRY(cudaGetDevice(&device));
  if (device != lat->device)
    return set_error(PVSC_ERR_ARG, "current device %d is not the lattice's device %d", device,
                     lat->device);
  if (dot_flags == 0)  // no reduction, no scratch
    return pvsc_cheb_step(lat, R, prec, x, y, z, alpha, beta, gamma, delta, 0, dots, nullptr, 0,
                          stream);
  const size_t need = dots_work_bytes(lat, R);
  if (need > kNoAllocScratchBytes)
    return set_error(PVSC_ERR_ARG,
                     "pvsc_cheb_step_noalloc: R = %d needs %zu bytes of scratch on this device, "
                     "more than the static %zu bytes; use pvsc_cheb_step with a work buffer",
                     R, need, kNoAllocScratchBytes);
  void* scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  return pvsc_cheb_step(lat, R, prec, x, y, z, alpha, beta, gamma, delta, dot_flags, dots, scratch,
                        kNoAllocScratchBytes, stream);
}
