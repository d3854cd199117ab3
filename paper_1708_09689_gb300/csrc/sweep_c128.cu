// complex128 storage, fp64 arithmetic: kernel instantiations and launchers
// (register-marching, flat, cp.async-prefetching and shared-memory staged TI
// sweeps; graphene sweep).
#include <mutex>
#include <set>

#include "internal.h"
#include "sweep.cuh"
#include "sweep_bulk.cuh"

namespace pvsc {

template <int MODEL, int FEAT>
static void* kernel_c128() {
  if constexpr (MODEL == 1) return reinterpret_cast<void*>(&ti_sweep<double, 1, FEAT>);
  else if constexpr (MODEL == kModelTIFlat) return reinterpret_cast<void*>(&ti_sweep_flat<double, 1, FEAT>);
  else if constexpr (MODEL == kModelTIAsync)
    return reinterpret_cast<void*>(&ti_sweep<double, 1, FEAT, kAsyncDepth, 6>);
  else if constexpr (MODEL == kModelTIAsyncDeep)
    return reinterpret_cast<void*>(&ti_sweep<double, 1, FEAT, kAsyncDeepDepth, 2>);
  else if constexpr (MODEL == kModelWSM) return reinterpret_cast<void*>(&wsm_sweep<double, 1, FEAT>);
  else if constexpr (MODEL == kModelWSMMarch) return reinterpret_cast<void*>(&wsm_march_sweep<double, 1, FEAT>);
  else if constexpr (MODEL == kModelGrapheneQD) return reinterpret_cast<void*>(&gr_sweep<double, 1, FEAT, true>);
  else if constexpr (MODEL == kModelTIXMarch) return reinterpret_cast<void*>(&ti_sweep_xmarch<double, 1, FEAT>);
  else return reinterpret_cast<void*>(&gr_sweep<double, 1, FEAT>);
}

template <int MODEL>
static void* pick_c128(int feat) {
  switch (feat) {
    case 0: return kernel_c128<MODEL, 0>();
    case F_DOTS: return kernel_c128<MODEL, F_DOTS>();
    case F_Z: return kernel_c128<MODEL, F_Z>();
    case F_DOTS | F_Z: return kernel_c128<MODEL, F_DOTS | F_Z>();
    case F_ACC: return kernel_c128<MODEL, F_ACC>();
    case F_ADJ: return kernel_c128<MODEL, F_ADJ>();
    default: return nullptr;
  }
}

static void* pick(int model, int feat) {
  switch (model) {
    case 1: return pick_c128<1>(feat);
    case kModelTIFlat: return pick_c128<kModelTIFlat>(feat);
    case kModelTIAsync: return pick_c128<kModelTIAsync>(feat);
    case kModelTIAsyncDeep: return pick_c128<kModelTIAsyncDeep>(feat);
    case kModelWSM: return pick_c128<kModelWSM>(feat);
    case kModelWSMMarch: return pick_c128<kModelWSMMarch>(feat);
    case kModelGrapheneQD: return pick_c128<kModelGrapheneQD>(feat);
    case kModelTIXMarch: return pick_c128<kModelTIXMarch>(feat);
    default: return pick_c128<2>(feat);
  }
}

// Opt a kernel into the device's full dynamic shared memory (once per kernel).
int allow_max_smem(void* fn) {
  static std::mutex mu;
  static std::set<void*> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(fn)) return PVSC_OK;
  int dev = 0, optin = 0;
  PVSC_CUDA_TRY(cudaGetDevice(&dev));
  PVSC_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  PVSC_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
  PVSC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes));
  done.insert(fn);
  return PVSC_OK;
}

int launch_sweep_c128(int model, int feat, int grid, int threads, const Sweep& p,
                      cudaStream_t st) {
  void* fn = pick(model, feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no complex128 sweep for feature set %d", feat);
  const size_t smem = async_ring_bytes(model, threads);
  if (smem)
    if (int rc = allow_max_smem(fn)) return rc;
  void* args[] = {const_cast<Sweep*>(&p)};
  PVSC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st));
  return PVSC_OK;
}

int occupancy_c128(int model, int feat, int threads, int* blocks) {
  void* fn = pick(model, feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no complex128 sweep for feature set %d", feat);
  const size_t smem = async_ring_bytes(model, threads);
  if (smem)
    if (int rc = allow_max_smem(fn)) return rc;
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem));
  return PVSC_OK;
}

// ---------------------------------------------------------------- shared-memory staged TI sweep
static void* pick_bulk_c128(int feat) {
  switch (feat) {
    case 0: return reinterpret_cast<void*>(&ti_sweep_bulk<double, 0>);
    case F_DOTS: return reinterpret_cast<void*>(&ti_sweep_bulk<double, F_DOTS>);
    case F_Z: return reinterpret_cast<void*>(&ti_sweep_bulk<double, F_Z>);
    case F_DOTS | F_Z: return reinterpret_cast<void*>(&ti_sweep_bulk<double, F_DOTS | F_Z>);
    case F_ACC: return reinterpret_cast<void*>(&ti_sweep_bulk<double, F_ACC>);
    case F_ADJ: return reinterpret_cast<void*>(&ti_sweep_bulk<double, F_ADJ>);
    default: return nullptr;
  }
}

int launch_sweep_bulk_c128(int feat, int grid, int threads, size_t smem, const Sweep& p,
                           cudaStream_t st) {
  void* fn = pick_bulk_c128(feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no staged complex128 sweep for feature set %d", feat);
  if (int rc = allow_max_smem(fn)) return rc;
  void* args[] = {const_cast<Sweep*>(&p)};
  PVSC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st));
  return PVSC_OK;
}

int occupancy_bulk_c128(int feat, int threads, size_t smem, int* blocks) {
  void* fn = pick_bulk_c128(feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no staged complex128 sweep for feature set %d", feat);
  if (int rc = allow_max_smem(fn)) return rc;
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem));
  return PVSC_OK;
}

int bulk_error_c128(int clear, int* flag) {
  int h = 0;
  PVSC_CUDA_TRY(cudaMemcpyFromSymbol(&h, g_bulk_sweep_error, sizeof(int)));
  if (clear) {
    const int z = 0;
    PVSC_CUDA_TRY(cudaMemcpyToSymbol(g_bulk_sweep_error, &z, sizeof(int)));
  }
  *flag = h;
  return PVSC_OK;
}

}  // namespace pvsc
