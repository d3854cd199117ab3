// complex64 storage, fp32 stencil arithmetic, fp64 reductions and
// accumulators: kernel instantiations and launchers (register-marching,
// flat, cp.async-prefetching and shared-memory staged TI sweeps; graphene
// sweep).
#include "internal.h"
#include "sweep.cuh"
#include "sweep_bulk.cuh"

namespace pvsc {

template <int MODEL, int VPT, int FEAT>
static void* kernel_c64() {
  if constexpr (MODEL == 1) return reinterpret_cast<void*>(&ti_sweep<float, VPT, FEAT>);
  else if constexpr (MODEL == kModelTIFlat) return reinterpret_cast<void*>(&ti_sweep_flat<float, VPT, FEAT>);
  else if constexpr (MODEL == kModelTIAsync)
    return reinterpret_cast<void*>(&ti_sweep<float, VPT, FEAT, kAsyncDepth, 6>);
  else if constexpr (MODEL == kModelTIAsyncDeep)
    return reinterpret_cast<void*>(&ti_sweep<float, VPT, FEAT, kAsyncDeepDepth, 2>);
  else if constexpr (MODEL == kModelWSM) return reinterpret_cast<void*>(&wsm_sweep<float, VPT, FEAT>);
  else if constexpr (MODEL == kModelWSMMarch) return reinterpret_cast<void*>(&wsm_march_sweep<float, VPT, FEAT>);
  else if constexpr (MODEL == kModelGrapheneQD) return reinterpret_cast<void*>(&gr_sweep<float, VPT, FEAT, true>);
  else if constexpr (MODEL == kModelTIXMarch) return reinterpret_cast<void*>(&ti_sweep_xmarch<float, VPT, FEAT>);
  else return reinterpret_cast<void*>(&gr_sweep<float, VPT, FEAT>);
}

template <int MODEL, int VPT>
static void* pick_c64(int feat) {
  switch (feat) {
    case 0: return kernel_c64<MODEL, VPT, 0>();
    case F_DOTS: return kernel_c64<MODEL, VPT, F_DOTS>();
    case F_Z: return kernel_c64<MODEL, VPT, F_Z>();
    case F_DOTS | F_Z: return kernel_c64<MODEL, VPT, F_DOTS | F_Z>();
    case F_ACC: return kernel_c64<MODEL, VPT, F_ACC>();
    default: return nullptr;
  }
}

static void* pick(int model, int vpt, int feat) {
  switch (model) {
    case 1: return vpt == 1 ? pick_c64<1, 1>(feat) : pick_c64<1, 2>(feat);
    case kModelTIFlat: return vpt == 1 ? pick_c64<kModelTIFlat, 1>(feat) : pick_c64<kModelTIFlat, 2>(feat);
    case kModelTIAsync: return vpt == 1 ? pick_c64<kModelTIAsync, 1>(feat) : pick_c64<kModelTIAsync, 2>(feat);
    case kModelTIAsyncDeep:
      return vpt == 1 ? pick_c64<kModelTIAsyncDeep, 1>(feat) : pick_c64<kModelTIAsyncDeep, 2>(feat);
    case kModelWSM: return vpt == 1 ? pick_c64<kModelWSM, 1>(feat) : pick_c64<kModelWSM, 2>(feat);
    case kModelWSMMarch:
      return vpt == 1 ? pick_c64<kModelWSMMarch, 1>(feat) : pick_c64<kModelWSMMarch, 2>(feat);
    case kModelGrapheneQD:
      return vpt == 1 ? pick_c64<kModelGrapheneQD, 1>(feat) : pick_c64<kModelGrapheneQD, 2>(feat);
    case kModelTIXMarch:
      return vpt == 1 ? pick_c64<kModelTIXMarch, 1>(feat) : pick_c64<kModelTIXMarch, 2>(feat);
    default: return vpt == 1 ? pick_c64<2, 1>(feat) : pick_c64<2, 2>(feat);
  }
}

int launch_sweep_c64(int model, int vpt, int feat, int grid, int threads, const Sweep& p,
                     cudaStream_t st) {
  void* fn = pick(model, vpt, feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no complex64 sweep for feature set %d", feat);
  const size_t smem = async_ring_bytes(model, threads);
  if (smem)
    if (int rc = allow_max_smem(fn)) return rc;
  void* args[] = {const_cast<Sweep*>(&p)};
  PVSC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st));
  return PVSC_OK;
}

int occupancy_c64(int model, int vpt, int feat, int threads, int* blocks) {
  void* fn = pick(model, vpt, feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no complex64 sweep for feature set %d", feat);
  const size_t smem = async_ring_bytes(model, threads);
  if (smem)
    if (int rc = allow_max_smem(fn)) return rc;
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem));
  return PVSC_OK;
}

// ---------------------------------------------------------------- shared-memory staged TI sweep
static void* pick_bulk_c64(int feat) {
  switch (feat) {
    case 0: return reinterpret_cast<void*>(&ti_sweep_bulk<float, 0>);
    case F_DOTS: return reinterpret_cast<void*>(&ti_sweep_bulk<float, F_DOTS>);
    case F_Z: return reinterpret_cast<void*>(&ti_sweep_bulk<float, F_Z>);
    case F_DOTS | F_Z: return reinterpret_cast<void*>(&ti_sweep_bulk<float, F_DOTS | F_Z>);
    case F_ACC: return reinterpret_cast<void*>(&ti_sweep_bulk<float, F_ACC>);
    default: return nullptr;
  }
}

int launch_sweep_bulk_c64(int feat, int grid, int threads, size_t smem, const Sweep& p,
                          cudaStream_t st) {
  void* fn = pick_bulk_c64(feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no staged complex64 sweep for feature set %d", feat);
  if (int rc = allow_max_smem(fn)) return rc;
  void* args[] = {const_cast<Sweep*>(&p)};
  PVSC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st));
  return PVSC_OK;
}

int occupancy_bulk_c64(int feat, int threads, size_t smem, int* blocks) {
  void* fn = pick_bulk_c64(feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no staged complex64 sweep for feature set %d", feat);
  if (int rc = allow_max_smem(fn)) return rc;
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem));
  return PVSC_OK;
}

int bulk_error_c64(int clear, int* flag) {
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
