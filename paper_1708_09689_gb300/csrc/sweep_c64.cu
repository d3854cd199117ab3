// complex64 storage, fp32 stencil arithmetic, fp64 reductions and
// accumulators: kernel instantiations and launchers.
#include "internal.h"
#include "sweep.cuh"

namespace pvsc {

template <int MODEL, int VPT, int FEAT>
static void* kernel_c64() {
  if constexpr (MODEL == 1) return reinterpret_cast<void*>(&ti_sweep<float, VPT, FEAT>);
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
  if (model == 1) return vpt == 1 ? pick_c64<1, 1>(feat) : pick_c64<1, 2>(feat);
  return vpt == 1 ? pick_c64<2, 1>(feat) : pick_c64<2, 2>(feat);
}

int launch_sweep_c64(int model, int vpt, int feat, int grid, int threads, const Sweep& p,
                     cudaStream_t st) {
  void* fn = pick(model, vpt, feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no complex64 sweep for feature set %d", feat);
  void* args[] = {const_cast<Sweep*>(&p)};
  PVSC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, st));
  return PVSC_OK;
}

int occupancy_c64(int model, int vpt, int feat, int threads, int* blocks) {
  void* fn = pick(model, vpt, feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no complex64 sweep for feature set %d", feat);
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, 0));
  return PVSC_OK;
}

}  // namespace pvsc
