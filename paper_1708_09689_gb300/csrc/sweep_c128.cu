// complex128 storage, fp64 arithmetic: kernel instantiations and launchers.
#include "internal.h"
#include "sweep.cuh"

namespace pvsc {

template <int MODEL, int FEAT>
static void* kernel_c128() {
  if constexpr (MODEL == 1) return reinterpret_cast<void*>(&ti_sweep<double, 1, FEAT>);
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
  return model == 1 ? pick_c128<1>(feat) : pick_c128<2>(feat);
}

int launch_sweep_c128(int model, int feat, int grid, int threads, const Sweep& p,
                      cudaStream_t st) {
  void* fn = pick(model, feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no complex128 sweep for feature set %d", feat);
  void* args[] = {const_cast<Sweep*>(&p)};
  PVSC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, st));
  return PVSC_OK;
}

int occupancy_c128(int model, int feat, int threads, int* blocks) {
  void* fn = pick(model, feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no complex128 sweep for feature set %d", feat);
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, 0));
  return PVSC_OK;
}

}  // namespace pvsc
