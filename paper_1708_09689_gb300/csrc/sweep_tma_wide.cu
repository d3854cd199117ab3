// Instantiations of the TMA-staged sweep (sweep_tma.cuh) for the Weyl-semimetal
// cells at R = 4, 8, 16 (the large tile on 8 warps).  This unit's kernels report
// copy-wait timeouts in its own error word.
#include "sweep_tma.cuh"

namespace pvsc {

int launch_tma_wide(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  switch (p.R) {
    case 4: return launch_tma_r<4, false, 8, PVSC_WSM>(lat, feat, p, sh, st);
    case 8: return launch_tma_r<8, false, 8, PVSC_WSM>(lat, feat, p, sh, st);
    default: return launch_tma_r<16, false, 8, PVSC_WSM>(lat, feat, p, sh, st);
  }
}

int tma_error_wide(int clear, int* flag) {
  int h = 0;
  PVSC_CUDA_TRY(cudaMemcpyFromSymbol(&h, g_tma_sweep_error, sizeof(int)));
  if (clear) {
    const int z = 0;
    PVSC_CUDA_TRY(cudaMemcpyToSymbol(g_tma_sweep_error, &z, sizeof(int)));
  }
  *flag = h;
  return PVSC_OK;
}

}  // namespace pvsc
