// Instantiations of the TMA-staged sweep (sweep_tma.cuh) for the Weyl-semimetal
// cells at R = 4, 8, 16 on 8 warps: the large tile, and the half tile with
// rings one plane deeper (more units for a small cuboid).  This unit's kernels report
// copy-wait timeouts in its own error word.
#include "sweep_tma.cuh"

namespace pvsc {

bool tma_tile_deep(int R, int tile_y);

// tile_y selects the large tile or the half tile with rings one plane deeper
int launch_tma_wide(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  const bool deep = tma_tile_deep(p.R, sh.tile_y);
  switch (p.R) {
    case 4:
      return deep ? launch_tma_r<4, true, 8, PVSC_WSM>(lat, feat, p, sh, st)
                  : launch_tma_r<4, false, 8, PVSC_WSM>(lat, feat, p, sh, st);
    case 8:
      return deep ? launch_tma_r<8, true, 8, PVSC_WSM>(lat, feat, p, sh, st)
                  : launch_tma_r<8, false, 8, PVSC_WSM>(lat, feat, p, sh, st);
    default:
      return deep ? launch_tma_r<16, true, 8, PVSC_WSM>(lat, feat, p, sh, st)
                  : launch_tma_r<16, false, 8, PVSC_WSM>(lat, feat, p, sh, st);
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
