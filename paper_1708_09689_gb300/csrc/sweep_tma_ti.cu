// Instantiations of the TMA-staged sweep (sweep_tma.cuh) for TI lattices with
// R = 4, 8, 16 in every launch variant: the large tile on 8 warps (two items
// per thread) or 16 warps (one item), and the half tile with deeper rings.
// This unit's kernels report copy-wait timeouts in its own error word.
#include "sweep_tma.cuh"

namespace pvsc {

bool tma_tile_deep(int R, int tile_y);

// tile_y selects the tile (and ring depth) of this R: the larger tile with two
// planes in flight, or half of it with three (0: the default); threads = 512
// the large tile with one item per thread (16 warps)
int launch_tma_ti(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  const bool deep = tma_tile_deep(p.R, sh.tile_y);
  const bool wide = !deep && sh.threads == 512;
  switch (p.R) {
    case 4:
      return deep ? launch_tma_r<4, true, 8>(lat, feat, p, sh, st)
                  : (wide ? launch_tma_r<4, false, 16>(lat, feat, p, sh, st)
                          : launch_tma_r<4, false, 8>(lat, feat, p, sh, st));
    case 8:
      return deep ? launch_tma_r<8, true, 8>(lat, feat, p, sh, st)
                  : (wide ? launch_tma_r<8, false, 16>(lat, feat, p, sh, st)
                          : launch_tma_r<8, false, 8>(lat, feat, p, sh, st));
    default:
      return deep ? launch_tma_r<16, true, 8>(lat, feat, p, sh, st)
                  : (wide ? launch_tma_r<16, false, 16>(lat, feat, p, sh, st)
                          : launch_tma_r<16, false, 8>(lat, feat, p, sh, st));
  }
}

int tma_error_ti(int clear, int* flag) {
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
