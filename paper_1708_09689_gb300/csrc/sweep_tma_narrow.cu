// Instantiations of the TMA-staged sweep (sweep_tma.cuh) for narrow blocks:
// R = 1 and 2, whose 32- and 64-byte sites are narrower than the 128-byte row
// of the wider blocks.  A copied row is one whole site under the 32- or 64-byte
// swizzle, one thread owns one site (both vectors at R = 2), and the 8 sites a
// quarter-warp reads are consecutive along x, which that swizzle spreads over
// the 8 bank groups.  TI lattices in every launch variant (the large tile on
// 8 or 16 warps, the half tile with deeper rings), Weyl cells on the large
// and the half tile.  This unit's kernels report copy-wait timeouts in its own error word.
#include "sweep_tma.cuh"

namespace pvsc {

bool tma_tile_deep(int R, int tile_y);

template <int R>
static int launch_narrow(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  if (lat->g.model == PVSC_WSM)
    return tma_tile_deep(R, sh.tile_y) ? launch_tma_r<R, true, 8, PVSC_WSM>(lat, feat, p, sh, st)
                                       : launch_tma_r<R, false, 8, PVSC_WSM>(lat, feat, p, sh, st);
  if (tma_tile_deep(R, sh.tile_y)) return launch_tma_r<R, true, 8>(lat, feat, p, sh, st);
  if (sh.threads == 512) return launch_tma_r<R, false, 16>(lat, feat, p, sh, st);
  return launch_tma_r<R, false, 8>(lat, feat, p, sh, st);
}

int launch_tma_narrow(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  return p.R == 1 ? launch_narrow<1>(lat, feat, p, sh, st) : launch_narrow<2>(lat, feat, p, sh, st);
}

int tma_error_narrow(int clear, int* flag) {
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
