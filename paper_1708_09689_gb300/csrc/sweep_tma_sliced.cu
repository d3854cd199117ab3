// Instantiations of the TMA-staged sweep (sweep_tma.cuh) for blocks of R = 32
// and 64 vectors, swept as 2 or 4 slices of 16 vectors on the tiles of R = 16
// (8 x 8 sites, or the 8 x 4 half tile with deeper rings): the 4 x 4 and 4 x 2
// tiles that fit shared memory with whole 1 KB and 2 KB sites copy halo strips as
// large as the tile.  TI lattices in every launch variant, Weyl-semimetal cells
// on the large and the half tile.  This unit's kernels report copy-wait timeouts in its own
// error word.
#include "sweep_tma.cuh"

namespace pvsc {

bool tma_tile_deep(int R, int tile_y);

template <int SL>
static int launch_sliced(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  if (lat->g.model == PVSC_WSM)
    return tma_tile_deep(p.R, sh.tile_y) ? launch_tma_r<16, true, 8, PVSC_WSM, SL>(lat, feat, p, sh, st)
                                         : launch_tma_r<16, false, 8, PVSC_WSM, SL>(lat, feat, p, sh, st);
  if (tma_tile_deep(p.R, sh.tile_y)) return launch_tma_r<16, true, 8, PVSC_TI, SL>(lat, feat, p, sh, st);
  if (sh.threads == 512) return launch_tma_r<16, false, 16, PVSC_TI, SL>(lat, feat, p, sh, st);
  return launch_tma_r<16, false, 8, PVSC_TI, SL>(lat, feat, p, sh, st);
}

int launch_tma_sliced(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  return p.R == 32 ? launch_sliced<2>(lat, feat, p, sh, st) : launch_sliced<4>(lat, feat, p, sh, st);
}

int tma_error_sliced(int clear, int* flag) {
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
