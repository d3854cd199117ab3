// Instantiations of the TMA-staged sweep (sweep_tma.cuh) marching along the
// lattice's x axis (tuning kernel 8): tiles over (y, z) columns, for lattices
// whose z columns are short (the cuboids of the dispersion and
// filter-diagonalisation runs, 6 to 8 planes, where a z-march pays two extra x
// planes per few planes swept).  R = 4, 8, 16, and 32, 64 as slices of 16
// vectors; TI sites on the large tile and the half tile with deeper rings,
// Weyl cells on the large tile; the KPM, series and plain sweeps (the fused
// step with z runs the z-march of kernel 7).  This unit's kernels report
// copy-wait timeouts in its own error word.
#include "sweep_tma.cuh"

namespace pvsc {

bool tma_tile_deep(int R, int tile_y);

template <int R, int SL>
static int launch_xm(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  if (lat->g.model == PVSC_WSM) return launch_tma_r<R, false, 8, PVSC_WSM, SL, true>(lat, feat, p, sh, st);
  if (tma_tile_deep(R * SL, sh.tile_y)) return launch_tma_r<R, true, 8, PVSC_TI, SL, true>(lat, feat, p, sh, st);
  return launch_tma_r<R, false, 8, PVSC_TI, SL, true>(lat, feat, p, sh, st);
}

int launch_tma_xm(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  switch (p.R) {
    case 4: return launch_xm<4, 1>(lat, feat, p, sh, st);
    case 8: return launch_xm<8, 1>(lat, feat, p, sh, st);
    case 16: return launch_xm<16, 1>(lat, feat, p, sh, st);
    case 32: return launch_xm<16, 2>(lat, feat, p, sh, st);
    default: return launch_xm<16, 4>(lat, feat, p, sh, st);
  }
}

bool tma_xm_feature(int feat) { return feat == 0 || feat == F_DOTS || feat == F_ACC; }

int tma_error_xm(int clear, int* flag) {
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
