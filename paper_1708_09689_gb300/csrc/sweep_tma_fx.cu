// Instantiations of the TMA-staged sweep (sweep_tma.cuh) for the fixed-point
// (PVSC_Q64) TI KPM sweep, tuning kernel 7 of that precision.  A fixed-point
// site of R vectors (16 bytes per value) has the byte layout of a complex64
// site of 2R vectors, so the complex64 tiles, rings and swizzle of layout 2R
// serve it unchanged; each thread updates one vector of one site.  This unit's
// kernels report copy-wait timeouts in its own error word.
#include "sweep_tma.cuh"

namespace pvsc {

bool tma_tile_deep(int R, int tile_y);

// work units on the smaller (deep-ring) tiles, the most there are; R = 16 and 32
// (layouts of 32 and 64) run as 2 and 4 slices of 8 vectors on the tiles of layout 16
template <int R2>
static int64_t tma_fx_tiles(const Geometry& g) {
  constexpr int RT = R2 > 16 ? 16 : R2;
  using L = TmaLayout<RT, true, 8, 4>;
  return ((g.L[0] + L::TX - 1) / L::TX) * ((g.L[1] + L::TY - 1) / L::TY);
}

bool tma_fx_possible(const pvsc_lattice* lat, int R) {
  const Geometry& g = lat->g;
  if (!(g.model == PVSC_TI && (R == 1 || R == 2 || R == 4 || R == 8 || R == 16 || R == 32) && g.L[0] < 65536 &&
        g.L[1] < 65536 && g.L[2] < 65536))
    return false;
  const int64_t ntiles = R == 1    ? tma_fx_tiles<2>(g)
                         : R == 2  ? tma_fx_tiles<4>(g)
                         : R == 4  ? tma_fx_tiles<8>(g)
                         : R == 8  ? tma_fx_tiles<16>(g)
                         : R == 16 ? tma_fx_tiles<32>(g)
                                   : tma_fx_tiles<64>(g);
  const int64_t SL = R > 8 ? R / 8 : 1;  // slices of 8 vectors for R = 16, 32
  return ntiles <= (int64_t)kTmaUnitsPerSm * (lat->sm_count / SL);
}

// As the complex64 TI sweep: tile_y selects the large tile (two planes of
// copies in flight) or half of it (three); threads = 512 runs the large
// tile with one item per thread.  The block of R vectors uses the layout of 2R
// (R = 16 and 32: slices of 8 vectors, each in the layout of 16).
int launch_sweep_tma_fx(const pvsc_lattice* lat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  if (!tma_fx_possible(lat, p.R))
    return set_error(PVSC_ERR_UNSUPPORTED, "the TMA-staged fixed-point sweep needs a TI lattice and R = 1 .. 32");
  const bool deep = tma_tile_deep(2 * p.R, sh.tile_y);
  const bool wide = !deep && sh.threads == 512;
  constexpr int F = kModelTIFx;
  switch (p.R) {
    case 1:  // the 64-byte sites of layout 2
      return deep ? launch_tma_r<2, true, 8, F>(lat, F_DOTS, p, sh, st)
                  : (wide ? launch_tma_r<2, false, 16, F>(lat, F_DOTS, p, sh, st)
                          : launch_tma_r<2, false, 8, F>(lat, F_DOTS, p, sh, st));
    case 2:
      return deep ? launch_tma_r<4, true, 8, F>(lat, F_DOTS, p, sh, st)
                  : (wide ? launch_tma_r<4, false, 16, F>(lat, F_DOTS, p, sh, st)
                          : launch_tma_r<4, false, 8, F>(lat, F_DOTS, p, sh, st));
    case 4:
      return deep ? launch_tma_r<8, true, 8, F>(lat, F_DOTS, p, sh, st)
                  : (wide ? launch_tma_r<8, false, 16, F>(lat, F_DOTS, p, sh, st)
                          : launch_tma_r<8, false, 8, F>(lat, F_DOTS, p, sh, st));
    case 8:
      return deep ? launch_tma_r<16, true, 8, F>(lat, F_DOTS, p, sh, st)
                  : (wide ? launch_tma_r<16, false, 16, F>(lat, F_DOTS, p, sh, st)
                          : launch_tma_r<16, false, 8, F>(lat, F_DOTS, p, sh, st));
    case 16:  // two slices of 8 vectors
      return deep ? launch_tma_r<16, true, 8, F, 2>(lat, F_DOTS, p, sh, st)
                  : (wide ? launch_tma_r<16, false, 16, F, 2>(lat, F_DOTS, p, sh, st)
                          : launch_tma_r<16, false, 8, F, 2>(lat, F_DOTS, p, sh, st));
    default:  // four slices of 8 vectors
      return deep ? launch_tma_r<16, true, 8, F, 4>(lat, F_DOTS, p, sh, st)
                  : (wide ? launch_tma_r<16, false, 16, F, 4>(lat, F_DOTS, p, sh, st)
                          : launch_tma_r<16, false, 8, F, 4>(lat, F_DOTS, p, sh, st));
  }
}

int tma_error_fx(int clear, int* flag) {
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
