// TMA-staged plane-tile sweep (tuning kernel 7): host-side eligibility, tile
// choices and dispatch.  The kernels are instantiated in sweep_tma_ti.cu (TI,
// R = 4, 8, 16, all launch variants), sweep_tma_narrow.cu (R = 1, 2: one thread
// per 32- or 64-byte site), sweep_tma_wide.cu (the Weyl-semimetal
// cells, R = 4 .. 16) and sweep_tma_sliced.cu (R = 32 and 64 as two or four
// slices of 16 vectors on the tiles of R = 16, TI and Weyl cells), compiled in
// parallel; the kernel itself is in sweep_tma.cuh.
#include "sweep_tma.cuh"

namespace pvsc {

int launch_tma_ti(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
int launch_tma_wide(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
int launch_tma_sliced(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
int tma_error_ti(int clear, int* flag);
int tma_error_wide(int clear, int* flag);
int tma_error_sliced(int clear, int* flag);
int launch_tma_xm(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
int launch_tma_narrow(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
int tma_error_narrow(int clear, int* flag);
bool tma_xm_feature(int feat);
int tma_error_xm(int clear, int* flag);

// work units of a sweep on the smaller (deep-ring) tiles, the most there are; R = 32
// and 64 run as 2 and 4 slices of the 16-vector tiles
template <int R>
static int64_t tma_tiles(const Geometry& g) {
  constexpr int RT = R > 16 ? 16 : R;
  using L = TmaLayout<RT, true, 8>;
  const int64_t Lx = g.model == PVSC_WSM ? g.L[0] / 2 : g.L[0];
  return ((Lx + L::TX - 1) / L::TX) * ((g.L[1] + L::TY - 1) / L::TY);
}

// whole-column units of a slice that the blocks of that slice can hold in their tables
static bool tma_units_fit(const pvsc_lattice* lat, int64_t tiles_per_slice, int R) {
  const int64_t SL = R > 16 ? R / 16 : 1;
  return tiles_per_slice <= (int64_t)kTmaUnitsPerSm * (lat->sm_count / SL);
}

// The kernel's unit table holds the (x0, y0, z0, planes) of a block's units in
// 16-bit fields, at most kTmaMaxUnits of them (one z-chunk per column at least).
bool tma_sweep_possible(const pvsc_lattice* lat, int R, int prec) {
  const Geometry& g = lat->g;
  if (!((g.model == PVSC_TI || g.model == PVSC_WSM) && prec == PVSC_C64 && valid_R(R) && g.L[0] % 4 == 0 &&
        g.L[0] < 65536 && g.L[1] < 65536 && g.L[2] < 65536))
    return false;
  const int64_t ntiles = R == 1    ? tma_tiles<1>(g)
                         : R == 2  ? tma_tiles<2>(g)
                         : R == 4  ? tma_tiles<4>(g)
                         : R == 8  ? tma_tiles<8>(g)
                         : R == 16 ? tma_tiles<16>(g)
                         : R == 32 ? tma_tiles<32>(g)
                                   : tma_tiles<64>(g);
  return tma_units_fit(lat, ntiles, R);
}


static void tma_tiles_of(int R, int* tx_large, int* ty_large, int* tx_deep, int* ty_deep) {
  switch (R) {
    case 1: *tx_large = TmaLayout<1, false, 8>::TX; *ty_large = TmaLayout<1, false, 8>::TY;
            *tx_deep = TmaLayout<1, true, 8>::TX; *ty_deep = TmaLayout<1, true, 8>::TY; break;
    case 2: *tx_large = TmaLayout<2, false, 8>::TX; *ty_large = TmaLayout<2, false, 8>::TY;
            *tx_deep = TmaLayout<2, true, 8>::TX; *ty_deep = TmaLayout<2, true, 8>::TY; break;
    case 4: *tx_large = TmaLayout<4, false, 8>::TX; *ty_large = TmaLayout<4, false, 8>::TY;
            *tx_deep = TmaLayout<4, true, 8>::TX; *ty_deep = TmaLayout<4, true, 8>::TY; break;
    case 8: *tx_large = TmaLayout<8, false, 8>::TX; *ty_large = TmaLayout<8, false, 8>::TY;
            *tx_deep = TmaLayout<8, true, 8>::TX; *ty_deep = TmaLayout<8, true, 8>::TY; break;
    case 16: *tx_large = TmaLayout<16, false, 8>::TX; *ty_large = TmaLayout<16, false, 8>::TY;
             *tx_deep = TmaLayout<16, true, 8>::TX; *ty_deep = TmaLayout<16, true, 8>::TY; break;
    default:  // R = 32, 64: slices of 16 vectors on the tiles of R = 16
             *tx_large = TmaLayout<16, false, 8>::TX; *ty_large = TmaLayout<16, false, 8>::TY;
             *tx_deep = TmaLayout<16, true, 8>::TX; *ty_deep = TmaLayout<16, true, 8>::TY; break;
  }
}

bool tma_tile_deep(int R, int tile_y) {
  int a, b, c, d;
  tma_tiles_of(R, &a, &b, &c, &d);
  return tile_y == d;  // 0 and the large tile take the large tile
}

bool tma_tile_valid(int R, int tile_x, int tile_y) {
  if (tile_x == 0 && tile_y == 0) return true;
  int a, b, c, d;
  tma_tiles_of(R, &a, &b, &c, &d);
  return (tile_x == a && tile_y == b) || (tile_x == c && tile_y == d);
}

int launch_sweep_tma(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  if (!tma_sweep_possible(lat, p.R, PVSC_C64))
    return set_error(PVSC_ERR_UNSUPPORTED, "the TMA-staged sweep needs a complex64 TI or Weyl lattice "
                     "and Lx a multiple of 4");
  if (p.R >= 32) return launch_tma_sliced(lat, feat, p, sh, st);
  if (p.R <= 2) return launch_tma_narrow(lat, feat, p, sh, st);
  if (lat->g.model == PVSC_WSM) return launch_tma_wide(lat, feat, p, sh, st);
  return launch_tma_ti(lat, feat, p, sh, st);
}

// Marching along x: tiles over the (y, z) columns, the same unit-table limits.
bool tma_xm_possible(const pvsc_lattice* lat, int R, int prec) {
  const Geometry& g = lat->g;
  if (R < 4 || !tma_sweep_possible(lat, R, prec)) return false;  // TI sites or Weyl cells, complex64, R >= 4
  constexpr int TXd = TmaLayout<16, true, 8>::TX, TYd = TmaLayout<16, true, 8>::TY;  // the smallest tiles
  const int64_t ntiles = ((g.L[1] + TXd - 1) / TXd) * ((g.L[2] + TYd - 1) / TYd);
  return tma_units_fit(lat, ntiles, R);
}

int launch_sweep_tma_xm(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  if (!tma_xm_possible(lat, p.R, PVSC_C64))
    return set_error(PVSC_ERR_UNSUPPORTED, "kernel 8 (TMA-staged tiles marching along x) needs a complex64 TI "
                     "or Weyl lattice, R >= 4 and Lx a multiple of 4");
  if (!tma_xm_feature(feat)) return launch_sweep_tma(lat, feat, p, sh, st);  // the fused step with z
  return launch_tma_xm(lat, feat, p, sh, st);
}

int tma_error(int clear, int* flag) {
  int a = 0, b = 0, c = 0, d = 0, e = 0, f = 0;
  if (int rc = tma_error_narrow(clear, &f)) return rc;
  if (int rc = tma_error_ti(clear, &a)) return rc;
  if (int rc = tma_error_wide(clear, &b)) return rc;
  if (int rc = tma_error_fx(clear, &c)) return rc;
  if (int rc = tma_error_sliced(clear, &d)) return rc;
  if (int rc = tma_error_xm(clear, &e)) return rc;
  *flag = (a || b || c || d || e || f) ? 1 : 0;
  return PVSC_OK;
}

}  // namespace pvsc
