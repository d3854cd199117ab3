// Host drivers of the C ABI: sweep launch shapes, the fused Chebyshev step,
// KPM moments, Chebyshev series / filter / time propagation, the adjoint step
// and the CUDA-graph cache that replays captured recurrence loops.
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

#include "internal.h"
#include "sweep.cuh"

namespace pvsc {

using cd = std::complex<double>;

// ---------------------------------------------------------------- launch shapes
static LaunchShape shape_for(const pvsc_lattice* lat, int R, int prec) {
  LaunchShape sh;
  auto it = lat->tuning.find({R, prec});
  if (it != lat->tuning.end()) {
    sh.threads = it->second.threads;
    sh.blocks_per_sm = it->second.blocks_per_sm;
    sh.zslab = it->second.zslab;
    sh.vpt = it->second.vpt;
    sh.tile_x = it->second.tile_x;
    sh.tile_y = it->second.tile_y;
    sh.kernel = it->second.kernel;
  }
  return sh;
}

// 4 halo plane slots + 4 y_in tile slots + 2 potential slots + 4 mbarriers
size_t bulk_smem_bytes(int TX, int TY, int R, int prec) {
  const size_t SB = (size_t)4 * R * (prec == PVSC_C128 ? 16 : 8);
  return 4 * (size_t)(TX + 2) * (TY + 2) * SB + 4 * (size_t)TX * TY * SB +
         2 * (size_t)TX * TY * sizeof(double) + 64;
}

int launch_sweep_bulk(int prec, int feat, int grid, int threads, size_t smem, const Sweep& p,
                      cudaStream_t st) {
  return prec == PVSC_C128 ? launch_sweep_bulk_c128(feat, grid, threads, smem, p, st)
                           : launch_sweep_bulk_c64(feat, grid, threads, smem, p, st);
}

int occupancy_bulk(int prec, int feat, int threads, size_t smem, int* blocks) {
  return prec == PVSC_C128 ? occupancy_bulk_c128(feat, threads, smem, blocks)
                           : occupancy_bulk_c64(feat, threads, smem, blocks);
}

int bulk_sweep_error(int prec, int clear, int* flag) {
  return prec == PVSC_C128 ? bulk_error_c128(clear, flag) : bulk_error_c64(clear, flag);
}

// The shared-memory staged TI sweep: tiles of TX x TY columns, z-slabs, one
// vector per thread.
static int launch_sweep_staged(const pvsc_lattice* lat, int prec, int feat, Sweep& p,
                               const LaunchShape& sh, cudaStream_t st) {
  int threads = sh.threads;
  if (threads < 32 || threads > kMaxThreads || threads % 32 != 0 || threads % p.R != 0) threads = 256;
  if (sh.tile_x * sh.tile_y > 2 * threads)
    return set_error(PVSC_ERR_ARG, "staged tile %dx%d exceeds two sites per thread (%d threads)",
                     sh.tile_x, sh.tile_y, threads);
  p.C = p.R;
  p.tile_x = sh.tile_x;
  p.tile_y = sh.tile_y;
  const size_t smem = bulk_smem_bytes(sh.tile_x, sh.tile_y, p.R, prec);
  int occ = 0;
  if (int rc = occupancy_bulk(prec, feat, threads, smem, &occ)) return rc;
  if (occ < 1)
    return set_error(PVSC_ERR_ARG, "staged sweep tile %dx%d needs %zu bytes of shared memory: too large",
                     sh.tile_x, sh.tile_y, smem);
  int bps = sh.blocks_per_sm;
  if (bps <= 0 || bps > occ) bps = occ;
  if (bps > kMaxGridPerSM) bps = kMaxGridPerSM;
  const int64_t grid_max = (int64_t)lat->sm_count * bps;
  const int64_t Lx = lat->g.L[0], Ly = lat->g.L[1], Lz = lat->g.L[2];
  const int64_t ntiles = ((Lx + sh.tile_x - 1) / sh.tile_x) * ((Ly + sh.tile_y - 1) / sh.tile_y);
  int64_t zs = sh.zslab;
  if (zs <= 0) {
    int64_t nz = (6 * grid_max + ntiles - 1) / ntiles;
    if (nz < 1) nz = 1;
    if (nz > Lz) nz = Lz;
    zs = (Lz + nz - 1) / nz;
  }
  if (zs > Lz) zs = Lz;
  p.zslab = (int)zs;
  const int64_t units = ntiles * ((Lz + zs - 1) / zs);
  const int grid = (int)(units < grid_max ? units : grid_max);
  return launch_sweep_bulk(prec, feat, grid, threads, smem, p, st);
}

void sweep_init(Sweep& p, const pvsc_lattice* lat, int R, int prec) {
  std::memset(&p, 0, sizeof(Sweep));
  p.g = lat->g;
  p.qds = lat->qds;
  p.R = R;
  p.C = R / vpt_for(R, prec);
  for (int r = 0; r < R; ++r) p.coef[0][r] = 1.0;
  p.cx_re = 0; p.ph_re = 1.0;
}

static int coef_kind(double re, double im) {
  return (im == 0.0 ? 1 : 0) | (re == 0.0 ? 2 : 0);  // 1 real, 2 imaginary, 3 zero, 0 general
}

int launch_sweep(const pvsc_lattice* lat, int prec, int feat, Sweep& p, cudaStream_t st) {
  return launch_sweep_shape(lat, prec, feat, p, shape_for(lat, p.R, prec), st);
}

// As launch_sweep with the launch shape given instead of the lattice's tuning entry.
int launch_sweep_shape(const pvsc_lattice* lat, int prec, int feat, Sweep& p, LaunchShape sh, cudaStream_t st) {
  if ((feat & F_ACC) && (p.acc_mode & ACC_YIN) &&
      (!p.yin || !(p.acc_mode & ACC_X) || (p.acc_mode & (ACC_INIT | ACC_XSRC))))
    return set_error(PVSC_ERR_ARG, "an accumulating sweep with the y_in term needs y_in and the x term, "
                                   "and no INIT or XSRC");
  // an absent x or y_in term has the kind of a zero weight (3)
  p.acc_kind = ((p.acc_mode & ACC_X) ? coef_kind(p.cx_re, p.cx_im) : 3) | (coef_kind(p.cy_re, p.cy_im) << 2) |
               (((p.acc_mode & ACC_YIN) ? coef_kind(p.cz_re, p.cz_im) : 3) << 4);
  const double cv[3][2] = {{p.cx_re, p.cx_im}, {p.cy_re, p.cy_im}, {p.cz_re, p.cz_im}};
  for (int t = 0; t < 3; ++t)
    for (int q = 0; q < 2; ++q) {
      p.fc[t][q][0] = (float)cv[t][q];
      p.fc[t][q][1] = (float)(cv[t][q] - (double)p.fc[t][q][0]);
    }
  if (sh.kernel == kKernelKpm2) sh = LaunchShape{};  // a KPM-only choice: single sweeps take the default
  if (lat->g.zhalo) {  // a slab with halo planes: the z-march over its inner planes
    const int zs = sh.zslab;
    sh = LaunchShape{};
    sh.zslab = zs;
  }
  if (sh.kernel == kKernelTma || sh.kernel == kKernelTmaX) {
    p.tile_x = p.tile_y = 0;
    if (sh.kernel == kKernelTmaX && tma_xm_possible(lat, p.R, prec) && !(feat & F_ADJ))
      return launch_sweep_tma_xm(lat, feat, p, sh, st);
    if (tma_sweep_possible(lat, p.R, prec) && !(feat & F_ADJ)) return launch_sweep_tma(lat, feat, p, sh, st);
    sh = LaunchShape{};  // complex128 (or a shape it does not cover) on a lattice tuned for complex64
  }
  p.tile_x = p.tile_y = 0;  // set below by the tiled and staged sweeps only (p may come from another launch)
  const bool tiled = lat->g.model == PVSC_TI && sh.kernel == kKernelTiles;
  if (lat->g.model == PVSC_TI && !tiled && sh.kernel == 0 && sh.tile_x > 0 && sh.tile_y > 0)
    return launch_sweep_staged(lat, prec, feat, p, sh, st);
  const int vpt = vpt_tuned(sh.vpt, p.R, prec);
  p.C = p.R / vpt;
  int threads = sh.threads;
  if (tiled) {  // z-marching sweep over tile_x x tile_y column tiles (checked by pvsc_set_tuning)
    threads = sh.tile_x * sh.tile_y * p.C;
    p.tile_x = sh.tile_x;
    p.tile_y = sh.tile_y;
  }
  if (threads < 32 || threads > kMaxThreads || threads % 32 != 0 || threads % p.C != 0) {
    threads = 256;
    p.tile_x = p.tile_y = 0;
  }
  int occ = 0;
  const bool flat = lat->g.model == PVSC_TI && sh.kernel == 1;
  // the prefetch ring moves 16-byte granules: not for complex64 with one vector of R > 1
  const bool async = lat->g.model == PVSC_TI && (sh.kernel == 2 || sh.kernel == 3) &&
                     !(prec == PVSC_C64 && vpt == 1 && p.R > 1);
  // Weyl semimetal: the flat cell sweep (measured faster on the paper's 256 x 32 x 32
  // cuboid) unless a tuning entry selects the z-marching one (kernel 0)
  const bool wsm = lat->g.model == PVSC_WSM;
  const bool wsm_flat = wsm && (lat->tuning.count({p.R, prec}) == 0 || sh.kernel == 1);
  const bool qd = lat->g.model == PVSC_GRAPHENE && lat->g.v_mode == 3;
  const bool xmarch = lat->g.model == PVSC_TI && sh.kernel == kKernelXMarch;
  const int model = xmarch ? kModelTIXMarch
                    : flat ? kModelTIFlat
                    : async ? (sh.kernel == 2 ? kModelTIAsync : kModelTIAsyncDeep)
                    : wsm ? (wsm_flat ? kModelWSM : kModelWSMMarch)
                    : qd ? kModelGrapheneQD
                            : lat->g.model;
  int rc = prec == PVSC_C128 ? occupancy_c128(model, feat, threads, &occ)
                             : occupancy_c64(model, vpt, feat, threads, &occ);
  if (rc) return rc;
  int bps = sh.blocks_per_sm;
  if (bps <= 0 || bps > occ) bps = occ;
  if (bps < 1) bps = 1;
  if (bps > kMaxGridPerSM) bps = kMaxGridPerSM;
  const int64_t grid_max = (int64_t)lat->sm_count * bps;
  int64_t units;
  if (flat) {
    units = (lat->g.n_sites * p.C + threads - 1) / threads;
  } else if (xmarch) {
    // lines (y, z) marched along x; x-segments of p.zslab sites
    const int64_t Lx = lat->g.L[0];
    const int64_t nbx = (lat->g.L[1] * lat->g.L[2] * p.C + threads - 1) / threads;
    int64_t xs = sh.zslab;
    if (xs <= 0) {
      int64_t nx = (6 * grid_max + nbx - 1) / nbx;
      if (nx < 1) nx = 1;
      if (nx > Lx) nx = Lx;
      xs = (Lx + nx - 1) / nx;
    }
    if (xs > Lx) xs = Lx;
    p.zslab = (int)xs;
    units = nbx * ((Lx + xs - 1) / xs);
  } else if (lat->g.model == PVSC_TI || (wsm && !wsm_flat)) {
    // z-marching columns: TI sites, or Weyl cells (two sites along x); a
    // lattice with halo planes updates its inner planes only
    const int64_t plane = (wsm ? lat->g.L[0] / 2 : lat->g.L[0]) * lat->g.L[1];
    const int64_t Lz = lat->g.L[2] - (lat->g.zhalo & 1) - (lat->g.zhalo >> 1);
    const int64_t nbx = p.tile_x > 0 ? ((lat->g.L[0] + p.tile_x - 1) / p.tile_x) *
                                           ((lat->g.L[1] + p.tile_y - 1) / p.tile_y)
                                     : (plane * p.C + threads - 1) / threads;
    int64_t zs = sh.zslab;
    if (zs <= 0) {
      int64_t nz = (6 * grid_max + nbx - 1) / nbx;
      if (nz < 1) nz = 1;
      if (nz > Lz) nz = Lz;
      zs = (Lz + nz - 1) / nz;
    }
    if (zs > Lz) zs = Lz;
    p.zslab = (int)zs;
    units = nbx * ((Lz + zs - 1) / zs);
  } else {
    // graphene: 4-site cells; Weyl semimetal: cells of two sites
    const int64_t ncell = lat->g.model == PVSC_WSM ? lat->g.n_sites / 2 : lat->g.L[0] * lat->g.L[1];
    units = (ncell * p.C + threads - 1) / threads;
  }
  const int grid = (int)(units < grid_max ? units : grid_max);
  return prec == PVSC_C128 ? launch_sweep_c128(model, feat, grid, threads, p, st)
                           : launch_sweep_c64(model, vpt, feat, grid, threads, p, st);
}

static uint64_t bits(double d) {
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
}
static uint64_t bits(const void* p) { return (uint64_t)reinterpret_cast<uintptr_t>(p); }

// ---------------------------------------------------------------- argument checks
static int check_common(const pvsc_lattice* lat, int R, int prec) {
  if (int rc = check_lattice(lat)) return rc;
  if (!valid_R(R)) return set_error(PVSC_ERR_ARG, "R = %d: must be 1, 2, 4, 8, 16, 32 or 64", R);
  if (prec == PVSC_Q64) return set_error(PVSC_ERR_ARG, "PVSC_Q64 is a precision of pvsc_kpm_moments only");
  if (prec != PVSC_C128 && prec != PVSC_C64) return set_error(PVSC_ERR_ARG, "unknown precision %d", prec);
  return PVSC_OK;
}

static int check_scaling(double a, double b) {
  if (!(std::isfinite(a) && a > 0.0) || !std::isfinite(b))
    return set_error(PVSC_ERR_ARG, "scaling needs a > 0 and finite b (a = %g, b = %g)", a, b);
  return PVSC_OK;
}

static int check_work(void* work, size_t have, size_t need) {
  if (need == 0) return PVSC_OK;
  if (int rc = check_ptr(work, "work")) return rc;
  if (have < need) return set_error(PVSC_ERR_ARG, "work buffer too small: %zu < %zu bytes", have, need);
  return PVSC_OK;
}

static char* wptr(void* work, size_t off) { return static_cast<char*>(work) + off; }

// ---------------------------------------------------------------- Bessel coefficients
// J_0..J_n(x) by Miller's backward recurrence J_{k-1} = (2k/x) J_k - J_{k+1},
// started far above max(n, x) and normalised with J_0 + 2 sum_k J_2k = 1
// (Abramowitz & Stegun 9.12, Numerical Recipes 6.5).
static std::vector<double> bessel_miller(double x, int n) {
  std::vector<double> out(n + 1, 0.0);
  if (x == 0.0) {
    out[0] = 1.0;
    return out;
  }
  const double big = std::fmax((double)n, std::fabs(x));
  int start = (int)(big + 40.0 + 2.0 * std::sqrt(40.0 * big));
  if (start % 2) ++start;
  std::vector<double> j(start + 2, 0.0);
  j[start] = 1e-300;
  for (int k = start; k >= 1; --k) {
    j[k - 1] = (2.0 * k / x) * j[k] - j[k + 1];
    if (std::fabs(j[k - 1]) > 1e250)
      for (int q = k - 1; q <= start; ++q) j[q] *= 1e-250;
  }
  double norm = j[0];
  for (int k = 2; k <= start; k += 2) norm += 2.0 * j[k];
  for (int k = 0; k <= n; ++k) out[k] = j[k] / norm;
  return out;
}

static int propagation_weights(double adt, double trunc, std::vector<cd>& cw) {
  if (!std::isfinite(adt) || !(trunc > 0.0))
    return set_error(PVSC_ERR_ARG, "need finite a*dt and trunc > 0");
  const int kmax = (int)(2.0 * std::fabs(adt) + 60.0);
  std::vector<double> J = bessel_miller(adt, kmax);
  int M = 0;
  for (int k = 0; k <= kmax; ++k)
    if (std::fabs(J[k]) >= trunc) M = k;
  cw.assign(M + 1, cd(0, 0));
  static const cd mi[4] = {cd(1, 0), cd(0, -1), cd(-1, 0), cd(0, 1)};  // (-i)^k
  for (int k = 0; k <= M; ++k) cw[k] = (k == 0 ? 1.0 : 2.0) * mi[k % 4] * J[k];
  return PVSC_OK;
}

// ---------------------------------------------------------------- Chebyshev series
// y = phase * sum_k cw_k T_k(H~) x with the recurrence vectors in `prec`.
struct SeriesLayout {
  size_t hdr, wa, wb, acc, total;
};
static SeriesLayout series_layout(const pvsc_lattice* lat, int R, int prec) {
  SeriesLayout L;
  L.hdr = 0;
  L.wa = kWorkHeader;
  L.wb = L.wa + vec_bytes(lat, R, prec);
  L.acc = L.wb + vec_bytes(lat, R, prec);
  L.total = L.acc + vec_bytes(lat, R, PVSC_C128);
  return L;
}

// The accumulator touches of a series of K terms: terms[j] = the number of
// terms sweep j adds, ending with term j (sweep 1 starts with terms 0 and 1,
// then three terms on every third sweep, the last sweep the one to three
// left; 0 for sweeps that leave the accumulator alone).  K = 1 has no sweep:
// terms[0] = 1 (y = c_0 x directly).
static void series_plan(int K, std::vector<int>& terms) {
  terms.assign(K, 0);
  if (K == 1) {
    terms[0] = 1;
    return;
  }
  terms[1] = 2;
  int done = 1;  // the accumulator holds the terms 0 .. done
  for (int j = 2; j < K; ++j)
    if (j - done == 3 || j == K - 1) {
      terms[j] = j - done;
      done = j;
    }
}

static int run_series(const pvsc_lattice* lat, int R, int prec, const void* x, void* y,
                      const std::vector<cd>& cw, cd phase, double a, double b, void* work,
                      cudaStream_t st) {
  const SeriesLayout L = series_layout(lat, R, prec);
  const int64_t n = lat->g.n_sites * orbitals_of(lat->g.model) * (int64_t)R;
  void* wa = wptr(work, L.wa);
  void* wb = wptr(work, L.wb);
  double2* acc = reinterpret_cast<double2*>(wptr(work, L.acc));
  const int K = (int)cw.size();
  if (K == 1) {  // y = phase c_0 x (elementwise, safe when x and y alias)
    const cd c = phase * cw[0];
    return launch_scale_init(x, static_cast<double2*>(y), c.real(), c.imag(), n, st);
  }
  Sweep p;
  sweep_init(p, lat, R, prec);
  auto set_scal = [&](double alpha, double gamma) {
    for (int r = 0; r < R; ++r) {
      p.coef[0][r] = alpha;
      p.coef[1][r] = b;
      p.coef[2][r] = gamma;
      p.coef[3][r] = 0.0;
    }
  };
  // Sweep j makes w_j from x = w_{j-1} and y_in = w_{j-2}.  The accumulator
  // takes up to three terms per touch: sweep 1 starts it with cw_0 w_0 +
  // cw_1 w_1, sweeps j = 4, 7, 10, ... add cw_{j-2} w_{j-2} + cw_{j-1} w_{j-1}
  // + cw_j w_j, the others leave it alone, and the last sweep adds the one to
  // three terms left and writes phase * acc to y.
  auto set_acc = [&](int j, int mode, int nterms) {
    p.acc = acc;
    p.acc_out = static_cast<double2*>(y);
    p.acc_mode = mode | (nterms >= 2 ? ACC_X : 0) | (nterms == 3 ? ACC_YIN : 0);
    p.cx_re = nterms >= 2 ? cw[j - 1].real() : 0.0;
    p.cx_im = nterms >= 2 ? cw[j - 1].imag() : 0.0;
    p.cz_re = nterms == 3 ? cw[j - 2].real() : 0.0;
    p.cz_im = nterms == 3 ? cw[j - 2].imag() : 0.0;
    p.cy_re = cw[j].real();
    p.cy_im = cw[j].imag();
    p.ph_re = phase.real();
    p.ph_im = phase.imag();
  };
  const void* prev;  // w_{j-2}
  void* cur;         // w_{j-1}
  // j = 1
  set_scal(1.0 / a, 0.0);
  if (prec == PVSC_C128) {
    p.x = x;
    p.yout = wa;
    set_acc(1, ACC_INIT, 2);
    if (int rc = launch_sweep(lat, prec, F_ACC, p, st)) return rc;
    // y may alias x: the final write is a separate pass
    if (K == 2) return launch_scale_init(acc, static_cast<double2*>(y), phase.real(), phase.imag(), n, st);
    prev = x;
    cur = wa;
  } else {
    // w_0 rounded to complex64 for the recurrence; the accumulator takes w_0 exact
    if (int rc = launch_convert_c128_to_c64(x, wb, n, st)) return rc;
    p.x = wb;
    p.src = static_cast<const double2*>(x);
    p.yout = (K == 2) ? nullptr : wa;
    set_acc(1, ACC_INIT | ACC_XSRC | (K == 2 ? ACC_FINAL : 0), 2);
    if (int rc = launch_sweep(lat, prec, F_ACC, p, st)) return rc;
    p.src = nullptr;
    if (K == 2) return PVSC_OK;
    prev = wb;
    cur = wa;
  }
  p.yin = nullptr;
  std::vector<int> plan;
  series_plan(K, plan);
  for (int j = 2; j < K; ++j) {
    const bool last = (j == K - 1);
    void* out = (prev == x) ? wb : const_cast<void*>(prev);
    set_scal(2.0 / a, -1.0);
    p.x = cur;
    p.yin = prev;
    p.yout = last ? nullptr : out;
    int feat = 0;
    if (plan[j] > 0) {
      set_acc(j, ACC_ADD | (last ? ACC_FINAL : 0), plan[j]);
      feat = F_ACC;
    }
    if (int rc = launch_sweep(lat, prec, feat, p, st)) return rc;
    prev = cur;
    cur = out;
  }
  return PVSC_OK;
}

// The two-step KPM sweep exists for complex64 TI lattices with R >= 2 and runs
// when the tuning entry of (R, prec) selects it.
static bool kpm2_possible(const pvsc_lattice* lat, int R, int prec) {
  return lat->g.model == PVSC_TI && prec == PVSC_C64 && R >= 2 && !lat->g.zhalo;
}
static bool kpm2_selected(const pvsc_lattice* lat, int R, int prec) {
  if (!kpm2_possible(lat, R, prec)) return false;
  auto it = lat->tuning.find({R, prec});
  return it != lat->tuning.end() && it->second.kernel == kKernelKpm2;
}

// All kernels of one KPM run (the start block unless given, ceil(M/2) fused
// sweeps with the doubling identities) enqueued on cs; force: a launch shape for
// every sweep instead of the lattice's tuning entry (the batched runs).
int kpm_enqueue(const pvsc_lattice* lat, int R, int prec, const void* r0, uint64_t seed, int M, double a,
                double b, double* mu, void* work, const LaunchShape* force, cudaStream_t cs) {
  const size_t voff = (dots_work_bytes(lat, R) + 255) & ~size_t(255);
  void* wa = wptr(work, voff);
  void* wb = wptr(work, voff + vec_bytes(lat, R, prec));
  const int64_t D = lat->g.n_sites * orbitals_of(lat->g.model);
  const LaunchShape sh = force ? *force : shape_for(lat, R, prec);
  const bool two = !force && kpm2_selected(lat, R, prec);
  PVSC_CUDA_TRY(cudaMemsetAsync(work, 0, kWorkHeader, cs));
  const void* x0 = r0;
  if (!r0) {
    if (int rc = launch_random_phase(wa, prec, D, R, seed, cs)) return rc;
    x0 = wa;
  }
  Sweep p;
  sweep_init(p, lat, R, prec);
  p.counter = reinterpret_cast<unsigned*>(work);
  p.partials = reinterpret_cast<double*>(wptr(work, kWorkHeader));
  p.mu = mu;
  p.M = M;
  p.dot_flags = 3;
  for (int r = 0; r < R; ++r) {
    p.coef[0][r] = 1.0 / a;
    p.coef[1][r] = b;
    p.coef[2][r] = 0.0;
  }
  p.x = x0;
  p.yin = nullptr;
  p.yout = wb;
  p.dot_mode = 1;
  if (int rc = launch_sweep_shape(lat, prec, F_DOTS, p, sh, cs)) return rc;
  const void* prev = x0;
  void* cur = wb;
  const int nsteps = (M + 1) / 2;
  for (int r = 0; r < R; ++r) {
    p.coef[0][r] = 2.0 / a;
    p.coef[2][r] = -1.0;
  }
  int k = 1;
  if (two) {
    // steps k, k+1 per sweep into two buffers distinct from both inputs
    void* pool[4] = {wa, wb, wptr(work, voff + 2 * vec_bytes(lat, R, prec)),
                     wptr(work, voff + 3 * vec_bytes(lat, R, prec))};
    p.dot_mode = 3;
    p.dot_flags = 7;
    for (; k + 1 < nsteps; k += 2) {
      void* o[2];
      int no = 0;
      for (void* q : pool)
        if (q != prev && q != cur && no < 2) o[no++] = q;
      p.x = cur;
      p.yin = prev;
      p.yout = o[0];
      p.yout2 = o[1];
      p.kpm_k = k;
      if (int rc = launch_kpm2_sweep(lat, p, sh, cs)) return rc;
      prev = o[0];
      cur = o[1];
    }
    p.dot_flags = 3;
    p.yout2 = nullptr;
  }
  p.dot_mode = 2;
  for (; k < nsteps; ++k) {
    void* out = (r0 && prev == r0) ? (cur == wa ? wb : wa) : const_cast<void*>(prev);
    p.x = cur;
    p.yin = prev;
    p.yout = out;
    p.kpm_k = k;
    if (int rc = launch_sweep_shape(lat, prec, F_DOTS, p, sh, cs)) return rc;
    prev = cur;
    cur = out;
  }
  return PVSC_OK;
}

}  // namespace pvsc

using namespace pvsc;

extern "C" {

size_t pvsc_work_bytes(const pvsc_lattice* lat, int op, int R, int prec, int M) {
  if (lat && valid_R(R) && prec == PVSC_Q64 && op == PVSC_OP_KPM) return fx_layout(lat, R).total;
  if (!lat || !valid_R(R) || (prec != PVSC_C128 && prec != PVSC_C64)) return 0;
  switch (op) {
    case PVSC_OP_APPLY:
      return kWorkHeader + sizeof(double) * 2 * 2 * (size_t)lat->sm_count;
    case PVSC_OP_CHEB_STEP:
      return dots_work_bytes(lat, R);
    case PVSC_OP_KPM:  // two vectors, four when the tuning in force selects the two-step sweep
      return ((dots_work_bytes(lat, R) + 255) & ~size_t(255)) +
             (kpm2_selected(lat, R, prec) ? 4 : 2) * vec_bytes(lat, R, prec);
    case PVSC_OP_SERIES:
      return series_layout(lat, R, prec).total;
    case PVSC_OP_ADJOINT: {
      const int nvec = (M < 1 ? 1 : M) + 2;
      return kWorkHeader + (size_t)nvec * vec_bytes(lat, R, PVSC_C128);
    }
    default:
      return 0;
  }
}

int pvsc_random_vectors(const pvsc_lattice* lat, int R, int prec, uint64_t seed, void* out,
                        void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (int rc = check_ptr(out, "out")) return rc;
  const int64_t D = lat->g.n_sites * orbitals_of(lat->g.model);
  return launch_random_phase(out, prec, D, R, seed, static_cast<cudaStream_t>(stream));
}

int pvsc_apply_H(const pvsc_lattice* lat, int R, int prec, const void* x, void* y, void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (int rc = check_ptr(x, "x")) return rc;
  if (int rc = check_ptr(y, "y")) return rc;
  if (x == y) return set_error(PVSC_ERR_ARG, "x and y must not overlap");
  Sweep p;
  sweep_init(p, lat, R, prec);
  p.x = x;
  p.yout = y;
  return launch_sweep(lat, prec, 0, p, static_cast<cudaStream_t>(stream));
}

int pvsc_cheb_step(const pvsc_lattice* lat, int R, int prec, const void* x, void* y, void* z,
                   const double* alpha, const double* beta, const double* gamma,
                   const double* delta, int dot_flags, double* dots, void* work,
                   size_t work_bytes, void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (int rc = check_ptr(x, "x")) return rc;
  if (int rc = check_ptr(y, "y")) return rc;
  if (!alpha || !beta) return set_error(PVSC_ERR_ARG, "alpha and beta must not be NULL");
  if (x == y || x == z) return set_error(PVSC_ERR_ARG, "x must not overlap y or z");
  if (z) {
    if (int rc = check_ptr(z, "z")) return rc;
    if (!delta) return set_error(PVSC_ERR_ARG, "z needs delta");
    if (z == y) return set_error(PVSC_ERR_ARG, "z must not overlap y");
  }
  if (dot_flags & ~7) return set_error(PVSC_ERR_ARG, "unknown dot flags 0x%x", dot_flags);
  if (dot_flags && !dots) return set_error(PVSC_ERR_ARG, "dot_flags set but dots is NULL");
  for (int r = 0; r < R; ++r)
    if (!std::isfinite(alpha[r]) || !std::isfinite(beta[r]) || (gamma && !std::isfinite(gamma[r])) ||
        (z && !std::isfinite(delta[r])))
      return set_error(PVSC_ERR_ARG, "coefficients of vector %d are not finite", r);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Sweep p;
  sweep_init(p, lat, R, prec);
  for (int r = 0; r < R; ++r) {
    p.coef[0][r] = alpha[r];
    p.coef[1][r] = beta[r];
    p.coef[2][r] = gamma ? gamma[r] : 0.0;
    p.coef[3][r] = z ? delta[r] : 0.0;
  }
  p.x = x;
  p.yin = gamma ? y : nullptr;
  p.yout = y;
  p.z = z;
  int feat = z ? F_Z : 0;
  if (dot_flags) {
    if (int rc = check_work(work, work_bytes, dots_work_bytes(lat, R))) return rc;
    feat |= F_DOTS;
    p.dot_flags = dot_flags;
    p.dot_mode = 0;
    p.dots = dots;
    p.counter = reinterpret_cast<unsigned*>(work);
    p.partials = reinterpret_cast<double*>(wptr(work, kWorkHeader));
    PVSC_CUDA_TRY(cudaMemsetAsync(work, 0, kWorkHeader, st));
  }
  return launch_sweep(lat, prec, feat, p, st);
}

// KPM with fixed-point vectors (sweep_fx.cu); TI lattices only.
static int kpm_moments_fx(const pvsc_lattice* lat, int R, const void* r0, uint64_t seed, int M,
                          double a, double b, double* mu, void* work, size_t work_bytes,
                          cudaStream_t st) {
  if (lat->g.model != PVSC_TI)
    return set_error(PVSC_ERR_UNSUPPORTED, "PVSC_Q64 moments are implemented for the TI lattice only");
  if (lat->g.has_delta)
    return set_error(PVSC_ERR_UNSUPPORTED, "PVSC_Q64 moments do not include the Delta terms");
  if (lat->g.zhalo) return set_error(PVSC_ERR_UNSUPPORTED, "PVSC_Q64 moments do not take halo lattices");
  const FxLayout L = fx_layout(lat, R);
  if (int rc = check_work(work, work_bytes, L.total)) return rc;
  // The fixed-point range relies on ||T_k(H~)|| <= 1: (a, b) must hold the
  // Gershgorin interval.  It is computed once per potential (one synchronous
  // pass, on the first call after lattice creation or pvsc_set_potential) and
  // kept in the handle; later calls check against it without synchronising.
  {
    pvsc_lattice* ml = const_cast<pvsc_lattice*>(lat);
    if (!lat->gersh_valid) {
      const int grid = 2 * lat->sm_count;
      double* gw = reinterpret_cast<double*>(wptr(work, kWorkHeader));
      if (int rc = launch_gershgorin(lat->g, gw, grid, st)) return rc;
      std::vector<double> h(2 * grid);
      PVSC_CUDA_TRY(cudaMemcpyAsync(h.data(), gw, sizeof(double) * 2 * grid, cudaMemcpyDeviceToHost, st));
      PVSC_CUDA_TRY(cudaStreamSynchronize(st));
      double lo = h[0], hi = h[1];
      for (int i = 0; i < grid; ++i) {
        if (std::isnan(h[2 * i]) || std::isnan(h[2 * i + 1]))
          return set_error(PVSC_ERR_ARG, "the potential holds a non-finite value (PVSC_Q64 needs a bounded spectrum)");
        lo = std::fmin(lo, h[2 * i]);
        hi = std::fmax(hi, h[2 * i + 1]);
      }
      std::lock_guard<std::mutex> lk(ml->mu);
      ml->gersh_lo = lo;
      ml->gersh_hi = hi;
      ml->gersh_valid = true;
    }
    // the coupling coefficient kt = -t/a of the alpha = 2/a sweeps stays within
    // the range of the fixed-point products (|kt| <= 2); a lattice with any bond
    // has a >= |t| from the Gershgorin interval alone
    if (std::fabs(lat->g.t) > 2.0 * a)
      return set_error(PVSC_ERR_ARG, "PVSC_Q64 needs a >= |t| / 2 (a = %.17g, t = %.17g)", a, lat->g.t);
    const double lo = lat->gersh_lo, hi = lat->gersh_hi;
    const double slack = 1e-12 * a;
    if (lo < b - a - slack || hi > b + a + slack)
      return set_error(PVSC_ERR_ARG,
                       "PVSC_Q64 needs [b - a, b + a] to hold the spectrum bound [%.17g, %.17g] "
                       "(a = %.17g, b = %.17g)", lo, hi, a, b);
  }
  const std::vector<uint64_t> key = {7, (uint64_t)R, (uint64_t)PVSC_Q64, bits(r0), seed, (uint64_t)M,
                                     bits(a), bits(b), bits(mu), bits(work)};
  const LaunchShape sh = shape_for(lat, R, PVSC_Q64);
  const bool tuned = lat->tuning.count({R, PVSC_Q64}) != 0;
  auto body = [&](cudaStream_t cs) -> int {
    PVSC_CUDA_TRY(cudaMemsetAsync(work, 0, kWorkHeader, cs));
    if (int rc = launch_fx_prepare(lat, R, r0, seed, a, b, work, L, cs)) return rc;
    void* wa = wptr(work, L.wa);
    void* wb = wptr(work, L.wb);
    Sweep p;
    sweep_init(p, lat, R, PVSC_C128);
    p.C = R;
    p.counter = reinterpret_cast<unsigned*>(work);
    p.partials = reinterpret_cast<double*>(wptr(work, kWorkHeader));
    p.mu = mu;
    p.M = M;
    p.dot_flags = 3;
    p.fx_d = wptr(work, L.dfx);
    p.vscale = reinterpret_cast<const double*>(wptr(work, L.vscale));
    p.x = wa;
    p.yin = nullptr;
    p.yout = wb;
    p.dot_mode = 1;
    p.fx_dshift = 0;
    p.fx_kt = std::llrint(std::ldexp(-0.5 * lat->g.t / a, 60));
    if (int rc = launch_sweep_fx(lat, p, sh, tuned, cs)) return rc;
    void* prev = wa;
    void* cur = wb;
    p.fx_dshift = 1;
    p.fx_kt = std::llrint(std::ldexp(-lat->g.t / a, 60));
    p.dot_mode = 2;
    const int nsteps = (M + 1) / 2;
    for (int k = 1; k < nsteps; ++k) {
      p.x = cur;
      p.yin = prev;
      p.yout = prev;  // w_{k+1} overwrites w_{k-1} element by element
      p.kpm_k = k;
      if (int rc = launch_sweep_fx(lat, p, sh, tuned, cs)) return rc;
      std::swap(prev, cur);
    }
    return PVSC_OK;
  };
  return run_graph(lat, key, st, body);
}

int pvsc_kpm_moments(const pvsc_lattice* lat, int R, int prec, const void* r0, uint64_t seed,
                     int M, double a, double b, double* mu, void* work, size_t work_bytes,
                     void* stream) {
  if (prec == PVSC_Q64) {
    if (int rc = check_lattice(lat)) return rc;
    if (!valid_R(R)) return set_error(PVSC_ERR_ARG, "R = %d: must be 1, 2, 4, 8, 16, 32 or 64", R);
    if (int rc = check_scaling(a, b)) return rc;
    if (M < 1) return set_error(PVSC_ERR_ARG, "M = %d < 1", M);
    if (!mu) return set_error(PVSC_ERR_ARG, "mu is NULL");
    if (r0)
      if (int rc = check_ptr(r0, "r0")) return rc;
    return kpm_moments_fx(lat, R, r0, seed, M, a, b, mu, work, work_bytes,
                          static_cast<cudaStream_t>(stream));
  }
  if (int rc = check_common(lat, R, prec)) return rc;
  if (int rc = check_scaling(a, b)) return rc;
  if (M < 1) return set_error(PVSC_ERR_ARG, "M = %d < 1", M);
  if (!mu) return set_error(PVSC_ERR_ARG, "mu is NULL");
  if (r0)
    if (int rc = check_ptr(r0, "r0")) return rc;
  const size_t need = pvsc_work_bytes(lat, PVSC_OP_KPM, R, prec, M);
  if (int rc = check_work(work, work_bytes, need)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const std::vector<uint64_t> key = {1, (uint64_t)R, (uint64_t)prec, bits(r0), seed, (uint64_t)M,
                                     bits(a), bits(b), bits(mu), bits(work)};
  auto body = [&](cudaStream_t cs) -> int {
    return kpm_enqueue(lat, R, prec, r0, seed, M, a, b, mu, work, nullptr, cs);
  };
  return run_graph(lat, key, st, body);
}

int pvsc_kpm_sweeps(const pvsc_lattice* lat, int R, int prec, int k_begin, int k_end, void* wa, void* wb,
                    double a, double b, double* mu, int M, void* work, size_t work_bytes, void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (int rc = check_scaling(a, b)) return rc;
  if (int rc = check_ptr(wa, "wa")) return rc;
  if (int rc = check_ptr(wb, "wb")) return rc;
  if (wa == wb) return set_error(PVSC_ERR_ARG, "wa and wb must not overlap");
  if (M < 1 || !mu) return set_error(PVSC_ERR_ARG, "need M >= 1 and mu");
  const int nsweeps = (M + 1) / 2;
  if (k_begin < 0 || k_end < k_begin || k_end > nsweeps)
    return set_error(PVSC_ERR_ARG, "sweeps [%d, %d) outside [0, %d) for M = %d", k_begin, k_end, nsweeps, M);
  if (int rc = check_work(work, work_bytes, dots_work_bytes(lat, R))) return rc;
  if (k_end == k_begin) return PVSC_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PVSC_CUDA_TRY(cudaMemsetAsync(work, 0, kWorkHeader, st));
  Sweep p;
  sweep_init(p, lat, R, prec);
  p.counter = reinterpret_cast<unsigned*>(work);
  p.partials = reinterpret_cast<double*>(wptr(work, kWorkHeader));
  p.mu = mu;
  p.M = M;
  p.dot_flags = 3;
  for (int k = k_begin; k < k_end; ++k) {
    void* wk = (k % 2 == 0) ? wa : wb;    // w_j lives in wa for even j, in wb for odd j
    void* other = (k % 2 == 0) ? wb : wa;  // w_{k-1}, overwritten by w_{k+1}
    for (int r = 0; r < R; ++r) {
      p.coef[0][r] = (k == 0 ? 1.0 : 2.0) / a;
      p.coef[1][r] = b;
      p.coef[2][r] = k == 0 ? 0.0 : -1.0;
    }
    p.x = wk;
    p.yin = k == 0 ? nullptr : other;
    p.yout = other;
    p.dot_mode = k == 0 ? 1 : 2;
    p.kpm_k = k;
    if (int rc = launch_sweep(lat, prec, F_DOTS, p, st)) return rc;
  }
  return PVSC_OK;
}

int pvsc_debug_series_plan(int K, int* terms) {
  if (K < 1 || !terms) return set_error(PVSC_ERR_ARG, "need K >= 1 and an output array");
  std::vector<int> t;
  series_plan(K, t);
  std::copy(t.begin(), t.end(), terms);
  return PVSC_OK;
}

int pvsc_cheb_series(const pvsc_lattice* lat, int R, int prec, const void* x, void* y,
                     const double* coeffs, int K, const double* phase, double a, double b,
                     void* work, size_t work_bytes, void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (int rc = check_scaling(a, b)) return rc;
  if (int rc = check_ptr(x, "x")) return rc;
  if (int rc = check_ptr(y, "y")) return rc;
  if (K < 1 || !coeffs) return set_error(PVSC_ERR_ARG, "need K >= 1 coefficients");
  if (int rc = check_work(work, work_bytes, pvsc_work_bytes(lat, PVSC_OP_SERIES, R, prec, K))) return rc;
  std::vector<cd> cw(K);
  for (int k = 0; k < K; ++k) {
    cw[k] = cd(coeffs[2 * k], coeffs[2 * k + 1]);
    if (!std::isfinite(cw[k].real()) || !std::isfinite(cw[k].imag()))
      return set_error(PVSC_ERR_ARG, "coefficient %d is not finite", k);
  }
  const cd ph = phase ? cd(phase[0], phase[1]) : cd(1, 0);
  return run_series(lat, R, prec, x, y, cw, ph, a, b, work, static_cast<cudaStream_t>(stream));
}

int pvsc_cheb_filter(const pvsc_lattice* lat, int R, int prec, const void* x, void* y,
                     const double* g, int K, double a, double b, void* work,
                     size_t work_bytes, void* stream) {
  if (K < 1 || !g) return set_error(PVSC_ERR_ARG, "need K >= 1 coefficients");
  std::vector<double> c(2 * (size_t)K, 0.0);
  for (int k = 0; k < K; ++k) c[2 * k] = g[k];
  return pvsc_cheb_series(lat, R, prec, x, y, c.data(), K, nullptr, a, b, work, work_bytes, stream);
}

int pvsc_propagation_coeffs(double a_dt, double trunc, int max_terms, double* coeffs,
                            int* n_terms) {
  std::vector<cd> cw;
  if (int rc = propagation_weights(a_dt, trunc, cw)) return rc;
  if (n_terms) *n_terms = (int)cw.size();
  if (!coeffs || max_terms < (int)cw.size())
    return set_error(PVSC_ERR_ARG, "coefficient buffer holds %d < %d terms", max_terms, (int)cw.size());
  for (size_t k = 0; k < cw.size(); ++k) {
    coeffs[2 * k] = cw[k].real();
    coeffs[2 * k + 1] = cw[k].imag();
  }
  return PVSC_OK;
}

int pvsc_cheb_propagate(const pvsc_lattice* lat, int R, int prec, void* psi, double dt,
                        int nsteps, double a, double b, double trunc, void* work,
                        size_t work_bytes, void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (int rc = check_scaling(a, b)) return rc;
  if (int rc = check_ptr(psi, "psi")) return rc;
  if (nsteps < 0) return set_error(PVSC_ERR_ARG, "nsteps = %d < 0", nsteps);
  if (!std::isfinite(dt)) return set_error(PVSC_ERR_ARG, "dt is not finite");
  std::vector<cd> cw;
  if (int rc = propagation_weights(a * dt, trunc, cw)) return rc;
  if (int rc = check_work(work, work_bytes, pvsc_work_bytes(lat, PVSC_OP_SERIES, R, prec, (int)cw.size())))
    return rc;
  if (nsteps == 0) return PVSC_OK;
  const cd ph = std::exp(cd(0, -b * dt));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const std::vector<uint64_t> key = {2, (uint64_t)R, (uint64_t)prec, bits(psi), bits(dt), bits(a),
                                     bits(b), bits(trunc), bits(work)};
  auto body = [&](cudaStream_t cs) -> int {
    return run_series(lat, R, prec, psi, psi, cw, ph, a, b, work, cs);
  };
  for (int s = 0; s < nsteps; ++s)
    if (int rc = run_graph(lat, key, st, body)) return rc;
  return PVSC_OK;
}

int pvsc_cheb_adjoint_step(const pvsc_lattice* lat, int R, int prec, const void* psi_s,
                           void* G, double dt, double a, double b, double trunc,
                           double* dLdV, void* work, size_t work_bytes, void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (prec != PVSC_C128) return set_error(PVSC_ERR_UNSUPPORTED, "the adjoint runs in complex128 only");
  if (R != 1) return set_error(PVSC_ERR_UNSUPPORTED, "the adjoint takes one vector (R = 1)");
  if (int rc = check_scaling(a, b)) return rc;
  if (int rc = check_ptr(psi_s, "psi_s")) return rc;
  if (int rc = check_ptr(G, "G")) return rc;
  if (!dLdV) return set_error(PVSC_ERR_ARG, "dLdV is NULL");
  if (psi_s == G) return set_error(PVSC_ERR_ARG, "psi_s and G must not overlap");
  std::vector<cd> cw;
  if (int rc = propagation_weights(a * dt, trunc, cw)) return rc;
  const int M = (int)cw.size() - 1;
  if (int rc = check_work(work, work_bytes, pvsc_work_bytes(lat, PVSC_OP_ADJOINT, R, prec, M + 1)))
    return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vb = vec_bytes(lat, R, PVSC_C128);
  // work: [hdr | W_1 .. W_{M-1} | uA | uB]
  auto Wk = [&](int k) -> void* { return k == 0 ? const_cast<void*>(psi_s) : wptr(work, kWorkHeader + (k - 1) * vb); };
  void* ubuf[2] = {wptr(work, kWorkHeader + (size_t)(M > 1 ? M - 1 : 0) * vb),
                   wptr(work, kWorkHeader + (size_t)(M > 1 ? M : 1) * vb)};
  const cd cphi = std::exp(cd(0, b * dt));  // conj(e^{-i b dt})
  auto sigma = [&](int k) { return std::conj(cw[k]) * cphi; };
  const int64_t n = lat->g.n_sites * orbitals_of(lat->g.model);
  if (M == 0) {
    const cd s0 = sigma(0);
    return launch_scale_init(G, static_cast<double2*>(G), s0.real(), s0.imag(), n, st);
  }
  Sweep p;
  sweep_init(p, lat, R, prec);
  // forward: w_1 .. w_{M-1}
  for (int k = 1; k < M; ++k) {
    p.coef[0][0] = (k == 1 ? 1.0 : 2.0) / a;
    p.coef[1][0] = b;
    p.coef[2][0] = (k == 1 ? 0.0 : -1.0);
    p.x = Wk(k - 1);
    p.yin = k == 1 ? nullptr : Wk(k - 2);
    p.yout = Wk(k);
    if (int rc = launch_sweep(lat, prec, 0, p, st)) return rc;
  }
  // u_M = sigma_M G, grad += (f_{M-1}/a) Re conj(u_M) w_{M-1}
  {
    const cd s = sigma(M);
    const double f = (M - 1 == 0) ? 1.0 : 2.0;
    if (int rc = launch_adjoint_top(lat, R, static_cast<const double2*>(G), s.real(), s.imag(),
                                    static_cast<double2*>(ubuf[0]), static_cast<const double2*>(Wk(M - 1)),
                                    f / a, dLdV, st))
      return rc;
  }
  // u_k for k = M-1 .. 1 (u_{k+1} in cur, u_{k+2} in prev)
  void* cur = ubuf[0];
  void* prev = nullptr;
  for (int k = M - 1; k >= 1; --k) {
    void* out = prev ? prev : ubuf[1];
    const cd s = sigma(k);
    p.coef[0][0] = 2.0 / a;
    p.coef[1][0] = b;
    p.coef[2][0] = prev ? -1.0 : 0.0;
    p.x = cur;
    p.yin = prev;
    p.yout = out;
    p.src = static_cast<const double2*>(G);
    p.sg_re = s.real();
    p.sg_im = s.imag();
    p.wg = Wk(k - 1);
    p.grad = dLdV;
    p.gscale = ((k - 1 == 0) ? 1.0 : 2.0) / a;
    if (int rc = launch_sweep(lat, prec, F_ADJ, p, st)) return rc;
    prev = cur;
    cur = out;
  }
  // u_0 = sigma_0 G + H~ u_1 - u_2, written over G
  {
    const cd s = sigma(0);
    p.coef[0][0] = 1.0 / a;
    p.coef[1][0] = b;
    p.coef[2][0] = prev ? -1.0 : 0.0;
    p.x = cur;
    p.yin = prev;
    p.yout = G;
    p.src = static_cast<const double2*>(G);
    p.sg_re = s.real();
    p.sg_im = s.imag();
    p.wg = nullptr;
    p.grad = nullptr;
    if (int rc = launch_sweep(lat, prec, F_ADJ, p, st)) return rc;
  }
  return PVSC_OK;
}

int pvsc_cheb_propagate_checkpointed(const pvsc_lattice* lat, int R, int prec, void* psi, double dt,
                                     int nsteps, int every, double a, double b, double trunc, void* ckpts,
                                     void* work, size_t work_bytes, void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (int rc = check_ptr(psi, "psi")) return rc;
  if (int rc = check_ptr(ckpts, "ckpts")) return rc;
  if (every < 1) return set_error(PVSC_ERR_ARG, "every = %d < 1", every);
  if (nsteps < 0) return set_error(PVSC_ERR_ARG, "nsteps = %d < 0", nsteps);
  if (ckpts == psi || ckpts == work) return set_error(PVSC_ERR_ARG, "ckpts must not overlap psi or work");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vb = vec_bytes(lat, R, PVSC_C128);
  for (int s0 = 0, seg = 0; s0 < nsteps; s0 += every, ++seg) {
    PVSC_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(ckpts) + (size_t)seg * vb, psi, vb,
                                  cudaMemcpyDeviceToDevice, st));
    const int n = nsteps - s0 < every ? nsteps - s0 : every;
    if (int rc = pvsc_cheb_propagate(lat, R, prec, psi, dt, n, a, b, trunc, work, work_bytes, stream))
      return rc;
  }
  return PVSC_OK;
}

size_t pvsc_propagate_adjoint_work_bytes(const pvsc_lattice* lat, int R, int every, double a_dt,
                                         double trunc) {
  if (!lat || R != 1 || every < 1) return 0;
  std::vector<cd> cw;
  if (propagation_weights(a_dt, trunc, cw) != PVSC_OK) return 0;
  const int K = (int)cw.size();
  const size_t vb = vec_bytes(lat, R, PVSC_C128);
  const size_t ser = (pvsc_work_bytes(lat, PVSC_OP_SERIES, R, PVSC_C128, K) + 255) & ~size_t(255);
  const size_t adj = pvsc_work_bytes(lat, PVSC_OP_ADJOINT, R, PVSC_C128, K);
  return (size_t)every * vb + ser + adj;
}

int pvsc_cheb_propagate_adjoint(const pvsc_lattice* lat, int R, int prec, const void* ckpts, double dt,
                                int nsteps, int every, double a, double b, double trunc, void* G,
                                double* dLdV, void* work, size_t work_bytes, void* stream) {
  if (int rc = check_common(lat, R, prec)) return rc;
  if (prec != PVSC_C128) return set_error(PVSC_ERR_UNSUPPORTED, "the adjoint runs in complex128 only");
  if (R != 1) return set_error(PVSC_ERR_UNSUPPORTED, "the adjoint takes one vector (R = 1)");
  if (int rc = check_scaling(a, b)) return rc;
  if (int rc = check_ptr(ckpts, "ckpts")) return rc;
  if (int rc = check_ptr(G, "G")) return rc;
  if (!dLdV) return set_error(PVSC_ERR_ARG, "dLdV is NULL");
  if (every < 1) return set_error(PVSC_ERR_ARG, "every = %d < 1", every);
  if (nsteps < 0) return set_error(PVSC_ERR_ARG, "nsteps = %d < 0", nsteps);
  if (!std::isfinite(dt)) return set_error(PVSC_ERR_ARG, "dt is not finite");
  const size_t need = pvsc_propagate_adjoint_work_bytes(lat, R, every, a * dt, trunc);
  if (need == 0) return set_error(PVSC_ERR_ARG, "invalid a * dt or trunc");
  if (int rc = check_work(work, work_bytes, need)) return rc;
  if (nsteps == 0) return PVSC_OK;
  std::vector<cd> cw;
  if (int rc = propagation_weights(a * dt, trunc, cw)) return rc;
  const int K = (int)cw.size();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vb = vec_bytes(lat, R, PVSC_C128);
  const size_t ser = (pvsc_work_bytes(lat, PVSC_OP_SERIES, R, PVSC_C128, K) + 255) & ~size_t(255);
  const size_t adj = pvsc_work_bytes(lat, PVSC_OP_ADJOINT, R, PVSC_C128, K);
  char* states = static_cast<char*>(work);
  void* swork = states + (size_t)every * vb;
  void* awork = states + (size_t)every * vb + ser;
  const cd ph = std::exp(cd(0, -b * dt));
  const int nseg = (nsteps + every - 1) / every;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int s0 = seg * every;
    const int n = nsteps - s0 < every ? nsteps - s0 : every;
    // the states psi_{s0} .. psi_{s0+n-1} of this segment, from its checkpoint
    PVSC_CUDA_TRY(cudaMemcpyAsync(states, static_cast<const char*>(ckpts) + (size_t)seg * vb, vb,
                                  cudaMemcpyDeviceToDevice, st));
    for (int j = 1; j < n; ++j) {
      void* sj = states + (size_t)j * vb;
      PVSC_CUDA_TRY(cudaMemcpyAsync(sj, states + (size_t)(j - 1) * vb, vb, cudaMemcpyDeviceToDevice, st));
      if (int rc = run_series(lat, R, PVSC_C128, sj, sj, cw, ph, a, b, swork, st)) return rc;
    }
    // the adjoint steps, last to first
    for (int j = n - 1; j >= 0; --j)
      if (int rc = pvsc_cheb_adjoint_step(lat, R, prec, states + (size_t)j * vb, G, dt, a, b, trunc, dLdV,
                                          awork, adj, stream))
        return rc;
  }
  return PVSC_OK;
}

int pvsc_device_error(int* flag, int clear) {
  if (!flag) return set_error(PVSC_ERR_ARG, "flag is NULL");
  PVSC_CUDA_TRY(cudaDeviceSynchronize());
  int a = 0, b = 0, c = 0;
  if (int rc = bulk_sweep_error(PVSC_C128, clear, &a)) return rc;
  if (int rc = bulk_sweep_error(PVSC_C64, clear, &b)) return rc;
  if (int rc = tma_error(clear, &c)) return rc;
  *flag = (a || b || c) ? 1 : 0;
  return PVSC_OK;
}

// Launch shapes of the fixed-point KPM sweep: kernel 0, 2 or 3, one vector per
// thread; or kernel 7, the TMA-staged tiles of the complex64 layout of 2R vectors.
static int check_q64_tuning(const pvsc_lattice* lat, int R, const pvsc_tuning* t) {
  if (int rc = check_lattice(lat)) return rc;
  if (!valid_R(R)) return set_error(PVSC_ERR_ARG, "R = %d: must be 1, 2, 4, 8, 16, 32 or 64", R);
  if (lat->g.model != PVSC_TI) return set_error(PVSC_ERR_UNSUPPORTED, "PVSC_Q64 is for the TI lattice only");
  if (!t) return PVSC_OK;
  if (t->kernel == kKernelTma) {
    if (!tma_fx_possible(lat, R))
      return set_error(PVSC_ERR_ARG, "PVSC_Q64 kernel 7 (TMA-staged tiles) needs R = 1 .. 32");
    if (!tma_tile_valid(2 * R, t->tile_x, t->tile_y))
      return set_error(PVSC_ERR_ARG, "PVSC_Q64 kernel 7 takes no tile other than the two of R = %d (%dx%d given)",
                       R, t->tile_x, t->tile_y);
    if (t->blocks_per_sm < 0 || t->blocks_per_sm > 1 || t->zslab < 0)
      return set_error(PVSC_ERR_ARG, "kernel 7 takes blocks_per_sm 0 or 1 and zslab >= 0");
    return PVSC_OK;
  }
  if (t->kernel != 0 && t->kernel != 2 && t->kernel != 3)
    return set_error(PVSC_ERR_ARG, "PVSC_Q64 kernels are 0, 2, 3 and 7");
  if (t->vpt > 1 || t->tile_x || t->tile_y)
    return set_error(PVSC_ERR_ARG, "PVSC_Q64 sweeps take one vector per thread and no staged tile");
  if (t->threads < 32 || t->threads > kMaxThreads || t->threads % 32 || t->threads % R)
    return set_error(PVSC_ERR_ARG, "threads must be a multiple of 32 and of R, at most %d", kMaxThreads);
  if (t->blocks_per_sm < 0 || t->zslab < 0) return set_error(PVSC_ERR_ARG, "negative tuning value");
  return PVSC_OK;
}

int pvsc_set_tuning(pvsc_lattice* lat, int R, int prec, const pvsc_tuning* tuning) {
  if (prec == PVSC_Q64) {
    if (int rc = check_q64_tuning(lat, R, tuning)) return rc;
    if (tuning) lat->tuning[{R, prec}] = *tuning; else lat->tuning.erase({R, prec});
    drop_graphs(lat);
    return PVSC_OK;
  }
  if (int rc = check_common(lat, R, prec)) return rc;
  if (!tuning) {
    lat->tuning.erase({R, prec});
    drop_graphs(lat);
    return PVSC_OK;
  }
  if (tuning->vpt < 0 || tuning->vpt > 2) return set_error(PVSC_ERR_ARG, "vpt must be 0, 1 or 2");
  if (tuning->kernel < 0 || tuning->kernel > 8) return set_error(PVSC_ERR_ARG, "kernel must be 0 .. 8");
  if (tuning->kernel == kKernelTma || tuning->kernel == kKernelTmaX) {
    const int k = tuning->kernel;
    if (k == kKernelTma && !tma_sweep_possible(lat, R, prec))
      return set_error(PVSC_ERR_ARG, "kernel 7 (TMA-staged tiles) needs a TI or Weyl lattice, complex64 "
                       "and Lx a multiple of 4");
    if (k == kKernelTmaX && !tma_xm_possible(lat, R, prec))
      return set_error(PVSC_ERR_ARG, "kernel 8 (TMA-staged tiles marching along x) needs a TI or Weyl lattice, "
                       "complex64, R >= 4 and Lx a multiple of 4");
    if (k == kKernelTmaX && tuning->threads == 512)
      return set_error(PVSC_ERR_ARG, "kernel 8 runs eight warps (threads 256)");
    if (k == kKernelTmaX && lat->g.model == PVSC_WSM && tuning->tile_y != 0 && tma_tile_deep(R, tuning->tile_y))
      return set_error(PVSC_ERR_ARG, "kernel 8 runs the large tile on Weyl cells");
    if (!tma_tile_valid(R, tuning->tile_x, tuning->tile_y))
      return set_error(PVSC_ERR_ARG, "kernel %d takes no tile other than the two of R = %d (%dx%d given)", k, R,
                       tuning->tile_x, tuning->tile_y);
    if (tuning->blocks_per_sm < 0 || tuning->blocks_per_sm > 1 || tuning->zslab < 0)
      return set_error(PVSC_ERR_ARG, "kernels 7 and 8 take blocks_per_sm 0 or 1 and zslab >= 0");
    lat->tuning[{R, prec}] = *tuning;
    drop_graphs(lat);
    return PVSC_OK;
  }
  if (tuning->kernel == kKernelXMarch && lat->g.model != PVSC_TI)
    return set_error(PVSC_ERR_ARG, "kernel 6 (marching along x) needs a TI lattice");
  if (tuning->kernel == kKernelTiles) {
    const int C = R / vpt_tuned(tuning->vpt, R, prec);
    const int n = tuning->tile_x * tuning->tile_y * C;
    if (lat->g.model != PVSC_TI || tuning->tile_x < 1 || tuning->tile_y < 1 || n % 32 || n > kMaxThreads)
      return set_error(PVSC_ERR_ARG, "kernel 5 (column tiles) needs a TI lattice and tile_x tile_y R/VPT "
                       "a multiple of 32, at most %d (got %d)", kMaxThreads, n);
    if (tuning->vpt < 0 || tuning->vpt > 2 || tuning->blocks_per_sm < 0 || tuning->zslab < 0)
      return set_error(PVSC_ERR_ARG, "invalid tuning value");
    lat->tuning[{R, prec}] = *tuning;
    drop_graphs(lat);
    return PVSC_OK;
  }
  if (tuning->kernel == kKernelKpm2) {
    if (tuning->blocks_per_sm < 0 || tuning->zslab < 0 || tuning->tile_x < 0 || tuning->tile_y < 0)
      return set_error(PVSC_ERR_ARG, "negative tuning value");
    if (!kpm2_possible(lat, R, prec))
      return set_error(PVSC_ERR_ARG, "kernel 4 (two KPM steps per sweep) needs a TI lattice, complex64 and R >= 2");
    if (int rc = kpm2_check_tile(tuning->tile_x, tuning->tile_y, R)) return rc;
    lat->tuning[{R, prec}] = *tuning;
    drop_graphs(lat);
    return PVSC_OK;
  }
  const int C = R / vpt_tuned(tuning->vpt, R, prec);
  if (tuning->threads < 32 || tuning->threads > kMaxThreads || tuning->threads % 32 || tuning->threads % C)
    return set_error(PVSC_ERR_ARG, "threads must be a multiple of 32 and of R/VPT = %d, at most %d", C, kMaxThreads);
  if (tuning->blocks_per_sm < 0 || tuning->zslab < 0 || tuning->tile_x < 0 || tuning->tile_y < 0)
    return set_error(PVSC_ERR_ARG, "negative tuning value");
  if (tuning->tile_x > 0 || tuning->tile_y > 0) {
    if (tuning->kernel != 0)
      return set_error(PVSC_ERR_ARG, "kernel %d takes no tile: tile_x and tile_y select the staged "
                       "sweep of kernel 0 (and the tiles of kernels 4 and 5)", tuning->kernel);
    if (lat->g.model != PVSC_TI || tuning->tile_x < 1 || tuning->tile_y < 1)
      return set_error(PVSC_ERR_ARG, "a staged tile needs a TI lattice and tile_x, tile_y >= 1");
    if (tuning->threads % R) return set_error(PVSC_ERR_ARG, "staged sweeps need threads %% R == 0");
    if (bulk_smem_bytes(tuning->tile_x, tuning->tile_y, R, prec) > 200 * 1024)
      return set_error(PVSC_ERR_ARG, "staged tile %dx%d does not fit in shared memory", tuning->tile_x,
                       tuning->tile_y);
  }
  lat->tuning[{R, prec}] = *tuning;
  drop_graphs(lat);
  return PVSC_OK;
}

int pvsc_get_tuning(const pvsc_lattice* lat, int R, int prec, pvsc_tuning* tuning) {
  if (!tuning) return set_error(PVSC_ERR_ARG, "tuning is NULL");
  if (prec == PVSC_Q64) {
    if (int rc = check_q64_tuning(lat, R, nullptr)) return rc;
    auto it = lat->tuning.find({R, prec});
    if (it != lat->tuning.end()) {
      *tuning = it->second;
    } else {
      *tuning = pvsc_tuning{128, 0, 0, 0.f, 1, 0, 0, R >= 2 ? 2 : 0};
    }
    return PVSC_OK;
  }
  if (int rc = check_common(lat, R, prec)) return rc;
  auto it = lat->tuning.find({R, prec});
  if (it != lat->tuning.end()) {
    *tuning = it->second;
  } else {
    tuning->threads = 256;
    tuning->blocks_per_sm = 0;
    tuning->zslab = 0;
    tuning->time_ms = 0.f;
    tuning->vpt = vpt_for(R, prec);
    tuning->tile_x = 0;
    tuning->tile_y = 0;
    tuning->kernel = 0;
  }
  return PVSC_OK;
}

}  // extern "C"
