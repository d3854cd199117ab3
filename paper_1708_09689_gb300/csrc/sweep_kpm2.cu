// Two KPM recurrence steps per sweep (temporal blocking of the Chebyshev loop):
//   w_{k+1} = 2 H~ w_k - w_{k-1},   w_{k+2} = 2 H~ w_{k+1} - w_k,
// H of Eq. TB_H_topi, fused with the four dot products <w_k|w_k>,
// Re<w_{k+1}|w_k>, <w_{k+1}|w_{k+1}> and Re<w_{k+2}|w_{k+1}> that give the
// moments mu_2k .. mu_2k+3 (Sec. 4.1).  complex64 storage, fp32 stencil
// arithmetic, fp64 dot accumulation, as the single-step complex64 sweep.
//
// A block owns a tile of TX x TY columns (all R vectors, two per thread, the
// chunks of a site on adjacent lanes as in the single sweeps) and a z-range
// [z0, z1), and marches along z.  At plane z every thread computes
// w_{k+1} on its column: the threads of the tile, and those of a one-column
// ring around it (overlapped tiling: the ring columns belong to the
// neighbouring tiles, which compute them as well).  The last four planes of
// w_{k+1} on tile and ring are kept in shared memory; after one block barrier
// the tile threads compute w_{k+2} at plane z - 1 from them, with w_k(z - 1)
// still in registers from the march.  Per two steps a site's vectors make four
// passes through HBM (read w_{k-1}, w_k; write w_{k+1}, w_{k+2}) instead of the
// six of two single sweeps.
//
// The stencil arithmetic is the single sweep's (ti_axes / ti_combine with the
// neighbours in the same order), so w_{k+1} and w_{k+2} equal two single
// sweeps' results bit for bit; only the order of the dot-product sums differs.
#include "internal.h"
#include "sweep.cuh"

namespace pvsc {

// Threads per block: one per (column of tile and ring, vector chunk), rounded
// up to whole warps.  Blocks of up to 8 warps get the whole register budget
// (two warps per SM sub-partition); up to 12 warps run with 168 registers.
constexpr int kKpm2Threads = 384;

// Coordinate c in [-2, L + 1] wrapped onto [0, L) on a periodic axis; -1 past
// the end of an open axis.
__device__ __forceinline__ int64_t kpm2_wrap(int64_t c, int64_t L, int per) {
  if (c >= 0 && c < L) return c;
  if (!per) return -1;
  while (c < 0) c += L;
  while (c >= L) c -= L;
  return c;
}

// Ring of w_{k+1} planes in shared memory: 16-byte granule (orbital) k of
// chunk rc of local column n in slot q at (((q * 4 + k) * NS + n) * C + rc) *
// 16 bytes.  Consecutive threads hold consecutive (n, rc), so every access is
// conflict-free; the pointer passed is the granule of (q, k = 0, n, rc) and
// orbitals sit NS C granules apart.
__device__ __forceinline__ void kpm2_put(unsigned char* g0, int ostride, const Blk<float, 2>& b) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    *reinterpret_cast<float4*>(g0 + (size_t)k * ostride) =
        make_float4(b.v[k][0].re, b.v[k][0].im, b.v[k][1].re, b.v[k][1].im);
}
__device__ __forceinline__ void kpm2_get(const unsigned char* g0, int ostride, Blk<float, 2>& b) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(g0 + (size_t)k * ostride);
    b.v[k][0] = {a.x, a.y};
    b.v[k][1] = {a.z, a.w};
  }
}

// Dot-product partial sums of one thread: compensated fp32 pairs (TwoSum, as
// the single sweeps), flushed once per unit into an fp64 slot of this thread
// in shared memory, so the fp64 sums hold no registers during the march.
struct Kpm2Dots {
  float s[kNumDots][2], c[kNumDots][2];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int k = 0; k < kNumDots; ++k)
#pragma unroll
      for (int v = 0; v < 2; ++v) s[k][v] = c[k][v] = 0.f;
  }
  __device__ __forceinline__ void add(int k, int v, float x) {
    const float t = s[k][v] + x;
    const float bp = t - s[k][v];
    c[k][v] += (s[k][v] - (t - bp)) + (x - bp);
    s[k][v] = t;
  }
  // Per-site products of one step: dot d0 += <x|x>, d0 + 1 += Re<y|x>.
  __device__ __forceinline__ void site(int d0, const Blk<float, 2>& x, const Blk<float, 2>& y) {
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      float xx = 0.f, xy = 0.f;
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const cplx<float> a = x.v[o][v], b = y.v[o][v];
        xx = fmaf(a.re, a.re, fmaf(a.im, a.im, xx));
        xy = fmaf(b.re, a.re, fmaf(b.im, a.im, xy));
      }
      add(d0, v, xx);
      add(d0 + 1, v, xy);
    }
  }
  // fp64 slots: dsum[(k * 2 + v) * nthr + tid]
  __device__ __forceinline__ void flush(double* dsum, int nthr, int tid) {
#pragma unroll
    for (int k = 0; k < kNumDots; ++k)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        dsum[(k * 2 + v) * nthr + tid] += (double)s[k][v] + (double)c[k][v];
        s[k][v] = c[k][v] = 0.f;
      }
  }
};

// p.x = w_k, p.yin = w_{k-1}, p.yout = w_{k+1}, p.yout2 = w_{k+2} (four
// distinct buffers: the ring columns read w_k and w_{k-1} of the neighbouring
// tiles); p.tile_x, p.tile_y = TX, TY; p.zslab = z-range of a unit; thread t
// carries vector chunk t % C of local column t / C (C = R / 2 a power of two).
template <int MAXT>
__global__ void __launch_bounds__(MAXT) ti_kpm2_sweep(const __grid_constant__ Sweep p) {
  using T = float;
  constexpr int VPT = 2;
  using B = Blk<T, VPT>;
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = p.g;
  const int64_t Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], plane = Lx * Ly;
  const int TX = p.tile_x, TY = p.tile_y, GX = TX + 2, NS = GX * (TY + 2);
  const int R = p.R, C = p.C;
  const int cshift = __ffs(C) - 1;
  const int t = threadIdx.x, nthr = blockDim.x;
  const int rc = t & (C - 1), sl = t >> cshift;
  const VecCoef<T, VPT> cf = load_coef<T, VPT>(p, rc);
  const T* __restrict__ X = static_cast<const T*>(p.x);
  const T* __restrict__ Yin = static_cast<const T*>(p.yin);
  T* __restrict__ Y1 = static_cast<T*>(p.yout);
  T* __restrict__ Y2 = static_cast<T*>(p.yout2);
  unsigned char* ring = smem;
  double* dsum = reinterpret_cast<double*>(smem + (size_t)4 * 4 * NS * C * 16);

  // local position (li, lj) of column slot sl in the (TX + 2) x (TY + 2) grid
  // of tile and ring: slots [0, TX TY) the tile row by row, then the ring's
  // bottom, top, left and right edges (corners are not needed)
  const int ntile = TX * TY;
  int li = -1, lj = -1;
  if (sl < ntile) {
    li = 1 + sl % TX;
    lj = 1 + sl / TX;
  } else if (sl < ntile + 2 * (TX + TY)) {
    const int q = sl - ntile;
    if (q < TX) { li = 1 + q; lj = 0; }
    else if (q < 2 * TX) { li = 1 + q - TX; lj = TY + 1; }
    else if (q < 2 * TX + TY) { li = 0; lj = 1 + q - 2 * TX; }
    else { li = TX + 1; lj = 1 + q - 2 * TX - TY; }
  }
  const int me = lj * GX + li;
  // ring granule addressing (bytes): slot stride, orbital stride, own granule
  const int ostride = NS * C * 16, qstride = 4 * ostride;
  const int gme = (me * C + rc) * 16;
  const int gdx = C * 16, gdy = GX * C * 16;

  for (int k = 0; k < 2 * kNumDots; ++k) dsum[k * nthr + t] = 0.0;
  Kpm2Dots dacc;
  dacc.init();
  const int64_t ntx = (Lx + TX - 1) / TX, nty = (Ly + TY - 1) / TY, ntiles = ntx * nty;
  const int64_t zs = p.zslab, nzs = (Lz + zs - 1) / zs, nunits = ntiles * nzs;
  const int64_t SS = (int64_t)8 * R, PS = plane * SS, cofs = 2 * rc * VPT;

  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t bz = udiv64(u, ntiles), tile = u - bz * ntiles;
    const int64_t ty = udiv64(tile, ntx), tx = tile - ty * ntx;
    const int64_t x0 = tx * TX, y0 = ty * TY;
    const int wx = (int)min((int64_t)TX, Lx - x0), wy = (int)min((int64_t)TY, Ly - y0);
    const int64_t z0 = bz * zs, z1 = min(z0 + zs, Lz);
    // role in this unit: tile column, ring column (also the tile-grid
    // positions just past a partial tile's edge), or idle
    const bool in_x = li >= 1 && li <= wx, in_y = lj >= 1 && lj <= wy;
    const bool tile_role = in_x && in_y;
    const bool ring_role = (in_y && (li == 0 || li == wx + 1)) || (in_x && (lj == 0 || lj == wy + 1));
    int64_t col = -1, gx = 0, gy = 0;
    if (tile_role || ring_role) {
      gx = kpm2_wrap(x0 - 1 + li, Lx, g.per[0]);
      gy = kpm2_wrap(y0 - 1 + lj, Ly, g.per[1]);
      if (gx >= 0 && gy >= 0) col = gx + Lx * gy;  // else past an open edge: zero
    }
    const bool active = col >= 0;
    const int64_t c0 = active ? col : 0;
    const int64_t cxm = active ? nbr_minus(c0, gx, Lx, g.per[0], 1) : -1;
    const int64_t cxp = active ? nbr_plus(c0, gx, Lx, g.per[0], 1) : -1;
    const int64_t cym = active ? nbr_minus(c0, gy, Ly, g.per[1], Lx) : -1;
    const int64_t cyp = active ? nbr_plus(c0, gy, Ly, g.per[1], Lx) : -1;
    const T* Pc = X + c0 * SS + cofs;
    const T* Pxm = X + (cxm >= 0 ? cxm : 0) * SS + cofs;
    const T* Pxp = X + (cxp >= 0 ? cxp : 0) * SS + cofs;
    const T* Pym = X + (cym >= 0 ? cym : 0) * SS + cofs;
    const T* Pyp = X + (cyp >= 0 ? cyp : 0) * SS + cofs;
    const T* Py = Yin + c0 * SS + cofs;
    T* Q1 = Y1 + c0 * SS + cofs;
    T* Q2 = Y2 + c0 * SS + cofs;

    // w_k of this column at plane z (zero past an open end or an absent column)
    auto load_wk = [&](int64_t z, B& b) {
      const int64_t pz = kpm2_wrap(z, Lz, g.per[2]);
      if (active && pz >= 0) load_at<T, VPT, true>(Pc + pz * PS, R, b);
      else zero_blk(b);
    };
    B xm, xc, xp;  // w_k at planes z - 1, z, z + 1 of the step-1 plane z
    load_wk(z0 - 2, xm);
    load_wk(z0 - 1, xc);
    __syncthreads();  // the previous unit's last ring reads are done
    // step-1 planes z0 - 1 .. z1 (w_{k+1} one plane beyond the unit's range on
    // each side feeds the z-neighbours of step 2)
    const int n = (int)(z1 - z0) + 2;
    for (int i = 0; i < n; ++i) {
      const int64_t z = z0 - 1 + i;
      const int64_t pz = kpm2_wrap(z, Lz, g.per[2]);
      load_wk(z + 1, xp);
      B yn;
      if (active && pz >= 0) {
        const int64_t zoff = pz * PS;
        B yi, ax, bx, ay, by, S, D;
        load_at<T, VPT, false>(Py + zoff, R, yi);
        if (cxm >= 0) load_at<T, VPT, true>(Pxm + zoff, R, ax); else zero_blk(ax);
        if (cxp >= 0) load_at<T, VPT, true>(Pxp + zoff, R, bx); else zero_blk(bx);
        if (cym >= 0) load_at<T, VPT, true>(Pym + zoff, R, ay); else zero_blk(ay);
        if (cyp >= 0) load_at<T, VPT, true>(Pyp + zoff, R, by); else zero_blk(by);
        const T Vs = site_potential_t<T>(g, c0 + plane * pz);
        ti_axes(xm, xp, ax, bx, ay, by, S, D);
        ti_combine(cf, Vs, xc, S, D, &yi, yn, g);
        if (tile_role && z >= z0 && z < z1) {
          store_blk<T, VPT>(Q1 + zoff, 0, R, 0, yn);
          dacc.site(0, xc, yn);
        }
      } else {
        zero_blk(yn);
      }
      if (tile_role || ring_role) kpm2_put(ring + (i & 3) * qstride + gme, ostride, yn);
      __syncthreads();  // plane z of w_{k+1} complete on tile and ring
      if (tile_role && i >= 2) {
        // step 2 at plane z - 1 (inside [z0, z1)): slots i-2, i-1, i hold
        // w_{k+1} at planes z - 2, z - 1, z
        const int64_t zz = z - 1;
        const unsigned char* qc = ring + ((i - 1) & 3) * qstride + gme;
        B c1, a, b, S, D, y2;
        kpm2_get(ring + ((i - 2) & 3) * qstride + gme, ostride, a);
        kpm2_get(ring + (i & 3) * qstride + gme, ostride, b);
        axis_z_init(a, b, S, D);
        kpm2_get(qc - gdx, ostride, a);
        kpm2_get(qc + gdx, ostride, b);
        axis_x_add(a, b, S, D);
        kpm2_get(qc - gdy, ostride, a);
        kpm2_get(qc + gdy, ostride, b);
        axis_y_add(a, b, S, D);
        kpm2_get(qc, ostride, c1);
        const T Vs = site_potential_t<T>(g, c0 + plane * zz);
        ti_combine(cf, Vs, c1, S, D, &xm, y2, g);  // xm = w_k(z - 1)
        store_blk<T, VPT>(Q2 + zz * PS, 0, R, 0, y2);
        dacc.site(2, c1, y2);
      }
      xm = xc;
      xc = xp;
    }
    dacc.flush(dsum, nthr, t);  // one fp64 add per dot and unit
  }
  double acc[kNumDots][VPT];
#pragma unroll
  for (int k = 0; k < kNumDots; ++k)
#pragma unroll
    for (int v = 0; v < VPT; ++v) acc[k][v] = dsum[(k * 2 + v) * nthr + t];
  reduce_dots<VPT, MAXT / 32>(p, acc);
}

// default tile per number of vector chunks C = R / 2: about 380 threads or
// fewer (tile plus ring times C)
static void kpm2_default_tile(int C, int& TX, int& TY) {
  switch (C) {
    case 1: TX = 16; TY = 12; break;
    case 2: TX = 10; TY = 8; break;
    case 4: TX = 8; TY = 8; break;
    case 8: TX = 5; TY = 5; break;
    case 16: TX = 3; TY = 3; break;
    default: TX = 2; TY = 2; break;
  }
}

int kpm2_threads(int TX, int TY, int C) {
  const int n = (TX * TY + 2 * (TX + TY)) * C;
  return (n + 31) / 32 * 32;
}

size_t kpm2_smem_bytes(int TX, int TY, int C, int threads) {
  return (size_t)4 * 4 * 16 * (TX + 2) * (TY + 2) * C + (size_t)2 * kNumDots * sizeof(double) * threads;
}

int kpm2_check_tile(int TX, int TY, int R) {
  const int C = R / 2;
  int DX = 0, DY = 0;
  kpm2_default_tile(C, DX, DY);
  if (TX == 0) TX = DX;  // 0: the default of this R
  if (TY == 0) TY = DY;
  if (TX < 1 || TY < 1 || kpm2_threads(TX, TY, C) > kKpm2Threads)
    return set_error(PVSC_ERR_ARG,
                     "two-step KPM tile %dx%d: needs tile_x, tile_y >= 1 and (tile plus ring) "
                     "x R/2 = (tile_x tile_y + 2 (tile_x + tile_y)) x %d at most %d threads",
                     TX, TY, C, kKpm2Threads);
  return PVSC_OK;
}

int launch_kpm2_sweep(const pvsc_lattice* lat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  if (p.R < 2 || p.R % 2) return set_error(PVSC_ERR_ARG, "two-step KPM sweep needs R >= 2");
  p.C = p.R / 2;
  int TX = 0, TY = 0;
  kpm2_default_tile(p.C, TX, TY);
  if (sh.tile_x > 0) TX = sh.tile_x;
  if (sh.tile_y > 0) TY = sh.tile_y;
  if (int rc = kpm2_check_tile(TX, TY, p.R)) return rc;
  const int threads = kpm2_threads(TX, TY, p.C);
  const size_t smem = kpm2_smem_bytes(TX, TY, p.C, threads);
  void* fn = threads <= 256 ? reinterpret_cast<void*>(&ti_kpm2_sweep<256>)
                            : reinterpret_cast<void*>(&ti_kpm2_sweep<kKpm2Threads>);
  if (int rc = allow_max_smem(fn)) return rc;
  int occ = 0;
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem));
  if (occ < 1) return set_error(PVSC_ERR_ARG, "two-step KPM sweep does not fit on an SM");
  int bps = sh.blocks_per_sm;
  if (bps <= 0 || bps > occ) bps = occ;
  if (bps > kMaxGridPerSM) bps = kMaxGridPerSM;
  p.tile_x = TX;
  p.tile_y = TY;
  const int64_t Lx = lat->g.L[0], Ly = lat->g.L[1], Lz = lat->g.L[2];
  int64_t zs = sh.zslab > 0 ? sh.zslab : Lz;
  if (zs > Lz) zs = Lz;
  p.zslab = (int)zs;
  const int64_t units = ((Lx + TX - 1) / TX) * ((Ly + TY - 1) / TY) * ((Lz + zs - 1) / zs);
  const int64_t grid_max = (int64_t)lat->sm_count * bps;
  const int grid = (int)(units < grid_max ? units : grid_max);
  void* args[] = {&p};
  PVSC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st));
  return PVSC_OK;
}

}  // namespace pvsc
