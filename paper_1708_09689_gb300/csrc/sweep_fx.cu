// KPM moments of the TI Hamiltonian (Eq. TB_H_topi) with complex128-sized
// storage and exact integer arithmetic: the recurrence vectors are held as
// pairs of 64-bit fixed-point numbers instead of fp64.
//
// Why: on this part the fp64 pipe issues at 1/64 of the fp32 rate, and the
// fp64 stencil needs ~150 fp64 instructions per lattice update, so it runs
// at the fp64 roof, a tenth of the HBM roof.  The stencil is almost entirely
// additions (neighbour sums and the signed permutations of the Gamma
// matrices), which are exact on integers; the wide integer pipes do them.
//
// Format: a vector value v is the integer round(v 2^59 / 2^e_r) (Q4.59 after
// an exact power-of-two scaling 2^-e_r per vector r chosen so that the start
// vector has 2-norm <= 1).  With (a, b) from an interval that holds the
// spectrum, ||T_k(H~)|| <= 1, so every |w_k| <= 1, the stencil's neighbour
// combinations are <= 6 and the three-term update stays < 16 (no overflow).
// The coefficients d_o = (V_n - b)/a +- m/a and kt = -t/(2a) of the sweep are
// Q3.60; every output is d x + kt T, formed exactly and rounded once (2^-60,
// round half up), then - y_in added exactly.  The dot products are exact sums
// of the exact products per thread, converted to fp64 once per column segment
// and reduced in fp64 in a fixed order as in the other sweeps.  Products and
// sums are assembled from 32 x 32 -> 64-bit limb products (fx_arith.cuh).
#include "internal.h"
#include "fx_arith.cuh"
#include "sweep.cuh"

namespace pvsc {

// One KPM sweep on fixed-point vectors, z-marching as the floating-point
// sweeps (ti_march): y = alpha (H - b) x, minus y_in when given (gamma = -1),
// and the partial sums of <x|x> and Re<y|x>.  Sweep fields: x, yin, yout (i64
// pairs; yin and yout may be the same buffer), fx_d (per site (d_+, d_-) for
// alpha = 1/a, Q3.60), fx_dshift (1 when alpha = 2/a), fx_kt (Q3.60), vscale
// (per vector: 4^e_r 2^-118, the value of one unit of a dot).  DEPTH/NBUF: the
// cp.async prefetch ring of ti_march (DEPTH = 0: plain loads).
template <int DEPTH, int NBUF>
__global__ void __launch_bounds__(256) ti_sweep_fx(const __grid_constant__ Sweep p) {
  extern __shared__ __align__(16) unsigned char ring[];
  const int64_t plane = p.g.L[0] * p.g.L[1], Lz = p.g.L[2];
  const int R = p.R, C = p.R;  // one vector per thread
  const int rc = threadIdx.x % C;
  const int cshift = __ffs(C) - 1;  // R is a power of two
  const i64* __restrict__ X = static_cast<const i64*>(p.x);
  const i64* Yin = static_cast<const i64*>(p.yin);
  i64* Yout = static_cast<i64*>(p.yout);
  const longlong2* __restrict__ dfx = static_cast<const longlong2*>(p.fx_d);
  const FxLimbs kt = fx_split(p.fx_kt);
  const int dshift = p.fx_dshift ? 1 : 0;  // alpha = 2/a: coefficients doubled
  const double vs = p.vscale[rc];
  double dd[kNumDots][1];
#pragma unroll
  for (int k = 0; k < kNumDots; ++k) dd[k][0] = 0.0;

  const int64_t ncolthr = plane * C;
  const int64_t nbx = (ncolthr + blockDim.x - 1) / blockDim.x;
  const int zs = p.zslab;
  const int64_t nunits = nbx * ((Lz + zs - 1) / zs);
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t bz = udiv64(u, nbx), bx = u - bz * nbx;
    const int64_t tid = bx * blockDim.x + threadIdx.x;
    if (tid >= ncolthr) continue;
    const int64_t z0 = bz * zs, z1 = min(z0 + (int64_t)zs, Lz);
    FxAcc xx, xy;
    fx_acc_zero(xx);
    fx_acc_zero(xy);
    ti_march<i64, 1, true, DEPTH, NBUF>(
        p.g, X, Yin, R, rc, tid >> cshift, z0, z1, ring,
        [&](int64_t s) { return __ldg(dfx + s); },
        [&](const longlong2 dv, const Blk<i64, 1>& xm, const Blk<i64, 1>& xc, const Blk<i64, 1>& xp,
            const Blk<i64, 1>& ax, const Blk<i64, 1>& bx, const Blk<i64, 1>& ay, const Blk<i64, 1>& by,
            const Blk<i64, 1>* yi, Blk<i64, 1>& yn) {
          Blk<i64, 1> T;
          fx_axis_T<0, true>(xm, xp, T);
          fx_axis_T<1, false>(ax, bx, T);
          fx_axis_T<2, false>(ay, by, T);
          const FxLimbs dp = fx_split((i64)((u64)dv.x << dshift)), dm = fx_split((i64)((u64)dv.y << dshift));
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const FxLimbs d = (o & 1) ? dm : dp;
            i64 re = fx_mul2(d, fx_split(xc.v[o][0].re), kt, fx_split(T.v[o][0].re));
            i64 im = fx_mul2(d, fx_split(xc.v[o][0].im), kt, fx_split(T.v[o][0].im));
            if (yi != nullptr) {
              re -= yi->v[o][0].re;
              im -= yi->v[o][0].im;
            }
            yn.v[o][0] = {re, im};
          }
        },
        [&](int64_t s, const Blk<i64, 1>& xc, Blk<i64, 1>& yn) {
          store_blk<i64, 1>(Yout, s, R, rc, yn);
          FxLimbs xs[8], ys[8];
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            xs[2 * o] = fx_split(xc.v[o][0].re);
            xs[2 * o + 1] = fx_split(xc.v[o][0].im);
            ys[2 * o] = fx_split(yn.v[o][0].re);
            ys[2 * o + 1] = fx_split(yn.v[o][0].im);
          }
          fx_dot_item(xs, ys, xx, xy);
        });
    dd[0][0] += fx_acc_value(xx, vs);
    dd[1][0] += fx_acc_value(xy, vs);
  }
  reduce_dots<1>(p, dd);
}

// Per-block partial sums of |x|^2 for each vector of a complex128 block
// (n = D R elements; the thread's vector is fixed because blockDim and the
// grid stride are multiples of R).  part[blockIdx][r].
__global__ void fx_norm_partials(const double2* __restrict__ x, int64_t n, int R, double* part) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[e];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < R) {
    double t = 0.0;
    for (int i = threadIdx.x; i < blockDim.x; i += R) t += sm[i];
    part[(size_t)blockIdx.x * R + threadIdx.x] = t;
  }
}

// Exponent e_r with ||r||^2 <= 4^e_r, the conversion factor 2^(59 - e_r)
// and the dot unit 4^e_r 2^-118 (one thread per vector, blocks summed in order).
__global__ void fx_norm_scale(const double* __restrict__ part, int nb, int R, double* xscale,
                              double* vscale) {
  const int r = threadIdx.x;
  if (r >= R) return;
  double n2 = 0.0;
  for (int b = 0; b < nb; ++b) n2 += part[(size_t)b * R + r];
  int e = 0;
  if (n2 > 0.0) {
    int ex;
    frexp(n2, &ex);  // n2 = f 2^ex, f in [0.5, 1): n2 <= 2^ex
    e = (ex + 1) >> 1;  // ceil(ex / 2) for any sign
  }
  xscale[r] = ldexp(1.0, kFxVal - e);
  vscale[r] = ldexp(1.0, 2 * e - 2 * kFxVal);
}

// complex128 -> Q4.59 pairs with the per-vector factor (may run in place).
__global__ void fx_from_c128(const double2* in, longlong2* out, int64_t n, int R,
                             const double* __restrict__ xscale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double f = xscale[e & (R - 1)];  // R is a power of two
    const double2 v = in[e];
    out[e] = make_longlong2(__double2ll_rn(v.x * f), __double2ll_rn(v.y * f));
  }
}

// Per site (d_+, d_-) = ((V_n - b)/a + m/a, (V_n - b)/a - m/a) in Q3.60.
__global__ void fx_site_coefs(const Geometry g, double inv_a, double b, longlong2* dfx) {
  const double am = g.m * inv_a;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.n_sites;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double e = (site_potential(g, s) - b) * inv_a;
    dfx[s] = make_longlong2(__double2ll_rn(ldexp(e + am, kFxCoef)), __double2ll_rn(ldexp(e - am, kFxCoef)));
  }
}

// ---------------------------------------------------------------- host side
FxLayout fx_layout(const pvsc_lattice* lat, int R) {
  FxLayout L;
  const int nb = 2 * lat->sm_count;
  L.nb = nb;
  L.part = (dots_work_bytes(lat, R) + 255) & ~size_t(255);
  L.xscale = L.part + ((sizeof(double) * nb * R + 255) & ~size_t(255));
  L.vscale = L.xscale + 512;
  L.dfx = L.vscale + 512;
  L.wa = L.dfx + (((size_t)lat->g.n_sites * 16 + 255) & ~size_t(255));
  L.wb = L.wa + vec_bytes(lat, R, PVSC_C128);
  L.total = L.wb + vec_bytes(lat, R, PVSC_C128);
  return L;
}

int launch_fx_prepare(const pvsc_lattice* lat, int R, const void* r0, uint64_t seed, double a,
                      double b, void* work, const FxLayout& L, cudaStream_t st) {
  char* w = static_cast<char*>(work);
  const int64_t D = lat->g.n_sites * 4;
  const int64_t n = D * R;
  double2* wa = reinterpret_cast<double2*>(w + L.wa);
  if (r0) {
    PVSC_CUDA_TRY(cudaMemcpyAsync(wa, r0, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
  } else {
    if (int rc = launch_random_phase(wa, PVSC_C128, D, R, seed, st)) return rc;
  }
  double* part = reinterpret_cast<double*>(w + L.part);
  double* xscale = reinterpret_cast<double*>(w + L.xscale);
  double* vscale = reinterpret_cast<double*>(w + L.vscale);
  fx_norm_partials<<<L.nb, 256, 0, st>>>(wa, n, R, part);
  PVSC_CUDA_TRY(cudaGetLastError());
  fx_norm_scale<<<1, 64, 0, st>>>(part, L.nb, R, xscale, vscale);
  PVSC_CUDA_TRY(cudaGetLastError());
  fx_from_c128<<<L.nb * 4, 256, 0, st>>>(wa, reinterpret_cast<longlong2*>(wa), n, R, xscale);
  PVSC_CUDA_TRY(cudaGetLastError());
  fx_site_coefs<<<L.nb * 2, 256, 0, st>>>(lat->g, 1.0 / a, b, reinterpret_cast<longlong2*>(w + L.dfx));
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

// kernel 0: plain loads; 2: cp.async ring of all six blocks one plane ahead;
// 3: ring of the two HBM streams three planes ahead (the TI tuning kernels)
static void* fx_kernel(int kernel) {
  if (kernel == 2) return reinterpret_cast<void*>(&ti_sweep_fx<kAsyncDepth, 6>);
  if (kernel == 3) return reinterpret_cast<void*>(&ti_sweep_fx<kAsyncDeepDepth, 2>);
  return reinterpret_cast<void*>(&ti_sweep_fx<0, 2>);
}

int launch_sweep_fx(const pvsc_lattice* lat, Sweep& p, const LaunchShape& sh, bool tuned,
                    cudaStream_t st) {
  // untuned (measured on the 256 x 256 x 64 slab): the TMA-staged tiles, on 16
  // warps for R = 2 .. 8 and on 8 for R = 1 and the slices of R = 16, 32 (0.61
  // to 0.79 of the HBM roof, against 0.30 to 0.53 for the cp.async ring); the
  // six-block ring for R = 64
  if (!tuned && tma_fx_possible(lat, p.R)) {
    LaunchShape d;
    d.threads = p.R >= 2 && p.R <= 8 ? 512 : 256;
    return launch_sweep_tma_fx(lat, p, d, st);
  }
  const int kernel = tuned ? sh.kernel : (p.R >= 2 ? 2 : 0);
  if (kernel == kKernelTma) return launch_sweep_tma_fx(lat, p, sh, st);
  int threads = tuned ? sh.threads : 128;
  if (threads < 32 || threads > kMaxThreads || threads % 32 || threads % p.R) threads = 128;
  void* fn = fx_kernel(kernel);
  const size_t smem = kernel == 2 ? async_ring_bytes(kModelTIAsync, threads)
                      : kernel == 3 ? async_ring_bytes(kModelTIAsyncDeep, threads) : 0;
  if (smem)
    if (int rc = allow_max_smem(fn)) return rc;
  int occ = 0;
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem));
  if (occ < 1) occ = 1;
  int bps = tuned && sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ ? sh.blocks_per_sm : occ;
  const int64_t grid_max = (int64_t)lat->sm_count * bps;
  const int64_t plane = lat->g.L[0] * lat->g.L[1], Lz = lat->g.L[2];
  const int64_t nbx = (plane * p.R + threads - 1) / threads;
  int64_t zs = tuned ? sh.zslab : 0;
  if (zs <= 0) {
    int64_t nz = (6 * grid_max + nbx - 1) / nbx;
    if (nz < 1) nz = 1;
    if (nz > Lz) nz = Lz;
    zs = (Lz + nz - 1) / nz;
  }
  if (zs > Lz) zs = Lz;
  p.zslab = (int)zs;
  const int64_t units = nbx * ((Lz + zs - 1) / zs);
  const int grid = (int)(units < grid_max ? units : grid_max);
  void* args[] = {&p};
  PVSC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st));
  return PVSC_OK;
}

// ---------------------------------------------------------------- arithmetic checks
// The limb routines of fx_arith.cuh on caller-given operands (pvsc_debug_fx_arith).
__global__ void fx_debug_mul2(const i64* __restrict__ in, int64_t n, i64* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const i64* r = in + 4 * i;
    out[i] = fx_mul2(fx_split(r[0]), fx_split(r[1]), fx_split(r[2]), fx_split(r[3]));
  }
}

// one thread: the exact sums over all records, as the sweep accumulates them
__global__ void fx_debug_dots(const i64* __restrict__ in, int64_t n, i64* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  FxAcc xx, xy;
  fx_acc_zero(xx);
  fx_acc_zero(xy);
  for (int64_t i = 0; i < n; ++i) {
    FxLimbs xs[8], ys[8];
    for (int k = 0; k < 8; ++k) {
      xs[k] = fx_split(in[16 * i + k]);
      ys[k] = fx_split(in[16 * i + 8 + k]);
    }
    fx_dot_item(xs, ys, xx, xy);
  }
  fx_acc_add_shl<62>(xx, xx.u);
  fx_acc_add_shl<62>(xy, xy.u);
  out[0] = xx.hi;
  out[1] = (i64)xx.lo;
  out[2] = xy.hi;
  out[3] = (i64)xy.lo;
}

}  // namespace pvsc

using namespace pvsc;

extern "C" {

int pvsc_debug_fx_arith(int op, const int64_t* in, int64_t n, int64_t* out, void* stream) {
  if (op != 0 && op != 1) return set_error(PVSC_ERR_ARG, "op = %d: must be 0 (update) or 1 (dot sums)", op);
  if (n < 0) return set_error(PVSC_ERR_ARG, "n = %lld < 0", (long long)n);
  if (int rc = check_ptr(out, "out")) return rc;
  if (n > 0)
    if (int rc = check_ptr(in, "in")) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const i64* src = reinterpret_cast<const i64*>(in);
  i64* dst = reinterpret_cast<i64*>(out);
  if (op == 0) {
    if (n == 0) return PVSC_OK;
    const int64_t blocks = (n + 255) / 256;
    fx_debug_mul2<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(src, n, dst);
  } else {
    fx_debug_dots<<<1, 32, 0, st>>>(src, n, dst);
  }
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

}  // extern "C"
