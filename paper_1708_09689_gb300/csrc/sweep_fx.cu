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
// sums are <= 12 and the three-term update stays < 16 (no overflow).  The
// coefficients d_o = (V_n - b)/a +- m/a and kt = -t/(2a) of the sweep are
// Q3.60; every output is d x + kt T summed exactly in 128 bits and rounded
// once (2^-60, round half up), then - y_in added exactly.  The dot products
// are exact 128-bit sums of 128-bit products per thread, converted to fp64
// once per column segment and reduced in fp64 in a fixed order as in the
// other sweeps.
#include "internal.h"
#include "sweep.cuh"

namespace pvsc {

using i64 = long long;

constexpr int kFxVal = 59;   // fraction bits of vector values
constexpr int kFxCoef = 60;  // fraction bits of coefficients

// 128-bit two's-complement values as (hi, lo) pairs, built from the signed
// 64 x 64 -> 128 product (mul.hi.s64 and the wrapping low product).
struct W128 {
  i64 hi;
  unsigned long long lo;
};

__device__ __forceinline__ W128 wmul(i64 a, i64 b) {
  return W128{__mul64hi(a, b), (unsigned long long)a * (unsigned long long)b};
}

__device__ __forceinline__ void wadd(W128& acc, const W128& v) {
  const unsigned long long lo = acc.lo + v.lo;
  acc.hi += v.hi + (lo < acc.lo ? 1 : 0);
  acc.lo = lo;
}

// round((c1 x1 + c2 x2) 2^-60): Q3.60 x Q4.59 -> Q4.59 (round half up)
__device__ __forceinline__ i64 fx_mul2(i64 c1, i64 x1, i64 c2, i64 x2) {
  W128 P = wmul(c1, x1);
  wadd(P, wmul(c2, x2));
  wadd(P, W128{0, 1ull << (kFxCoef - 1)});
  return (i64)(((unsigned long long)P.hi << (64 - kFxCoef)) | (P.lo >> kFxCoef));
}

__device__ __forceinline__ double w128_to_double(const W128& v) {
  return fma((double)v.hi, 0x1p64, (double)v.lo);
}

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
  const i64 kt = p.fx_kt;
  const i64 dmul = p.fx_dshift ? 2 : 1;
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
    W128 xx{0, 0}, xy{0, 0};
    ti_march<i64, 1, true, DEPTH, NBUF>(
        p.g, X, Yin, R, rc, tid >> cshift, z0, z1, ring,
        [&](int64_t s) { return __ldg(dfx + s); },
        [&](const longlong2 dv, const Blk<i64, 1>& xm, const Blk<i64, 1>& xc, const Blk<i64, 1>& xp,
            const Blk<i64, 1>& ax, const Blk<i64, 1>& bx, const Blk<i64, 1>& ay, const Blk<i64, 1>& by,
            const Blk<i64, 1>* yi, Blk<i64, 1>& yn) {
          Blk<i64, 1> S, D;
          ti_axes(xm, xp, ax, bx, ay, by, S, D);
          const i64 dp = dv.x * dmul, dm = dv.y * dmul;
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const i64 d = (o & 1) ? dm : dp;
            const cplx<i64> T = (o & 1) ? csub(D.v[o][0], S.v[o][0]) : cadd(D.v[o][0], S.v[o][0]);
            i64 re = fx_mul2(d, xc.v[o][0].re, kt, T.re);
            i64 im = fx_mul2(d, xc.v[o][0].im, kt, T.im);
            if (yi != nullptr) {
              re -= yi->v[o][0].re;
              im -= yi->v[o][0].im;
            }
            yn.v[o][0] = {re, im};
          }
        },
        [&](int64_t s, const Blk<i64, 1>& xc, Blk<i64, 1>& yn) {
          store_blk<i64, 1>(Yout, s, R, rc, yn);
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const cplx<i64> a = xc.v[o][0], b = yn.v[o][0];
            wadd(xx, wmul(a.re, a.re));
            wadd(xx, wmul(a.im, a.im));
            wadd(xy, wmul(b.re, a.re));
            wadd(xy, wmul(b.im, a.im));
          }
        });
    dd[0][0] += w128_to_double(xx) * vs;
    dd[1][0] += w128_to_double(xy) * vs;
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
  // untuned: the six-block ring for R >= 2, plain loads for R = 1 (measured)
  const int kernel = tuned ? sh.kernel : (p.R >= 2 ? 2 : 0);
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

}  // namespace pvsc
