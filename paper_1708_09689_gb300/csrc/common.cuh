// Shared device/host definitions of the matrix-free Chebyshev stencil library.
//
// Everything here is written for sm_103a (GB300): 32-wide warps, 16-byte
// vector loads, warp shuffles and a fixed-order block reduction.  The two
// stencils are the topological-insulator Hamiltonian of Eq. TB_H_topi and the
// graphene Hamiltonian of Eq. graphene_model (Sec. 2 of Pieper, Hager and
// Fehske, arXiv 1708.09689).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pvsc {

constexpr int kMaxR = 64;
constexpr int kNumDots = 4;  // <x|x>, Re<y|x>, Im<y|x>, <y|y>

// ---------------------------------------------------------------- geometry
// Gate-defined quantum-dot array of Eq. qdotarray on the graphene lattice,
// regenerated inside the sweeps (v_mode 3): K x K dots of radius R on a square
// grid of spacing D = 4 R centred in the sample, dot (l, k) at physical
// (X_l, Y_k) with height V_k = V0 + dV |k - K/2|, and the step Theta smoothed
// to S(s) = (1 + tanh(s / w)) / 2, evaluated within rcut = R + 20 w of a dot
// centre (beyond it S < 4e-18).  Site positions in units of the C-C distance:
// X = 3 y + {0, 1/2, 3/2, 2}[nu], Y = sqrt(3) x + {sqrt(3)/2, 0, 0, sqrt(3)/2}[nu]
// for site nu of cell (x, y).  The dot centres are kept relative to a nearby
// cell row / column, X_l = 3 row[l] + ex[l] and Y_k = sqrt(3) col[k] + ey[k]
// with small residuals, so that X - X_l and Y - Y_k of the sites that matter
// are formed from small integers and keep their accuracy in fp32.
constexpr int kMaxQDots = 16;
// What the sweeps take as kernel parameters: the cell range test (dot (0, 0),
// cut-off, 1 / spacing) and the dot table (rows / columns with their
// residuals, heights), in fp32 and fp64.
struct QDScal {
  int K, row0, col0;
  float ex0f, ey0f, rcutf, invDf, Rf, inv_wf;
  double ex0, ey0, rcut, invD, R, w;
  int row[kMaxQDots], col[kMaxQDots];
  float exf[kMaxQDots], eyf[kMaxQDots], Vkf[kMaxQDots];
  double ex[kMaxQDots], ey[kMaxQDots], Vk[kMaxQDots];
};
struct QDots {
  QDScal s;
};

struct Geometry {
  int model;            // 1 TI, 2 graphene, 3 Weyl semimetal
  int per[3];           // periodic flags
  int64_t L[3];         // TI: Lx, Ly, Lz sites; graphene: Nx, Ny cells, 1
  int64_t n_sites;      // TI: Lx Ly Lz; graphene: 4 Nx Ny
  double t, m;          // hopping; TI mass, or for the Weyl semimetal 2 + cos k0
  const double* V;      // device [n_sites] when v_mode == 1
  const float* V32;     // the same potential rounded to fp32, for complex64 sweeps
  int v_mode;           // 0 zero, 1 stored, 2 regenerated from the hash, 3 quantum-dot array
  uint64_t vkey;        // mix(seed ^ stream*gamma) for stream 0
  double W;             // disorder width for v_mode 2
  double d1, d2;        // TI on-site Delta_1 Gamma^5 + Delta_2 Gamma^15 (Eq. TB_H_topi)
  float d1f, d2f;       // the same rounded to fp32, for complex64 sweeps
  int has_delta;        // d1 != 0 or d2 != 0
  int zhalo;            // TI: bit 0 a halo plane below, bit 1 above the updated planes
                        // (read as z-neighbours, never updated)
  const QDots* qd;      // v_mode 3 (graphene): device copy owned by the lattice
};

// Orbitals per site: 4 (TI), 1 (graphene site), 2 (Weyl semimetal).
__host__ __device__ __forceinline__ int orbitals_of(int model) {
  return model == 1 ? 4 : (model == 3 ? 2 : 1);
}

// Neighbour index along one axis: idx -/+ stride, wrapped on a periodic axis,
// -1 where an open axis ends.  A periodic axis of length 1 returns idx itself
// (the site is its own neighbour and both bond terms act on it).
__host__ __device__ __forceinline__ int64_t nbr_minus(int64_t idx, int64_t coord, int64_t L,
                                                      int per, int64_t stride) {
  return coord > 0 ? idx - stride : (per ? idx + (L - 1) * stride : -1);
}
__host__ __device__ __forceinline__ int64_t nbr_plus(int64_t idx, int64_t coord, int64_t L,
                                                     int per, int64_t stride) {
  return coord < L - 1 ? idx + stride : (per ? idx - (L - 1) * stride : -1);
}

// ---------------------------------------------------------------- index arithmetic
// Non-negative a / b with 32-bit unsigned division when both fit: the 64-bit
// division is a long instruction sequence that partly issues on the narrow
// fp64 pipe of this part.
__device__ __forceinline__ int64_t udiv64(int64_t a, int64_t b) {
  if (((uint64_t)a | (uint64_t)b) <= 0xffffffffull) return (int64_t)((uint32_t)a / (uint32_t)b);
  return a / b;
}

// SplitMix64 output finaliser (Steele, Lea & Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}
constexpr uint64_t kGoldenGamma = 0x9E3779B97F4A7C15ull;
__host__ __device__ __forceinline__ uint64_t hash_key(uint64_t seed, uint64_t stream) {
  return mix64(seed ^ (stream * kGoldenGamma));
}
// Uniform double in [0, 1) from the top 53 bits: exact conversion.
__host__ __device__ __forceinline__ double hash_uniform(uint64_t key, uint64_t idx) {
  return (double)(mix64(key + idx) >> 11) * 0x1.0p-53;
}

// Eq. qdotarray at the four sites of graphene cell (x, y), in the arithmetic
// type T.  One range test on the cell (its sites span [0, 2] in X and
// [0, sqrt(3)/2] in Y from the cell origin) finds the dot rows l and columns k
// that can lie within rcut; most cells have none and get zeros.  The dots
// (l, k) in range are then visited in order, the four sites together:
// V += V_k S with S = (1 + tanh((R - d) / w)) / 2 where d < rcut.  fp32 forms
// S as the equal 1 / (1 + exp(-2 (R - d) / w)).
template <typename T>
__device__ __forceinline__ void qd_cell_potentials(const QDScal& q, int64_t x, int64_t y, T (&V)[4]) {
  constexpr bool f = sizeof(T) == 4;
  const T s3 = T(1.7320508075688772), h3 = T(0.8660254037844386);
  const T rcut = f ? T(q.rcutf) : T(q.rcut), invD = f ? T(q.invDf) : T(q.invD);
  const T tx = T(3) * T(y - q.row0) - (f ? T(q.ex0f) : T(q.ex0));  // X - X_0 at the cell origin
  const T ty = s3 * T(x - q.col0) - (f ? T(q.ey0f) : T(q.ey0));    // Y - Y_0
  // conservative index ranges: floor / ceil leave one spare index per side
  const int l0 = max(0, (int)floor((tx - rcut) * invD));
  const int l1 = min(q.K - 1, (int)ceil((tx + T(2) + rcut) * invD));
  const int k0 = max(0, (int)floor((ty - rcut) * invD));
  const int k1 = min(q.K - 1, (int)ceil((ty + h3 + rcut) * invD));
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) V[nu] = T(0);
  if (l0 > l1 || k0 > k1) return;
  const T R = f ? T(q.Rf) : T(q.R);
  const T ox[4] = {T(0), T(0.5), T(1.5), T(2)}, oy[4] = {h3, T(0), T(0), h3};
  for (int l = l0; l <= l1; ++l) {
    const T dx0 = T(3) * T(y - q.row[l]) - (f ? T(q.exf[l]) : T(q.ex[l]));  // X - X_l at the origin
    if (!(dx0 + T(2) > -rcut && dx0 < rcut)) continue;
    for (int k = k0; k <= k1; ++k) {
      const T dy0 = s3 * T(x - q.col[k]) - (f ? T(q.eyf[k]) : T(q.ey[k]));
      if (!(dy0 + h3 > -rcut && dy0 < rcut)) continue;
      const T Vk = f ? T(q.Vkf[k]) : T(q.Vk[k]);
#pragma unroll
      for (int nu = 0; nu < 4; ++nu) {
        const T dx = dx0 + ox[nu], dy = dy0 + oy[nu];
        const T d = sqrt(fma(dx, dx, dy * dy));
        T S;
        if constexpr (f) S = 1.0f / (1.0f + __expf(-2.0f * (R - d) * q.inv_wf));
        else S = 0.5 * (1.0 + tanh((R - d) / q.w));
        if (d < rcut) V[nu] += Vk * S;
      }
    }
  }
}

// site -> (cell x, cell y, nu) of the graphene lattice
__device__ __forceinline__ void gr_site_coords(const Geometry& g, int64_t site, int64_t& x, int64_t& y,
                                               int& nu) {
  const int64_t c = site >> 2;
  nu = (int)(site & 3);
  y = udiv64(c, g.L[0]);
  x = c - y * g.L[0];
}

// Stored or hashed potential (the sweeps; the graphene sweep has its own
// instantiation for the quantum-dot array, so no other kernel carries that code).
__device__ __forceinline__ double site_potential(const Geometry& g, int64_t site) {
  if (g.v_mode == 1) return __ldg(g.V + site);
  if (g.v_mode == 2) return g.W * (hash_uniform(g.vkey, (uint64_t)site) - 0.5);
  return 0.0;
}

// Any potential mode, in fp64 (bounds, potential read-back).
__device__ __forceinline__ double site_potential_any(const Geometry& g, int64_t site) {
  if (g.v_mode == 3) {
    int64_t x, y;
    int nu;
    gr_site_coords(g, site, x, y, nu);
    double V[4];
    qd_cell_potentials<double>(g.qd->s, x, y, V);
    return V[nu];
  }
  return site_potential(g, site);
}

// The potential in the sweep's arithmetic type: complex64 sweeps read the fp32
// copy (the same rounding as converting the fp64 value, without a per-site
// conversion on GB300's narrow fp64 pipe and with half the bytes).
template <typename T>
__device__ __forceinline__ T site_potential_t(const Geometry& g, int64_t site) {
  if constexpr (sizeof(T) == 4) {
    if (g.v_mode == 1) return __ldg(g.V32 + site);
  }
  return T(site_potential(g, site));
}

// Random-phase entry exp(2 pi i u) scale (the KPM start vectors, u from the
// counter hash).  complex128 evaluates the phase in fp64; complex64 storage
// rounds to fp32 anyway, so the phase is evaluated in fp32 (sincospif) and
// stays off the narrow fp64 pipe.
template <typename T>
__device__ __forceinline__ void random_phase_entry(double u, double scale, T& re, T& im) {
  if constexpr (sizeof(T) == 8) {
    double s, c;
    sincospi(2.0 * u, &s, &c);
    re = c * scale;
    im = s * scale;
  } else {
    float s, c;
    sincospif((float)(2.0 * u), &s, &c);
    re = c * (float)scale;
    im = s * (float)scale;
  }
}

// ---------------------------------------------------------------- complex
template <typename T> struct CT;
template <> struct CT<double> { using c = double2; using v = double2; };  // one complex per 16 B
template <> struct CT<float>  { using c = float2;  using v = float4;  };  // two complex per 16 B

template <typename T> struct cplx { T re, im; };

template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }

// ---------------------------------------------------------------- sweep arguments
// One fused stencil sweep (see the sweep kernels):
//   y_new = alpha_r (H - beta_r) x + gamma_r y_in + sigma * src           (per vector r)
//   z    += delta_r y_new
//   acc   : init acc = cx x + cy y_new | add acc += cy y_new | final out = ph (acc + cy y_new)
//   grad[site] += gscale Re sum_{orbitals} conj(y_new) wg
//   dots  : <x|x>, Re/Im <y_new|x>, <y_new|y_new> per vector, fp64, fixed order
struct Sweep {
  Geometry g;
  int R;
  int C;                 // R / VPT vector chunks per site
  const void* x;
  const void* yin;       // may be null (gamma = 0)
  void* yout;            // may be null (final series step)
  void* yout2;           // two-step KPM sweep: w_{k+2} (yout holds w_{k+1})
  void* z;               // may be null
  double coef[4][kMaxR]; // alpha, beta, gamma, delta per vector
  // series accumulation (complex128 accumulator)
  int acc_mode;          // AccMode bits (below)
  int acc_kind;          // set at launch: bits 0-1 kind of cx, 2-3 of cy, 4-5 of cz (0 general, 1 real,
                         // 2 imaginary, 3 zero or no such term)
  double2* acc;
  double2* acc_out;      // final: written here
  double cx_re, cx_im, cy_re, cy_im, ph_re, ph_im;
  double cz_re, cz_im;   // weight of y_in (ACC_YIN)
  float fc[3][2][2];     // set at launch: [cx, cy, cz][re, im][hi, lo], value = hi + lo in fp32
  // adjoint source and gradient
  const double2* src;    // y_new += sigma * src (complex128)
  double sg_re, sg_im;
  const void* wg;        // grad partner vector (same precision as x)
  double* grad;          // [n_sites] fp64
  double gscale;
  // dot products
  int dot_flags;         // bit0 xx, bit1 xy, bit2 yy
  int dot_mode;          // 0 write dots[4][R]; 1 KPM first step; 2 KPM step k; 3 KPM steps k, k+1
  double* partials;      // [gridDim][4][R]
  unsigned* counter;     // zero before the first sweep; reset by the last block
  double* dots;          // [4][R]
  double* mu;            // [R][M]
  int M;
  int kpm_k;
  // fixed-point KPM sweep (sweep_fx.cu)
  const void* fx_d;      // per site (d_+, d_-) in Q3.60 for alpha = 1/a
  long long fx_kt;       // -alpha t / 2 in Q3.60
  int fx_dshift;         // 1: alpha = 2/a (d doubled)
  const double* vscale;  // per vector: value of one unit of a dot product
  int zslab;             // TI z-marching depth
  int tile_x, tile_y;    // TI shared-memory staged sweep: tile of columns (0: register marching)
  QDScal qds;            // graphene quantum-dot array (g.v_mode 3): range-test scalars
};

// acc_new = [INIT ? 0 : acc] + [YIN ? cz y_in : 0] + [X ? cx x : 0] + cy y_new,
// with x the sweep's input, or under XSRC the complex128 vector src, and y_in
// its value before the sweep (the series writes y_new over it); FINAL writes
// ph acc_new to acc_out instead of acc.  YIN comes with X, and with neither
// INIT nor XSRC.
enum AccMode { ACC_NONE = 0, ACC_INIT = 1, ACC_ADD = 2, ACC_FINAL = 4, ACC_X = 8, ACC_XSRC = 16, ACC_YIN = 32 };

// ---------------------------------------------------------------- deterministic dot reduction
// acc[d][v]: per-thread fp64 partial sums of dot d for vector rc*VPT+v.  Every
// block reduces them in a fixed order (warp xor tree, then warps in index
// order) to one value per (d, r), writes its row of `partials`, and the last
// block to arrive sums the rows in block order and writes the outputs.  The
// result is bitwise reproducible for a given launch configuration.
constexpr int kMaxThreads = 256;

// After every block has written its row of `partials`: the last block to
// arrive sums the rows in block order and writes the outputs of dot_mode.
__device__ __forceinline__ void finish_dots(const Sweep& p) {
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(p.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nb = gridDim.x;
  for (int q = warp; q < kNumDots * p.R; q += nwarps) {
    const int d = q / p.R, r = q % p.R;
    if (!((p.dot_flags >> (d == 0 ? 0 : (d == 3 ? 2 : 1))) & 1)) continue;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += __ldcg(p.partials + (size_t)b * kNumDots * p.R + q);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
      double* mu = p.mu + (size_t)r * p.M;
      if (p.dot_mode == 0) {
        p.dots[q] = s;
      } else if (p.dot_mode == 1) {  // KPM step 0: mu_0 = <w0|w0>, mu_1 = Re<w1|w0>
        if (d == 0) mu[0] = s;
        if (d == 1 && p.M > 1) mu[1] = s;
      } else if (p.dot_mode == 2) {  // KPM step k: mu_2k = 2<wk|wk> - mu_0, mu_2k+1 = 2 Re<wk+1|wk> - mu_1
        const int k = p.kpm_k;
        if (d == 0 && 2 * k < p.M) mu[2 * k] = 2.0 * s - __ldcg(mu);
        if (d == 1 && 2 * k + 1 < p.M) mu[2 * k + 1] = 2.0 * s - __ldcg(mu + 1);
      } else {  // KPM steps k and k+1 in one sweep: dots <wk|wk>, Re<wk+1|wk>,
                // <wk+1|wk+1>, Re<wk+2|wk+1> give mu_2k .. mu_2k+3
        const int m = 2 * p.kpm_k + d;
        if (m < p.M) mu[m] = 2.0 * s - __ldcg(mu + (d & 1));
      }
    }
  }
  if (threadIdx.x == 0) *p.counter = 0u;
}

template <int VPT, int MAXW = kMaxThreads / 32>
__device__ void reduce_dots(const Sweep& p, double (&acc)[kNumDots][VPT]) {
  __shared__ double sm[MAXW][kNumDots][VPT][32];  // [warp][dot][v][lane]
  const int C = p.C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int d = 0; d < kNumDots; ++d)
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      double s = acc[d][v];
      for (int off = 16; off >= C; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane < C) sm[warp][d][v][lane] = s;
    }
  __syncthreads();
  double* row = p.partials + (size_t)blockIdx.x * kNumDots * p.R;
  for (int t = threadIdx.x; t < C; t += blockDim.x) {
    const int stride = C < 32 ? 1 : C / 32;  // warps that carry chunk t
    const int w0 = C < 32 ? 0 : t / 32;
    const int l = C < 32 ? t : t % 32;
    for (int d = 0; d < kNumDots; ++d)
      for (int v = 0; v < VPT; ++v) {
        double s = 0.0;
        for (int w = w0; w < nwarps; w += stride) s += sm[w][d][v][l];
        row[d * p.R + t * VPT + v] = s;
      }
  }
  finish_dots(p);
}


}  // namespace pvsc
