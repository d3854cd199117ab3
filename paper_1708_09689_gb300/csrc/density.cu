// Spectral densities from KPM moments: the density of states (Eq. DOS) and
// the momentum-resolved spectral function A(k, E) (Eq. ak), Sec. 2.2, with the
// damping kernels of the kernel polynomial method the paper cites (Weisse,
// Wellein, Alvermann, Fehske, Rev. Mod. Phys. 78, 275 (2006), Sec. II), and
// the Bloch start states psi(k, nu) of Eq. ak.
#include <cmath>

#include "internal.h"

namespace pvsc {

// Damping factor g_k of M moments: 0 none, 1 Jackson, 2 Lorentz(lambda).
__device__ __forceinline__ double damping(int kernel, int k, int M, double lambda) {
  if (kernel == PVSC_KERNEL_JACKSON) {
    const double q = M_PI / (M + 1);
    double s, c;
    sincos(q * k, &s, &c);
    return ((M - k + 1) * c + s * (cos(q) / sin(q))) / (M + 1);
  }
  if (kernel == PVSC_KERNEL_LORENTZ) return sinh(lambda * (1.0 - (double)k / M)) / sinh(lambda);
  return 1.0;
}

constexpr int kDensityChunk = 1024;  // series coefficients staged in shared memory per pass

// rho(E_j) = scale sum_r [g_0 mu_0^r + 2 sum_{k>=1} g_k mu_k^r T_k(x_j)] / (pi a sqrt(1 - x_j^2)),
// x_j = (E_j - b)/a, rho = 0 for |x_j| >= 1.  One thread per energy; the block
// forms the coefficients c_k = g_k sum_r mu_k^r chunk by chunk in shared
// memory and every thread runs the Chebyshev recurrence T_{k+1} = 2 x T_k - T_{k-1}
// through them.
__global__ void __launch_bounds__(256) kpm_density_kernel(int R, int M, const double* __restrict__ mu,
                                                          int kernel, double lambda, double a, double b,
                                                          double scale, int NE,
                                                          const double* __restrict__ E,
                                                          double* __restrict__ rho) {
  __shared__ double c[kDensityChunk];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const double x = j < NE ? (E[j] - b) / a : 2.0;
  const bool inside = fabs(x) < 1.0;
  double Tm = 0.0, T = 1.0;  // T_{k-1}, T_k (k = 0: T_{-1} unused)
  double sum = 0.0;
  for (int k0 = 0; k0 < M; k0 += kDensityChunk) {
    const int n = min(kDensityChunk, M - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int k = k0 + i;
      double s = 0.0;
      for (int r = 0; r < R; ++r) s += mu[(size_t)r * M + k];
      c[i] = (k == 0 ? 1.0 : 2.0) * damping(kernel, k, M, lambda) * s;
    }
    __syncthreads();
    if (inside) {
      for (int i = 0; i < n; ++i) {
        const int k = k0 + i;
        sum = fma(c[i], T, sum);
        const double Tn = k == 0 ? x : 2.0 * x * T - Tm;
        Tm = T;
        T = Tn;
      }
    }
  }
  if (j < NE) rho[j] = inside ? scale * sum / (M_PI * a * sqrt(1.0 - x * x)) : 0.0;
}

// psi(k_q, nu) for nk k-points on a lattice of O orbitals per site (TI 4,
// Weyl semimetal 2): vector r = O q + nu holds exp(i k_q . r_n)/sqrt(N) on
// orbital nu of every site n, zero elsewhere.  Phases in fp64 (k.r reaches
// thousands of radians), rounded to the storage type.
struct KPoints {
  double k[16][3];
};

template <typename T>
__global__ void bloch_kernel(const Geometry g, int O, int R, const KPoints kp, T* out) {
  const int64_t n = O * g.n_sites * (int64_t)R;  // complex elements
  const double inv = 1.0 / sqrt((double)g.n_sites);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = udiv64(e, R);  // site * O + orbital
    const int r = (int)(e - i * R);
    const int64_t s = i / O;
    const int o = (int)(i - s * O);
    double re = 0.0, im = 0.0;
    if (r % O == o) {
      const int q = r / O;
      const int64_t yz = udiv64(s, g.L[0]);
      const int64_t x = s - yz * g.L[0];
      const int64_t z = udiv64(yz, g.L[1]);
      const int64_t y = yz - z * g.L[1];
      const double ph = kp.k[q][0] * (double)x + kp.k[q][1] * (double)y + kp.k[q][2] * (double)z;
      double sn, cs;
      sincos(ph, &sn, &cs);
      re = cs * inv;
      im = sn * inv;
    }
    out[2 * e] = T(re);
    out[2 * e + 1] = T(im);
  }
}

static int launch_kpm_density(int R, int M, const double* mu, int kernel, double lambda, double a,
                       double b, double scale, int NE, const double* E, double* rho,
                       cudaStream_t st) {
  const int threads = 256;
  const int grid = (NE + threads - 1) / threads;
  kpm_density_kernel<<<grid, threads, 0, st>>>(R, M, mu, kernel, lambda, a, b, scale, NE, E, rho);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

static int launch_bloch(const Geometry& g, int O, int R, int prec, const KPoints& kp, void* out,
                        cudaStream_t st) {
  const int64_t n = O * g.n_sites * (int64_t)R;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  if (prec == PVSC_C128)
    bloch_kernel<double><<<(int)blocks, 256, 0, st>>>(g, O, R, kp, static_cast<double*>(out));
  else
    bloch_kernel<float><<<(int)blocks, 256, 0, st>>>(g, O, R, kp, static_cast<float*>(out));
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

}  // namespace pvsc

using namespace pvsc;

extern "C" {

int pvsc_kpm_density(int R, int M, const double* mu, int kernel, double lambda, double a, double b,
                     double scale, int NE, const double* E, double* rho, void* stream) {
  if (R < 1 || M < 1 || NE < 0) return set_error(PVSC_ERR_ARG, "need R >= 1, M >= 1, NE >= 0");
  if (kernel != PVSC_KERNEL_NONE && kernel != PVSC_KERNEL_JACKSON && kernel != PVSC_KERNEL_LORENTZ)
    return set_error(PVSC_ERR_ARG, "unknown damping kernel %d", kernel);
  if (kernel == PVSC_KERNEL_LORENTZ && !(std::isfinite(lambda) && lambda > 0))
    return set_error(PVSC_ERR_ARG, "the Lorentz kernel needs lambda > 0");
  if (!(std::isfinite(a) && a > 0) || !std::isfinite(b) || !std::isfinite(scale))
    return set_error(PVSC_ERR_ARG, "need a > 0 and finite b, scale");
  if (NE == 0) return PVSC_OK;
  if (int rc = check_ptr(mu, "mu")) return rc;
  if (int rc = check_ptr(E, "E")) return rc;
  if (int rc = check_ptr(rho, "rho")) return rc;
  return launch_kpm_density(R, M, mu, kernel, lambda, a, b, scale, NE, E, rho,
                            static_cast<cudaStream_t>(stream));
}

int pvsc_bloch_vectors(const pvsc_lattice* lat, int nk, const double* k, int prec, void* out,
                       void* stream) {
  if (int rc = check_lattice(lat)) return rc;
  if (lat->g.model == PVSC_GRAPHENE)
    return set_error(PVSC_ERR_UNSUPPORTED, "Bloch states are built for the cubic lattices (TI, Weyl semimetal)");
  const int O = orbitals_of(lat->g.model);
  if (!valid_R(O * nk) || nk > 16)
    return set_error(PVSC_ERR_ARG, "nk = %d: %d nk must be a block width 1 .. 64", nk, O);
  if (prec != PVSC_C128 && prec != PVSC_C64) return set_error(PVSC_ERR_ARG, "unknown precision %d", prec);
  if (!k) return set_error(PVSC_ERR_ARG, "k is NULL");
  for (int i = 0; i < 3 * nk; ++i)
    if (!std::isfinite(k[i])) return set_error(PVSC_ERR_ARG, "k[%d] is not finite", i);
  if (int rc = check_ptr(out, "out")) return rc;
  KPoints kp{};  // passed by value in the kernel parameters
  for (int q = 0; q < nk; ++q)
    for (int d = 0; d < 3; ++d) kp.k[q][d] = k[3 * q + d];
  return launch_bloch(lat->g, O, O * nk, prec, kp, out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
