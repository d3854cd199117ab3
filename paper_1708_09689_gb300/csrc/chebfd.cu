// Chebyshev filter diagonalization (ChebFD, Sec. 5.3 "Interior eigenvalues":
// the scheme of A. Pieper et al., J. Comput. Phys. 325, 226 (2016)).
//
// One block of n_s <= 64 search vectors (complex128, the library's block
// layout).  Each iteration: filter the block with the Jackson-damped
// Chebyshev series of the indicator of the target interval (pvsc_cheb_filter,
// the stencil sweeps), orthonormalize it (shifted CholeskyQR3: Gram matrices
// by cuBLAS, Cholesky factors on the host), Rayleigh-Ritz (H Q by the stencil,
// the projected n_s x n_s matrix by cuBLAS, its eigen-decomposition by cyclic
// Jacobi on the host), rotate to the Ritz vectors (cuBLAS) and take every
// residual ||H x - theta x|| in one fused sweep (pvsc_cheb_step with
// beta_r = theta_r and the <y|y> dot).
//
// Layout: a (D x n) block stored element (i, r) at i n + r is, column-major,
// the n x D matrix A = Y^T with leading dimension n; the products below are
// written for that view (G = Y^H Y = conj(A A^H) and so on).
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace pvsc {
namespace dense {

using cd = std::complex<double>;

// A = L L^H for a Hermitian positive definite n x n column-major A; L
// overwrites the lower triangle (upper set to 0).  False if a pivot is not
// positive.
static bool cholesky(int n, std::vector<cd>& A) {
  for (int j = 0; j < n; ++j) {
    double d = A[j + j * n].real();
    for (int k = 0; k < j; ++k) d -= std::norm(A[j + k * n]);
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    A[j + j * n] = ljj;
    for (int i = j + 1; i < n; ++i) {
      cd s = A[i + j * n];
      for (int k = 0; k < j; ++k) s -= A[i + k * n] * std::conj(A[j + k * n]);
      A[i + j * n] = s / ljj;
    }
    for (int i = 0; i < j; ++i) A[i + j * n] = 0.0;
  }
  return true;
}

// Inverse of a lower-triangular n x n column-major L (forward substitution per column).
static std::vector<cd> lower_inverse(int n, const std::vector<cd>& L) {
  std::vector<cd> X(n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    X[c + c * n] = 1.0 / L[c + c * n];
    for (int i = c + 1; i < n; ++i) {
      cd s = 0.0;
      for (int k = c; k < i; ++k) s += L[i + k * n] * X[k + c * n];
      X[i + c * n] = -s / L[i + i * n];
    }
  }
  return X;
}

// Eigen-decomposition A = V diag(w) V^H of a Hermitian n x n column-major A
// by cyclic Jacobi rotations: each 2 x 2 block (p, q) is made real by the
// phase of a_pq and then diagonalised by the real symmetric Jacobi rotation
// (Golub and Van Loan, Matrix Computations, Sec. 8.5).  w ascending, V's
// columns in the same order.
static void jacobi_eigh(int n, std::vector<cd> A, std::vector<double>& w, std::vector<cd>& V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i + i * n] = 1.0;
  double fro = 0.0;
  for (const cd& x : A) fro += std::norm(x);
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int q = 0; q < n; ++q)
      for (int p = 0; p < q; ++p) off += std::norm(A[p + q * n]);
    if (std::sqrt(2.0 * off) <= 1e-15 * fro || fro == 0.0) break;
    for (int q = 1; q < n; ++q)
      for (int p = 0; p < q; ++p) {
        const cd apq = A[p + q * n];
        const double r = std::abs(apq);
        if (r == 0.0) continue;
        const cd e = apq / r;  // e^{i phi}
        const double app = A[p + p * n].real(), aqq = A[q + q * n].real();
        const double tau = (aqq - app) / (2.0 * r);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::abs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // U = diag(1, conj(e)) [[c, s], [-s, c]]: columns p, q of A and V
        const cd up_q = -s * std::conj(e), uq_q = c * std::conj(e);
        for (int k = 0; k < n; ++k) {
          const cd akp = A[k + p * n], akq = A[k + q * n];
          A[k + p * n] = akp * c + akq * up_q;
          A[k + q * n] = akp * s + akq * uq_q;
          const cd vkp = V[k + p * n], vkq = V[k + q * n];
          V[k + p * n] = vkp * c + vkq * up_q;
          V[k + q * n] = vkp * s + vkq * uq_q;
        }
        // rows p, q: A <- U^H A
        for (int k = 0; k < n; ++k) {
          const cd apk = A[p + k * n], aqk = A[q + k * n];
          A[p + k * n] = c * apk + std::conj(up_q) * aqk;
          A[q + k * n] = s * apk + std::conj(uq_q) * aqk;
        }
        A[p + q * n] = 0.0;
        A[q + p * n] = 0.0;
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int i, int j) { return A[i + i * n].real() < A[j + j * n].real(); });
  std::vector<cd> Vs(n * n);
  w.resize(n);
  for (int c = 0; c < n; ++c) {
    w[c] = A[order[c] + order[c] * n].real();
    for (int k = 0; k < n; ++k) Vs[k + c * n] = V[k + order[c] * n];
  }
  V.swap(Vs);
}

}  // namespace dense

namespace {

using dense::cd;

struct Blas {
  cublasHandle_t h = nullptr;
  ~Blas() {
    if (h) cublasDestroy(h);
  }
};

#define PVSC_BLAS_TRY(call)                                                                   \
  do {                                                                                        \
    cublasStatus_t s_ = (call);                                                               \
    if (s_ != CUBLAS_STATUS_SUCCESS) return set_error(PVSC_ERR_CUDA, "%s failed (%d)", #call, (int)s_); \
  } while (0)

// Jackson-damped Chebyshev coefficients of the indicator of [lo, hi] on x = (E - b)/a
// (x = cos(theta): c_0 = (theta_lo - theta_hi)/pi, c_k = 2 (sin k theta_lo - sin k theta_hi)/(pi k)).
std::vector<double> window_coefficients(double lo, double hi, double a, double b, int degree) {
  auto clampx = [](double x) { return x < -1.0 ? -1.0 : (x > 1.0 ? 1.0 : x); };
  const double tl = std::acos(clampx((lo - b) / a)), th = std::acos(clampx((hi - b) / a));
  const int M = degree + 1;
  const double q = M_PI / (M + 1);
  std::vector<double> c(M);
  for (int k = 0; k < M; ++k) {
    const double ck = k == 0 ? (tl - th) / M_PI : 2.0 * (std::sin(k * tl) - std::sin(k * th)) / (M_PI * k);
    const double gk = ((M - k + 1) * std::cos(q * k) + std::sin(q * k) / std::tan(q)) / (M + 1);
    c[k] = ck * gk;
  }
  return c;
}

struct FdLayout {
  size_t y, hq, gram, dots, sub, total;
};

FdLayout fd_layout(const pvsc_lattice* lat, int n, int prec, int degree) {
  FdLayout L;
  const size_t vb = vec_bytes(lat, n, PVSC_C128);
  L.y = 0;
  L.hq = L.y + vb;
  L.gram = L.hq + vb;
  L.dots = L.gram + (((size_t)n * n * 16 + 255) & ~size_t(255));
  L.sub = L.dots + (((size_t)4 * n * 8 + 255) & ~size_t(255));
  size_t sub = pvsc_work_bytes(lat, PVSC_OP_SERIES, n, prec, degree + 1);
  sub = std::max(sub, pvsc_work_bytes(lat, PVSC_OP_CHEB_STEP, n, PVSC_C128, 0));
  L.total = L.sub + ((sub + 255) & ~size_t(255));
  return L;
}

char* at(void* w, size_t off) { return static_cast<char*>(w) + off; }

// conj(A A^H) into the host n x n matrix G (column-major), A = n x D (ld n).
int gram(cublasHandle_t h, int n, int64_t D, const void* A, void* dG, std::vector<cd>& G,
         cudaStream_t st) {
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  const auto* a = static_cast<const cuDoubleComplex*>(A);
  PVSC_BLAS_TRY(cublasZgemm(h, CUBLAS_OP_N, CUBLAS_OP_C, n, n, (int)D, &one, a, n, a, n, &zero,
                            static_cast<cuDoubleComplex*>(dG), n));
  G.resize((size_t)n * n);
  PVSC_CUDA_TRY(cudaMemcpyAsync(G.data(), dG, sizeof(cd) * n * n, cudaMemcpyDeviceToHost, st));
  PVSC_CUDA_TRY(cudaStreamSynchronize(st));
  for (auto& x : G) x = std::conj(x);
  return PVSC_OK;
}

// out = M^T-applied block: column-major out (n x D) = op(M) A with op = N (M as given) or T.
int apply_small(cublasHandle_t h, cublasOperation_t op, int n, int64_t D, const std::vector<cd>& M,
                void* dM, const void* A, void* out, cudaStream_t st) {
  PVSC_CUDA_TRY(cudaMemcpyAsync(dM, M.data(), sizeof(cd) * n * n, cudaMemcpyHostToDevice, st));
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  PVSC_BLAS_TRY(cublasZgemm(h, op, CUBLAS_OP_N, n, (int)D, n, &one, static_cast<const cuDoubleComplex*>(dM),
                            n, static_cast<const cuDoubleComplex*>(A), n, &zero,
                            static_cast<cuDoubleComplex*>(out), n));
  // M is pageable host memory: the copy above completed before returning
  return PVSC_OK;
}

// One CholeskyQR pass on the block Y (in place through tmp): Y <- Y R^{-1} with
// Y^H Y + shift I = R^H R.  Returns PVSC_ERR_ARG if the Gram matrix is not
// positive definite even with the shift.
int cholqr_pass(cublasHandle_t h, int n, int64_t D, void* Y, void* tmp, void* dG, double shift_rel,
                cudaStream_t st) {
  std::vector<cd> G;
  if (int rc = gram(h, n, D, Y, dG, G, st)) return rc;
  double tr = 0.0;
  for (int i = 0; i < n; ++i) tr += G[i + i * n].real();
  for (int i = 0; i < n; ++i) G[i + i * n] += shift_rel * tr;
  if (!dense::cholesky(n, G))
    return set_error(PVSC_ERR_ARG, "ChebFD: the filtered block lost rank (Gram matrix not positive definite)");
  // G = L L^H, Y^H Y = L L^H, R = L^H: Y R^{-1} = Y L^{-H}; in the column-major
  // view A = Y^T: A_new = (L^{-H})^T A = conj(L^{-1}) A
  std::vector<cd> Li = dense::lower_inverse(n, G);
  for (auto& x : Li) x = std::conj(x);
  if (int rc = apply_small(h, CUBLAS_OP_N, n, D, Li, dG, Y, tmp, st)) return rc;
  PVSC_CUDA_TRY(cudaMemcpyAsync(Y, tmp, sizeof(cd) * n * D, cudaMemcpyDeviceToDevice, st));
  return PVSC_OK;
}

}  // namespace
}  // namespace pvsc

using namespace pvsc;

extern "C" {

int pvsc_debug_eigh(int n, const double* A, double* w, double* V) {
  if (n < 1 || n > 1024 || !A || !w || !V) return set_error(PVSC_ERR_ARG, "bad arguments");
  std::vector<cd> M(n * n);
  for (int i = 0; i < n * n; ++i) M[i] = cd(A[2 * i], A[2 * i + 1]);
  std::vector<double> ww;
  std::vector<cd> VV;
  dense::jacobi_eigh(n, M, ww, VV);
  for (int i = 0; i < n; ++i) w[i] = ww[i];
  for (int i = 0; i < n * n; ++i) {
    V[2 * i] = VV[i].real();
    V[2 * i + 1] = VV[i].imag();
  }
  return PVSC_OK;
}

size_t pvsc_chebfd_work_bytes(const pvsc_lattice* lat, int n_search, int prec, int degree) {
  if (!lat || !valid_R(n_search) || (prec != PVSC_C128 && prec != PVSC_C64) || degree < 1) return 0;
  return fd_layout(lat, n_search, prec, degree).total;
}

int pvsc_chebfd(const pvsc_lattice* lat, const pvsc_chebfd_params* prm, double a, double b,
                void* X, double* theta, double* resid, int* n_inside, int* iterations, void* work,
                size_t work_bytes, void* stream) {
  if (int rc = check_lattice(lat)) return rc;
  if (!prm || !theta || !resid || !n_inside || !iterations) return set_error(PVSC_ERR_ARG, "null argument");
  const int n = prm->n_search;
  if (!valid_R(n)) return set_error(PVSC_ERR_ARG, "n_search = %d: must be 1, 2, 4, 8, 16, 32 or 64", n);
  if (prm->prec != PVSC_C128 && prm->prec != PVSC_C64) return set_error(PVSC_ERR_ARG, "unknown precision");
  if (prm->degree < 1 || prm->max_iter < 1 || !(prm->tol > 0) || !(prm->hi > prm->lo))
    return set_error(PVSC_ERR_ARG, "need degree >= 1, max_iter >= 1, tol > 0, lo < hi");
  if (!(std::isfinite(a) && a > 0) || !std::isfinite(b)) return set_error(PVSC_ERR_ARG, "bad scaling a, b");
  if (int rc = check_ptr(X, "X")) return rc;
  const FdLayout L = fd_layout(lat, n, prm->prec, prm->degree);
  if (int rc = check_ptr(work, "work")) return rc;
  if (work_bytes < L.total) return set_error(PVSC_ERR_ARG, "work too small: %zu < %zu", work_bytes, L.total);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t D = lat->g.n_sites * orbitals_of(lat->g.model);
  void* Y = at(work, L.y);
  void* HQ = at(work, L.hq);
  void* dG = at(work, L.gram);
  double* dots = reinterpret_cast<double*>(at(work, L.dots));
  void* sub = at(work, L.sub);
  const size_t sub_bytes = L.total - L.sub;
  Blas blas;
  PVSC_BLAS_TRY(cublasCreate(&blas.h));
  PVSC_BLAS_TRY(cublasSetStream(blas.h, st));
  const std::vector<double> c = window_coefficients(prm->lo, prm->hi, a, b, prm->degree);
  if (int rc = pvsc_random_vectors(lat, n, PVSC_C128, prm->seed, X, stream)) return rc;
  std::vector<double> w(n), res(n), ones(n, 1.0);
  *iterations = 0;
  *n_inside = 0;
  for (int it = 1; it <= prm->max_iter; ++it) {
    *iterations = it;
    // filter
    if (int rc = pvsc_cheb_filter(lat, n, prm->prec, X, Y, c.data(), (int)c.size(), a, b, sub, sub_bytes, stream))
      return rc;
    // orthonormalize: shifted CholeskyQR, then two plain passes
    if (int rc = cholqr_pass(blas.h, n, D, Y, HQ, dG, 1e-13 * (double)(n + 1), st)) return rc;
    for (int pass = 0; pass < 2; ++pass)
      if (int rc = cholqr_pass(blas.h, n, D, Y, HQ, dG, 0.0, st)) return rc;
    // Rayleigh-Ritz: Hs = Q^H H Q = conj(A_Q B^H), B = (H Q)^T
    if (int rc = pvsc_apply_H(lat, n, PVSC_C128, Y, HQ, stream)) return rc;
    {
      const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
      PVSC_BLAS_TRY(cublasZgemm(blas.h, CUBLAS_OP_N, CUBLAS_OP_C, n, n, (int)D, &one,
                                static_cast<const cuDoubleComplex*>(Y), n,
                                static_cast<const cuDoubleComplex*>(HQ), n, &zero,
                                static_cast<cuDoubleComplex*>(dG), n));
    }
    std::vector<cd> Hs((size_t)n * n);
    PVSC_CUDA_TRY(cudaMemcpyAsync(Hs.data(), dG, sizeof(cd) * n * n, cudaMemcpyDeviceToHost, st));
    PVSC_CUDA_TRY(cudaStreamSynchronize(st));
    for (auto& x : Hs) x = std::conj(x);
    for (int j = 0; j < n; ++j)  // exact Hermitian symmetry
      for (int i = 0; i < j; ++i) {
        const cd m = 0.5 * (Hs[i + j * n] + std::conj(Hs[j + i * n]));
        Hs[i + j * n] = m;
        Hs[j + i * n] = std::conj(m);
      }
    std::vector<cd> Wv;
    dense::jacobi_eigh(n, Hs, w, Wv);
    // Ritz vectors X = Q W: column-major A_X = W^T A_Q
    if (int rc = apply_small(blas.h, CUBLAS_OP_T, n, D, Wv, dG, Y, X, st)) return rc;
    // residuals ||(H - theta_r) x_r|| in one fused sweep
    if (int rc = pvsc_cheb_step(lat, n, PVSC_C128, X, HQ, nullptr, ones.data(), w.data(), nullptr, nullptr,
                                PVSC_DOT_YY, dots, sub, sub_bytes, stream))
      return rc;
    std::vector<double> hd(4 * n);
    PVSC_CUDA_TRY(cudaMemcpyAsync(hd.data(), dots, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, st));
    PVSC_CUDA_TRY(cudaStreamSynchronize(st));
    int inside = 0;
    bool done = true;
    for (int r = 0; r < n; ++r) {
      res[r] = std::sqrt(std::max(hd[3 * n + r], 0.0));
      if (w[r] >= prm->lo && w[r] <= prm->hi) {
        ++inside;
        if (!(res[r] < prm->tol)) done = false;
      }
    }
    *n_inside = inside;
    if (done) break;
  }
  for (int r = 0; r < n; ++r) {
    theta[r] = w[r];
    resid[r] = res[r];
  }
  return PVSC_OK;
}

}  // extern "C"
