// Elementwise kernels around the sweeps: start vectors from the counter hash,
// precision conversion, series initialisation, the top of the adjoint
// recurrence, potential generation, the Gershgorin bound and the neighbour
// table export.
#include "internal.h"

namespace pvsc {

namespace {

inline int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

// r_i = exp(2 pi i u)/sqrt(D), u from stream 1 with idx = r D + i; element (i, r) at i R + r.
template <typename T>
__global__ void random_phase_kernel(T* out, int64_t D, int R, uint64_t key, double scale) {
  const int64_t n = D * R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = udiv64(e, R), r = e - i * R;
    random_phase_entry<T>(hash_uniform(key, (uint64_t)(r * D + i)), scale, out[2 * e], out[2 * e + 1]);
  }
}

__global__ void convert_kernel(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = in[e];
    out[e] = make_float2((float)a.x, (float)a.y);
  }
}

__global__ void scale_init_kernel(const double2* __restrict__ x, double2* __restrict__ acc, double cr,
                                  double ci, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = x[e];
    acc[e] = make_double2(cr * a.x - ci * a.y, cr * a.y + ci * a.x);
  }
}

// u_M = sigma G and grad[site] += gscale Re sum conj(u_M) w (one thread per site, R = 1 block)
__global__ void adjoint_top_kernel(const double2* __restrict__ G, double sr, double si,
                                   double2* __restrict__ uM, const double2* __restrict__ w,
                                   double gscale, double* __restrict__ grad, int64_t n_sites,
                                   int per_site) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_sites;
       s += (int64_t)gridDim.x * blockDim.x) {
    double g = 0.0;
    for (int k = 0; k < per_site; ++k) {
      const int64_t e = s * per_site + k;
      const double2 a = G[e];
      const double2 u = make_double2(sr * a.x - si * a.y, sr * a.y + si * a.x);
      uM[e] = u;
      const double2 b = w[e];
      g += u.x * b.x + u.y * b.y;
    }
    grad[s] += gscale * g;
  }
}

__global__ void seed_potential_kernel(double* V, int64_t n, uint64_t key, double W) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    V[s] = W * (hash_uniform(key, (uint64_t)s) - 0.5);
}

__global__ void potential_f32_kernel(const double* __restrict__ V, float* __restrict__ V32, int64_t n) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    V32[s] = (float)V[s];
}

__global__ void get_potential_kernel(Geometry g, double* out) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.n_sites;
       s += (int64_t)gridDim.x * blockDim.x) {
    out[s] = site_potential_any(g, s);
  }
}

// Per-row Gershgorin interval, reduced to one (min, max) per block.
__global__ void gershgorin_kernel(Geometry g, double* out /* [gridDim][2] */) {
  double lo = 1e300, hi = -1e300;
  bool bad = false;  // a non-finite potential (fmin / fmax would drop it silently)
  const double at = fabs(g.t);
  if (g.model == 1) {
    const int64_t Lx = g.L[0], Ly = g.L[1], Lz = g.L[2];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.n_sites;
         s += (int64_t)gridDim.x * blockDim.x) {
      const int64_t x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
      if (z < (g.zhalo & 1) || z >= Lz - (g.zhalo >> 1)) continue;  // halo planes: rows of another domain
      const int64_t co[3] = {x, y, z};
      double radius = 0.0, self = 0.0;  // self: coefficient of -t Gamma^1 from length-1 periodic axes
      for (int d = 0; d < 3; ++d) {
        const int64_t L = g.L[d];
        const int64_t mn = nbr_minus(co[d], co[d], L, g.per[d], 1);
        const int64_t pl = nbr_plus(co[d], co[d], L, g.per[d], 1);
        if (mn == co[d]) {            // L == 1 periodic: B + B^+ = -t Gamma^1 on the diagonal
          self += 1.0;
        } else if (mn >= 0 && mn == pl) {  // L == 2 periodic: one neighbour, B + B^+ = -t Gamma^1
          radius += at;
        } else {                      // each existing bond block has row abs-sum t
          if (mn >= 0) radius += at;
          if (pl >= 0) radius += at;
        }
      }
      const double V = site_potential_any(g, s);
      bad |= !isfinite(V);
      radius += sqrt(g.d1 * g.d1 + g.d2 * g.d2);  // one Delta entry per row, |D1 +- i D2|
      for (int sign = -1; sign <= 1; sign += 2) {  // Gamma^1 = +1 / -1 rows
        const double c = V + sign * (g.m - self * g.t);
        lo = fmin(lo, c - radius);
        hi = fmax(hi, c + radius);
      }
    }
  } else if (g.model == 3) {
    // Weyl semimetal (Eq. TB_H_wsm), rows a and b of each site: |A_x| rows 1/2,
    // A_y = [[0,1],[0,0]] reaches row a from y-1 and row b (A_y^+) from y+1,
    // |A_z| rows 1; a periodic axis of length 2 folds both bonds into sigma_x
    // (row sum 1), of length 1 into the on-site sigma_x coefficient -c0 + 1.
    const int64_t Lx = g.L[0], Ly = g.L[1], Lz = g.L[2];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.n_sites;
         s += (int64_t)gridDim.x * blockDim.x) {
      const int64_t x = s % Lx, y = (s / Lx) % Ly, z = s / (Lx * Ly);
      const int64_t co[3] = {x, y, z};
      double ra = 0.0, rb = 0.0, sx = -g.m;
      for (int d = 0; d < 3; ++d) {
        const int64_t mn = nbr_minus(co[d], co[d], g.L[d], g.per[d], 1);
        const int64_t pl = nbr_plus(co[d], co[d], g.L[d], g.per[d], 1);
        if (mn == co[d]) {
          sx += 1.0;
        } else if (mn >= 0 && mn == pl) {
          ra += 1.0;
          rb += 1.0;
        } else if (d == 0) {
          const double h = 0.5 * ((mn >= 0) + (pl >= 0));
          ra += h;
          rb += h;
        } else if (d == 1) {
          ra += (mn >= 0) ? 1.0 : 0.0;
          rb += (pl >= 0) ? 1.0 : 0.0;
        } else {
          const double h = (double)((mn >= 0) + (pl >= 0));
          ra += h;
          rb += h;
        }
      }
      const double V = site_potential_any(g, s);
      bad |= !isfinite(V);
      const double r = fmax(ra, rb) + fabs(sx);
      lo = fmin(lo, V - r);
      hi = fmax(hi, V + r);
    }
  } else {
    const int64_t Nx = g.L[0], Ny = g.L[1];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.n_sites;
         s += (int64_t)gridDim.x * blockDim.x) {
      const int64_t c = s / 4, nu = s % 4, x = c % Nx, y = c / Nx;
      // every coupling is -t, same sign, so coinciding entries do not cancel:
      // radius = t * (number of bond terms present in the row)
      int nb = 0;
      const bool hx = nbr_plus(x, x, Nx, g.per[0], 1) >= 0;
      const bool hxm = nbr_minus(x, x, Nx, g.per[0], 1) >= 0;
      const bool hym = nbr_minus(y, y, Ny, g.per[1], 1) >= 0;
      const bool hyp = nbr_plus(y, y, Ny, g.per[1], 1) >= 0;
      if (nu == 0) nb = 1 + (hx ? 1 : 0) + (hym ? 1 : 0);
      if (nu == 1) nb = 2 + (hxm ? 1 : 0);
      if (nu == 2) nb = 2 + (hxm ? 1 : 0);
      if (nu == 3) nb = 1 + (hx ? 1 : 0) + (hyp ? 1 : 0);
      const double V = site_potential_any(g, s);
      bad |= !isfinite(V);
      lo = fmin(lo, V - nb * at);
      hi = fmax(hi, V + nb * at);
    }
  }
  __shared__ double slo[256], shi[256];
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  bad = __syncthreads_or(bad) != 0;
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + w]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // a block that met a non-finite potential reports NaN
    out[2 * blockIdx.x] = bad ? __longlong_as_double(0x7ff8000000000000ll) : slo[0];
    out[2 * blockIdx.x + 1] = bad ? __longlong_as_double(0x7ff8000000000000ll) : shi[0];
  }
}

// Neighbour table with the sweeps' own index helpers.
__global__ void neighbours_kernel(Geometry g, int64_t* nbr) {
  if (g.model != 2) {  // cubic lattices (TI, Weyl semimetal): per site
    const int64_t Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], plane = Lx * Ly;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.n_sites;
         s += (int64_t)gridDim.x * blockDim.x) {
      const int64_t col = s % plane, z = s / plane, x = col % Lx, y = col / Lx;
      int64_t* o = nbr + 7 * s;
      o[0] = s;
      o[1] = nbr_minus(s, x, Lx, g.per[0], 1);
      o[2] = nbr_plus(s, x, Lx, g.per[0], 1);
      o[3] = nbr_minus(s, y, Ly, g.per[1], Lx);
      o[4] = nbr_plus(s, y, Ly, g.per[1], Lx);
      o[5] = nbr_minus(s, z, Lz, g.per[2], plane);
      o[6] = nbr_plus(s, z, Lz, g.per[2], plane);
    }
  } else {
    const int64_t Nx = g.L[0], Ny = g.L[1], nc = Nx * Ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * blockDim.x) {
      const int64_t x = c % Nx, y = c / Nx;
      int64_t* o = nbr + 7 * c;
      o[0] = c;
      o[1] = nbr_minus(c, x, Nx, g.per[0], 1);
      o[2] = nbr_plus(c, x, Nx, g.per[0], 1);
      o[3] = nbr_minus(c, y, Ny, g.per[1], Nx);
      o[4] = nbr_plus(c, y, Ny, g.per[1], Nx);
      o[5] = -1;
      o[6] = -1;
    }
  }
}

}  // namespace

int launch_random_phase(void* out, int prec, int64_t D, int R, uint64_t seed, cudaStream_t st) {
  const uint64_t key = hash_key(seed, 1);
  const double scale = 1.0 / sqrt((double)D);
  const int g = grid_for(D * R, 256);
  if (prec == PVSC_C128)
    random_phase_kernel<double><<<g, 256, 0, st>>>(static_cast<double*>(out), D, R, key, scale);
  else
    random_phase_kernel<float><<<g, 256, 0, st>>>(static_cast<float*>(out), D, R, key, scale);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

int launch_convert_c128_to_c64(const void* in, void* out, int64_t n, cudaStream_t st) {
  convert_kernel<<<grid_for(n, 256), 256, 0, st>>>(static_cast<const double2*>(in),
                                                   static_cast<float2*>(out), n);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

int launch_scale_init(const void* x128, double2* acc, double cr, double ci, int64_t n,
                      cudaStream_t st) {
  scale_init_kernel<<<grid_for(n, 256), 256, 0, st>>>(static_cast<const double2*>(x128), acc, cr,
                                                      ci, n);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

int launch_adjoint_top(const pvsc_lattice* lat, int R, const double2* G, double sr, double si,
                       double2* uM, const double2* w, double gscale, double* grad,
                       cudaStream_t st) {
  const int per_site = orbitals_of(lat->g.model) * R;
  adjoint_top_kernel<<<grid_for(lat->g.n_sites, 256), 256, 0, st>>>(G, sr, si, uM, w, gscale, grad,
                                                                  lat->g.n_sites, per_site);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

int launch_seed_potential(double* V, int64_t n, uint64_t seed, double W, cudaStream_t st) {
  seed_potential_kernel<<<grid_for(n, 256), 256, 0, st>>>(V, n, hash_key(seed, 0), W);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

int launch_potential_f32(const double* V, float* V32, int64_t n, cudaStream_t st) {
  potential_f32_kernel<<<grid_for(n, 256), 256, 0, st>>>(V, V32, n);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

int launch_get_potential(const Geometry& g, double* out, cudaStream_t st) {
  get_potential_kernel<<<grid_for(g.n_sites, 256), 256, 0, st>>>(g, out);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

int launch_gershgorin(const Geometry& g, double* out, int grid, cudaStream_t st) {
  gershgorin_kernel<<<grid, 256, 0, st>>>(g, out);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

int launch_neighbours(const Geometry& g, int64_t* nbr, cudaStream_t st) {
  const int64_t n = g.model != 2 ? g.n_sites : g.L[0] * g.L[1];
  neighbours_kernel<<<grid_for(n, 256), 256, 0, st>>>(g, nbr);
  PVSC_CUDA_TRY(cudaGetLastError());
  return PVSC_OK;
}

}  // namespace pvsc
