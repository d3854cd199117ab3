// Lattice handles, argument checking, error reporting and the geometry-side
// entry points of the C ABI (create/destroy/info, potential, Gershgorin
// bounds, neighbour-table export).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <vector>

#include "internal.h"

namespace pvsc {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

bool valid_R(int R) {
  return R == 1 || R == 2 || R == 4 || R == 8 || R == 16 || R == 32 || R == 64;
}

int vpt_for(int R, int prec) { return (prec == PVSC_C64 && R >= 2) ? 2 : 1; }

int vpt_tuned(int tuned, int R, int prec) {
  if (tuned == 1) return 1;
  if (tuned == 2 && prec == PVSC_C64 && R >= 2) return 2;
  return vpt_for(R, prec);
}

int check_lattice(const pvsc_lattice* lat) {
  if (!lat) return set_error(PVSC_ERR_ARG, "lattice handle is NULL");
  return PVSC_OK;
}

int check_ptr(const void* p, const char* name) {
  if (!p) return set_error(PVSC_ERR_ARG, "%s is NULL", name);
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0)
    return set_error(PVSC_ERR_ARG, "%s is not 16-byte aligned", name);
  return PVSC_OK;
}

size_t vec_bytes(const pvsc_lattice* lat, int R, int prec) {
  const int64_t D = lat->g.n_sites * orbitals_of(lat->g.model);
  const size_t b = (size_t)D * R * (prec == PVSC_C128 ? 16 : 8);
  return (b + 255) & ~size_t(255);
}

size_t dots_work_bytes(const pvsc_lattice* lat, int R) {
  return kWorkHeader + (size_t)lat->sm_count * kMaxGridPerSM * kNumDots * R * sizeof(double);
}

}  // namespace pvsc

pvsc_lattice::~pvsc_lattice() {
  for (auto& kv : graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  if (V_dev) cudaFree(V_dev);
  if (V32_dev) cudaFree(V32_dev);
  if (qd_dev) cudaFree(qd_dev);
}

using namespace pvsc;

// Dot centres of Eq. qdotarray relative to the nearest cell row / column
// (see QDScal): X_l = 3 row[l] + ex[l], Y_k = sqrt(3) col[k] + ey[k].
static void qdots_setup(const pvsc_lattice_desc& d, QDScal& q) {
  const double s3 = std::sqrt(3.0);
  const int K = d.qd_count;
  const double Nx = (double)d.dims[0], Ny = (double)d.dims[1];
  const double Xc = 1.5 * Ny, Yc = 0.5 * s3 * Nx;
  const double D = 4.0 * d.qd_radius;
  q = QDScal{};
  q.K = K;
  q.R = d.qd_radius;
  q.w = d.qd_width;
  q.rcut = q.R + 20.0 * q.w;
  q.invD = 1.0 / D;
  for (int i = 0; i < K; ++i) {
    const double off = (i - (K - 1) / 2.0) * D;
    const double X = Xc + off, Y = Yc + off;
    q.row[i] = (int)std::llround(X / 3.0);
    q.ex[i] = X - 3.0 * q.row[i];
    q.col[i] = (int)std::llround(Y / s3);
    q.ey[i] = Y - s3 * q.col[i];
    q.Vk[i] = d.qd_V0 + d.qd_dV * std::fabs(i - K / 2.0);
    q.exf[i] = (float)q.ex[i];
    q.eyf[i] = (float)q.ey[i];
    q.Vkf[i] = (float)q.Vk[i];
  }
  q.row0 = q.row[0];
  q.col0 = q.col[0];
  q.ex0 = q.ex[0];
  q.ey0 = q.ey[0];
  q.ex0f = (float)q.ex0;
  q.ey0f = (float)q.ey0;
  q.rcutf = (float)q.rcut;
  q.invDf = (float)q.invD;
  q.Rf = (float)q.R;
  q.inv_wf = (float)(1.0 / q.w);
}

extern "C" {

const char* pvsc_last_error(void) { return g_err.c_str(); }

const char* pvsc_version(void) { return "pvsc-gb300 1.0 (sm_103a)"; }

int pvsc_lattice_create(const pvsc_lattice_desc* desc, void* stream, pvsc_lattice** out) {
  if (!desc || !out) return set_error(PVSC_ERR_ARG, "desc and out must not be NULL");
  if (desc->model != PVSC_TI && desc->model != PVSC_GRAPHENE && desc->model != PVSC_WSM)
    return set_error(PVSC_ERR_ARG, "unknown model %d", desc->model);
  if (desc->model == PVSC_WSM && (desc->dims[0] % 2 != 0 || !std::isfinite(desc->k0)))
    return set_error(PVSC_ERR_ARG, "the Weyl semimetal needs an even Lx (its sweep pairs sites "
                     "along x) and a finite k0");
  for (int d = 0; d < 3; ++d)
    if (desc->dims[d] < 1) return set_error(PVSC_ERR_ARG, "dims[%d] = %lld < 1", d, (long long)desc->dims[d]);
  if (desc->model == PVSC_GRAPHENE && desc->dims[2] != 1)
    return set_error(PVSC_ERR_ARG, "graphene lattices are 2D: dims[2] must be 1");
  if (!std::isfinite(desc->t) || !std::isfinite(desc->m))
    return set_error(PVSC_ERR_ARG, "t and m must be finite");
  if (!std::isfinite(desc->delta1) || !std::isfinite(desc->delta2))
    return set_error(PVSC_ERR_ARG, "delta1 and delta2 must be finite");
  if (desc->model != PVSC_TI && (desc->delta1 != 0.0 || desc->delta2 != 0.0))
    return set_error(PVSC_ERR_ARG, "Delta terms belong to the TI model");
  if (desc->v_source < PVSC_V_ZERO || desc->v_source > PVSC_V_QDOT)
    return set_error(PVSC_ERR_ARG, "unknown v_source %d", desc->v_source);
  if (desc->v_source == PVSC_V_QDOT) {
    if (desc->model != PVSC_GRAPHENE)
      return set_error(PVSC_ERR_ARG, "the quantum-dot array potential belongs to the graphene model");
    if (desc->qd_count < 1 || desc->qd_count > kMaxQDots)
      return set_error(PVSC_ERR_ARG, "qd_count = %d: must be 1 .. %d", desc->qd_count, kMaxQDots);
    if (!(std::isfinite(desc->qd_radius) && desc->qd_radius > 0.0) ||
        !(std::isfinite(desc->qd_width) && desc->qd_width > 0.0) || !std::isfinite(desc->qd_V0) ||
        !std::isfinite(desc->qd_dV))
      return set_error(PVSC_ERR_ARG, "quantum dots need a positive finite radius and width and finite V0, dV");
  }
  if ((desc->v_source == PVSC_V_HOST || desc->v_source == PVSC_V_DEVICE) && !desc->V)
    return set_error(PVSC_ERR_ARG, "v_source needs desc->V");
  if ((desc->v_source == PVSC_V_SEED || desc->v_source == PVSC_V_ON_THE_FLY) && !std::isfinite(desc->W))
    return set_error(PVSC_ERR_ARG, "W must be finite");
  const double cells = (double)desc->dims[0] * (double)desc->dims[1] * (double)desc->dims[2];
  if (cells * 4.0 * kMaxR > 4.0e18) return set_error(PVSC_ERR_ARG, "lattice too large");
  if (desc->flags & ~PVSC_LATTICE_Z_HALO) return set_error(PVSC_ERR_ARG, "unknown lattice flags 0x%x", desc->flags);
  const int nhalo = ((desc->flags & PVSC_LATTICE_Z_HALO_LO) ? 1 : 0) + ((desc->flags & PVSC_LATTICE_Z_HALO_HI) ? 1 : 0);
  if (nhalo &&
      (desc->model != PVSC_TI || desc->periodic[2] || desc->dims[2] < nhalo + 1 ||
       !(desc->v_source == PVSC_V_ZERO || desc->v_source == PVSC_V_HOST || desc->v_source == PVSC_V_DEVICE)))
    return set_error(PVSC_ERR_ARG, "halo planes need a TI lattice, an open z axis with at least one plane "
                     "besides them and a given potential (zero, host or device: the slab's part of the global one)");

  pvsc_lattice* lat = new (std::nothrow) pvsc_lattice();
  if (!lat) return set_error(PVSC_ERR_OOM, "out of host memory");
  Geometry& g = lat->g;
  g.model = desc->model;
  for (int d = 0; d < 3; ++d) {
    g.per[d] = desc->periodic[d] ? 1 : 0;
    g.L[d] = desc->dims[d];
  }
  g.n_sites = desc->model == PVSC_GRAPHENE ? 4 * desc->dims[0] * desc->dims[1]
                                          : desc->dims[0] * desc->dims[1] * desc->dims[2];
  g.t = desc->t;
  g.m = desc->model == PVSC_TI ? desc->m : (desc->model == PVSC_WSM ? 2.0 + std::cos(desc->k0) : 0.0);
  g.d1 = desc->model == PVSC_TI ? desc->delta1 : 0.0;
  g.d2 = desc->model == PVSC_TI ? desc->delta2 : 0.0;
  g.d1f = (float)g.d1;
  g.d2f = (float)g.d2;
  g.has_delta = (g.d1 != 0.0 || g.d2 != 0.0) ? 1 : 0;
  g.zhalo = desc->flags & PVSC_LATTICE_Z_HALO;
  g.v_mode = 0;
  g.W = desc->W;
  g.vkey = hash_key(desc->seed, 0);
  lat->v_source = desc->v_source;
  lat->seed = desc->seed;
  cudaError_t e = cudaGetDevice(&lat->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&lat->sm_count, cudaDevAttrMultiProcessorCount, lat->device);
  if (e != cudaSuccess) {
    delete lat;
    return set_error(PVSC_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = PVSC_OK;
  if (desc->v_source == PVSC_V_HOST || desc->v_source == PVSC_V_DEVICE || desc->v_source == PVSC_V_SEED) {
    e = cudaMalloc(&lat->V_dev, sizeof(double) * g.n_sites);
    if (e == cudaSuccess) e = cudaMalloc(&lat->V32_dev, sizeof(float) * g.n_sites);
    if (e != cudaSuccess) {
      delete lat;
      return set_error(PVSC_ERR_OOM, "cudaMalloc of V failed: %s", cudaGetErrorString(e));
    }
    g.V = lat->V_dev;
    g.V32 = lat->V32_dev;
    g.v_mode = 1;
    if (desc->v_source == PVSC_V_SEED) {
      rc = launch_seed_potential(lat->V_dev, g.n_sites, desc->seed, desc->W, st);
    } else {
      e = cudaMemcpyAsync(lat->V_dev, desc->V, sizeof(double) * g.n_sites,
                          desc->v_source == PVSC_V_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) rc = set_error(PVSC_ERR_CUDA, "copy of V failed: %s", cudaGetErrorString(e));
    }
    if (rc == PVSC_OK) rc = launch_potential_f32(lat->V_dev, lat->V32_dev, g.n_sites, st);
  } else if (desc->v_source == PVSC_V_ON_THE_FLY) {
    g.v_mode = 2;
  } else if (desc->v_source == PVSC_V_QDOT) {
    QDots q;
    qdots_setup(*desc, q.s);
    e = cudaMalloc(&lat->qd_dev, sizeof(QDots));
    if (e != cudaSuccess) {
      delete lat;
      return set_error(PVSC_ERR_OOM, "cudaMalloc of the quantum-dot table failed: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(lat->qd_dev, &q, sizeof(QDots), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = set_error(PVSC_ERR_CUDA, "copy of the quantum-dot table failed: %s", cudaGetErrorString(e));
    g.qd = lat->qd_dev;
    lat->qds = q.s;
    g.v_mode = 3;
  }
  if (rc == PVSC_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = set_error(PVSC_ERR_CUDA, "lattice setup failed: %s", cudaGetErrorString(e));
  }
  if (rc != PVSC_OK) {
    delete lat;
    return rc;
  }
  lat->generation = next_generation();
  *out = lat;
  return PVSC_OK;
}

int pvsc_lattice_destroy(pvsc_lattice* lat) {
  delete lat;
  return PVSC_OK;
}

int pvsc_lattice_info(const pvsc_lattice* lat, int64_t* n_sites, int32_t* orbitals) {
  if (int rc = check_lattice(lat)) return rc;
  if (n_sites) *n_sites = lat->g.n_sites;
  if (orbitals) *orbitals = orbitals_of(lat->g.model);
  return PVSC_OK;
}

int pvsc_set_potential(pvsc_lattice* lat, const double* V_dev, void* stream) {
  if (int rc = check_lattice(lat)) return rc;
  if (!V_dev) return set_error(PVSC_ERR_ARG, "V_dev is NULL");
  if (lat->g.v_mode == 2 || lat->g.v_mode == 3)
    return set_error(PVSC_ERR_ARG, "the potential of this lattice is regenerated on the fly");
  if (!lat->V_dev) {
    cudaError_t e = cudaMalloc(&lat->V_dev, sizeof(double) * lat->g.n_sites);
    if (e == cudaSuccess) e = cudaMalloc(&lat->V32_dev, sizeof(float) * lat->g.n_sites);
    if (e != cudaSuccess) return set_error(PVSC_ERR_OOM, "cudaMalloc of V failed: %s", cudaGetErrorString(e));
    lat->g.V = lat->V_dev;
    lat->g.V32 = lat->V32_dev;
    lat->g.v_mode = 1;
    // cached graphs captured with V = 0 read no potential: drop them
    drop_graphs(lat);
  }
  lat->gersh_valid = false;
  PVSC_CUDA_TRY(cudaMemcpyAsync(lat->V_dev, V_dev, sizeof(double) * lat->g.n_sites,
                                cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
  return launch_potential_f32(lat->V_dev, lat->V32_dev, lat->g.n_sites, static_cast<cudaStream_t>(stream));
}

int pvsc_get_potential(const pvsc_lattice* lat, double* V_out_dev, void* stream) {
  if (int rc = check_lattice(lat)) return rc;
  if (!V_out_dev) return set_error(PVSC_ERR_ARG, "V_out_dev is NULL");
  return launch_get_potential(lat->g, V_out_dev, static_cast<cudaStream_t>(stream));
}

int pvsc_spectral_bounds(const pvsc_lattice* lat, double eps, double* emin, double* emax,
                         double* a, double* b, void* work, size_t work_bytes, void* stream) {
  if (int rc = check_lattice(lat)) return rc;
  if (int rc = check_ptr(work, "work")) return rc;
  if (!std::isfinite(eps) || eps < 0) return set_error(PVSC_ERR_ARG, "eps must be finite and >= 0");
  const int grid = 2 * lat->sm_count;
  if (work_bytes < sizeof(double) * 2 * grid)
    return set_error(PVSC_ERR_ARG, "work too small: %zu < %zu", work_bytes, sizeof(double) * 2 * grid);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (int rc = launch_gershgorin(lat->g, static_cast<double*>(work), grid, st)) return rc;
  std::vector<double> h(2 * grid);
  PVSC_CUDA_TRY(cudaMemcpyAsync(h.data(), work, sizeof(double) * 2 * grid, cudaMemcpyDeviceToHost, st));
  PVSC_CUDA_TRY(cudaStreamSynchronize(st));
  double lo = h[0], hi = h[1];
  for (int i = 0; i < grid; ++i) {
    if (std::isnan(h[2 * i]) || std::isnan(h[2 * i + 1]))
      return set_error(PVSC_ERR_ARG, "the potential holds a non-finite value (spectral bounds undefined)");
    lo = std::fmin(lo, h[2 * i]);
    hi = std::fmax(hi, h[2 * i + 1]);
  }
  if (emin) *emin = lo;
  if (emax) *emax = hi;
  if (a) *a = (hi - lo + eps) / 2.0;
  if (b) *b = (hi + lo) / 2.0;
  return PVSC_OK;
}

int pvsc_debug_neighbours(const pvsc_lattice* lat, int64_t* nbr_dev, void* stream) {
  if (int rc = check_lattice(lat)) return rc;
  if (!nbr_dev) return set_error(PVSC_ERR_ARG, "nbr_dev is NULL");
  return launch_neighbours(lat->g, nbr_dev, static_cast<cudaStream_t>(stream));
}

// Sparsity pattern of H as the stencil applies it (host only).  Per row, one
// entry per stencil term in the order the sweeps take them; a term whose
// coefficient block entry is structurally zero is not listed.
//   TI (row = 4 n + o): the diagonal (m Gamma^1 + V), the Delta terms (o ^ 1)
//     when present, then for the neighbours z-, z+, x-, x+, y-, y+ the
//     Gamma^1 part (same orbital) and the Gamma^{j+1} part (orbital 3 - o along
//     x and y, o ^ 1 along z) of the bond block.
//   Graphene (row = 4 c + nu): the diagonal, then the chain and bond couplings
//     of Eq. graphene_model in the order of the graphene sweep.
//   Weyl semimetal (row = 2 n + o): the diagonal, the on-site sigma_x term
//     (orbital 1 - o), the x-/x+ bonds (1 - o), one term along y (row 0 takes
//     orbital 1 of n - e_y, row 1 orbital 0 of n + e_y), and along z both
//     orbitals of both neighbours ((sigma_x + i sigma_z)/2 has no zero entry).
int pvsc_debug_export_pattern(const pvsc_lattice* lat, int64_t* rowptr, int32_t* col) {
  if (int rc = check_lattice(lat)) return rc;
  if (!rowptr) return set_error(PVSC_ERR_ARG, "rowptr is NULL");
  const Geometry& g = lat->g;
  const int O = orbitals_of(g.model);
  const int64_t D = g.n_sites * O;
  if (D > (int64_t(1) << 24)) return set_error(PVSC_ERR_ARG, "pattern export is for small lattices (D = %lld > 2^24)", (long long)D);
  std::vector<int64_t> cols;
  cols.reserve(16);
  int64_t nnz = 0;
  auto put = [&](int64_t c) {
    if (c >= 0) cols.push_back(c);
  };
  for (int64_t row = 0; row < D; ++row) {
    cols.clear();
    if (g.model == PVSC_GRAPHENE) {
      const int64_t Nx = g.L[0], Ny = g.L[1];
      const int64_t c = row >> 2, nu = row & 3, y = c / Nx, x = c - y * Nx;
      const int64_t cxm = nbr_minus(c, x, Nx, g.per[0], 1), cxp = nbr_plus(c, x, Nx, g.per[0], 1);
      const int64_t cym = nbr_minus(c, y, Ny, g.per[1], Nx), cyp = nbr_plus(c, y, Ny, g.per[1], Nx);
      auto at = [](int64_t cell, int s) { return cell >= 0 ? 4 * cell + s : (int64_t)-1; };
      put(row);
      if (nu == 0) { put(at(c, 1)); put(at(cxp, 1)); put(at(cym, 3)); }
      if (nu == 1) { put(at(c, 0)); put(at(c, 2)); put(at(cxm, 0)); }
      if (nu == 2) { put(at(c, 1)); put(at(c, 3)); put(at(cxm, 3)); }
      if (nu == 3) { put(at(c, 2)); put(at(cxp, 2)); put(at(cyp, 0)); }
    } else {
      const int64_t Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], plane = Lx * Ly;
      const int64_t n = row / O, o = row - n * O;
      const int64_t z = n / plane, y = (n - z * plane) / Lx, x = n - z * plane - y * Lx;
      const int64_t zm = nbr_minus(n, z, Lz, g.per[2], plane), zp = nbr_plus(n, z, Lz, g.per[2], plane);
      const int64_t xm = nbr_minus(n, x, Lx, g.per[0], 1), xp = nbr_plus(n, x, Lx, g.per[0], 1);
      const int64_t ym = nbr_minus(n, y, Ly, g.per[1], Lx), yp = nbr_plus(n, y, Ly, g.per[1], Lx);
      auto at = [&](int64_t site, int64_t orb) { return site >= 0 ? O * site + orb : (int64_t)-1; };
      put(row);
      if (g.model == PVSC_TI) {
        if (g.has_delta) put(at(n, o ^ 1));
        const int64_t nb[6] = {zm, zp, xm, xp, ym, yp};
        for (int k = 0; k < 6; ++k) {
          put(at(nb[k], o));                                // Gamma^1 part of the bond block
          put(at(nb[k], k < 2 ? (o ^ 1) : (3 - o)));        // Gamma^{j+1} part
        }
      } else {  // Weyl semimetal
        put(at(n, 1 - o));
        put(at(xm, 1 - o));
        put(at(xp, 1 - o));
        put(o == 0 ? at(ym, 1) : at(yp, 0));
        put(at(zm, 1 - o));  // (sigma_x + i sigma_z)/2 and its conjugate: both orbitals
        put(at(zp, 1 - o));
        put(at(zm, o));
        put(at(zp, o));
      }
    }
    rowptr[row] = nnz;
    if (col)
      for (size_t k = 0; k < cols.size(); ++k) col[nnz + (int64_t)k] = (int32_t)cols[k];
    nnz += (int64_t)cols.size();
  }
  rowptr[D] = nnz;
  return PVSC_OK;
}

}  // extern "C"
