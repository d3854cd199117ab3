// Batched KPM: many independent TI lattices (disorder realisations of uneven
// size) x R random-phase vectors, all moments, in ONE persistent cooperative
// launch.
//
// Work list.  Every lattice is cut into units of one block of columns x one
// z-slab (the single-lattice sweep's units); all units of all lattices form one
// list that the resident blocks walk round-robin, phase after phase.  Phase 0
// writes the random-phase start block w_0 of the unit; phase 1 + k is the
// fused Chebyshev step k of the kernel polynomial method (stencil, recurrence
// update and the dot products <w_k|w_k>, <w_k+1|w_k>).
//
// Dependencies.  A unit of lattice i may start phase p only when every unit of
// lattice i has finished phase p - 1 and the moments of that phase have been
// reduced (per-lattice counters, no grid-wide barrier): lattices advance
// independently.  The last unit of a phase to arrive reduces the per-unit
// partial sums in unit order (bitwise reproducible), writes mu_2k, mu_2k+1 and
// publishes the phase.  Every wait spins at most `wait_limit` times; past that
// it sets an error word, and every block returns at its next check.  The
// launch is cooperative, so all blocks are co-resident and a wait can only be
// for work that some running block will do (units are processed in phase
// order by every block).
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include <algorithm>

#include "internal.h"
#include "sweep.cuh"

namespace pvsc {

static unsigned long long g_wait_limit = 1ull << 26;
static int g_inject_stall = 0;  // fault injection: the first wait targets a phase nobody publishes

struct BatchLat {
  Geometry g;
  int64_t nbx;       // column blocks
  int64_t units;     // nbx * nzs
  int64_t unit0;     // first global unit
  int zs;            // z-slab depth
  double a_inv;      // 1/a
  double b;
  uint64_t key;      // counter-hash key of the start vectors (stream 1)
  void* wa;
  void* wb;
  double* mu;        // [R][M]
  double* partials;  // [units][2][R]
  unsigned* arrive;  // units that finished the current phase (monotonic)
  unsigned* phase;   // phases completed and reduced (monotonic)
};

constexpr int kMaxBatch = 128;

// The whole lattice table travels as the kernel parameter (no upload, so the
// launch can be captured in a CUDA graph).
struct BatchArgs {
  BatchLat lats[kMaxBatch];
  int nlat;
  int64_t total_units;
  int R, C, M, nphases;
  int* err;
  unsigned long long wait_limit;
  int inject_stall;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *p >= target (bounded); the block learns the outcome.
__device__ bool block_wait_geq(const unsigned* p, unsigned target, const BatchArgs& a) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned long long n = 0;
    while (ld_acquire(p) < target) {
      if (*(volatile int*)a.err) { ok = 0; break; }
      if (++n > a.wait_limit) {
        atomicExch(a.err, 1);
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    s_ok = ok;
  }
  __syncthreads();
  __threadfence();  // every thread: later loads observe the published phase
  return s_ok != 0;
}

__device__ __forceinline__ int find_lattice(const BatchArgs& a, int64_t u) {
  int lo = 0, hi = a.nlat - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (a.lats[mid].unit0 <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T, int VPT>
__global__ void __launch_bounds__(256) kpm_batched_kernel(const __grid_constant__ BatchArgs a) {
  __shared__ double sm[kMaxThreads / 32][2][VPT][32];
  __shared__ int s_last;
  const int R = a.R, C = a.C;
  const int rc = threadIdx.x % C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int ph = 0; ph < a.nphases; ++ph) {
    for (int64_t u = blockIdx.x; u < a.total_units; u += gridDim.x) {
      const int li = find_lattice(a, u);
      const BatchLat& L = a.lats[li];
      if (ph > 0 && !block_wait_geq(L.phase, a.inject_stall ? 0xffffffffu : (unsigned)ph, a)) return;
      const int64_t lu = u - L.unit0;
      const int64_t bz = udiv64(lu, L.nbx), bx = lu - bz * L.nbx;
      const int64_t plane = L.g.L[0] * L.g.L[1], Lz = L.g.L[2];
      const int64_t tid = bx * blockDim.x + threadIdx.x;
      const bool active = tid < plane * C;
      const int64_t z0 = bz * L.zs, z1 = min(z0 + (int64_t)L.zs, Lz);
      const int64_t col = udiv64(tid, C);
      // per-site partials in (compensated, for complex64) working precision,
      // flushed to fp64 once per column segment
      DotAcc<T, VPT> dacc;
      dacc.init();
      if (ph == 0) {
        // w_0: random-phase vectors exp(2 pi i u)/sqrt(D), idx = r D + i
        if (active) {
          const int64_t D = 4 * L.g.n_sites;
          const double scale = 1.0 / sqrt((double)D);
          T* W0 = static_cast<T*>(L.wa);
          for (int64_t z = z0; z < z1; ++z) {
            const int64_t s = col + plane * z;
            Blk<T, VPT> b;
#pragma unroll
            for (int o = 0; o < 4; ++o)
#pragma unroll
              for (int v = 0; v < VPT; ++v) {
                const int64_t r = rc * VPT + v, i = 4 * s + o;
                random_phase_entry<T>(hash_uniform(L.key, (uint64_t)(r * D + i)), scale, b.v[o][v].re,
                                      b.v[o][v].im);
              }
            store_blk<T, VPT>(W0, s, R, rc, b);
          }
        }
      } else {
        const int k = ph - 1;
        const T* X = static_cast<const T*>(k == 0 ? L.wa : ((k & 1) ? L.wb : L.wa));
        T* Yout = static_cast<T*>(k == 0 ? L.wb : ((k & 1) ? L.wa : L.wb));
        const T* Yin = k == 0 ? nullptr : Yout;
        VecCoef<T, VPT> cf;
        const double alpha = (k == 0 ? 1.0 : 2.0) * L.a_inv;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          cf.alpha[v] = T(alpha);
          cf.ab[v] = T(alpha * L.b);
          cf.am[v] = T(alpha * L.g.m);
          cf.kt[v] = T(-0.5 * alpha * L.g.t);
          cf.gamma[v] = T(k == 0 ? 0.0 : -1.0);
          cf.delta[v] = T(0);
        }
        // the Delta terms are decided once per unit, outside the march: the
        // lattice (and its geometry) is picked at run time from the parameter
        // block, and a per-site branch on it costs the march its load overlap
        auto march = [&](auto with_delta) {
          // x is written by this kernel in other phases: coherent loads only (NC = false)
          ti_march<T, VPT, false, 0, 2>(L.g, X, Yin, R, rc, col, z0, z1, nullptr,
                                  [&](int64_t s) { return site_potential_t<T>(L.g, s); },
                                  [&](T Vs, const Blk<T, VPT>& xm, const Blk<T, VPT>& xc,
                                      const Blk<T, VPT>& xp, const Blk<T, VPT>& ax, const Blk<T, VPT>& bx,
                                      const Blk<T, VPT>& ay, const Blk<T, VPT>& by,
                                      const Blk<T, VPT>* yi, Blk<T, VPT>& yn) {
                                    Blk<T, VPT> S, D;
                                    ti_axes(xm, xp, ax, bx, ay, by, S, D);
                                    ti_combine_core(cf, Vs, xc, S, D, yi, yn);
                                    if constexpr (decltype(with_delta)::value) ti_add_delta(L.g, cf, xc, yn);
                                  },
                                  [&](int64_t s, const Blk<T, VPT>& xc, Blk<T, VPT>& yn) {
                                    store_blk<T, VPT>(Yout, s, R, rc, yn);
#pragma unroll
                                    for (int v = 0; v < VPT; ++v) {
                                      T xx = 0, xy = 0;
#pragma unroll
                                      for (int o = 0; o < 4; ++o) {
                                        const cplx<T> p = xc.v[o][v], q = yn.v[o][v];
                                        xx = fma(p.re, p.re, fma(p.im, p.im, xx));
                                        xy = fma(q.re, p.re, fma(q.im, p.im, xy));
                                      }
                                      dacc.add(0, v, xx);
                                      dacc.add(1, v, xy);
                                    }
                                  });
        };
        if (active) {
          if (L.g.has_delta) march(std::true_type{});
          else march(std::false_type{});
        }
        dacc.flush();
        // fixed-order block reduction to one row of partials for this unit
#pragma unroll
        for (int d = 0; d < 2; ++d)
#pragma unroll
          for (int v = 0; v < VPT; ++v) {
            double s = dacc.d[d][v];
            for (int off = 16; off >= C; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane < C) sm[warp][d][v][lane] = s;
          }
        __syncthreads();
        double* row = L.partials + (size_t)lu * 2 * R;
        for (int t = threadIdx.x; t < C; t += blockDim.x) {
          const int stride = C < 32 ? 1 : C / 32;
          const int w0 = C < 32 ? 0 : t / 32;
          const int l = C < 32 ? t : t % 32;
          for (int d = 0; d < 2; ++d)
            for (int v = 0; v < VPT; ++v) {
              double s = 0.0;
              for (int w = w0; w < nwarps; w += stride) s += sm[w][d][v][l];
              row[d * R + t * VPT + v] = s;
            }
        }
      }
      // arrive; the last unit of lattice li in this phase reduces and publishes
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = (atomicAdd(L.arrive, 1u) == (unsigned)((ph + 1) * L.units - 1));
      __syncthreads();
      if (s_last) {
        __threadfence();
        if (ph > 0) {
          const int k = ph - 1;
          for (int q = warp; q < 2 * R; q += nwarps) {
            const int d = q / R, r = q % R;
            double s = 0.0;
            for (int64_t b = lane; b < L.units; b += 32) s += __ldcg(L.partials + (size_t)b * 2 * R + q);
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) {
              double* mu = L.mu + (size_t)r * a.M;
              if (k == 0) {
                if (d == 0) mu[0] = s;
                if (d == 1 && a.M > 1) mu[1] = s;
              } else {
                if (d == 0 && 2 * k < a.M) mu[2 * k] = 2.0 * s - __ldcg(mu);
                if (d == 1 && 2 * k + 1 < a.M) mu[2 * k + 1] = 2.0 * s - __ldcg(mu + 1);
              }
            }
          }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(L.phase, (unsigned)(ph + 1));
      }
      __syncthreads();
    }
  }
}

// work: [error word + 2 counters per lattice | per lattice: w_a, w_b, partials]
static size_t batch_header_bytes(int n) {
  return (kWorkHeader + 2 * sizeof(unsigned) * (size_t)n + 255) & ~size_t(255);
}

// Launch shape of the batched kernel: threads per block, z-segment length and
// blocks per SM, from the tuning entry (R, prec) of the first lattice when set
// (pvsc_set_tuning), else 256 threads, whole columns (zs = 0), occupancy
// maximum.  Whole columns measured fastest on the 64-lattice batch (each unit
// pays a phase wait, a block reduction and a partial-row write).
struct BatchShape {
  int threads = 256, zs = 0, bps = 0;
  bool per_lattice = false;  // kernel 7: every lattice's KPM on the TMA-staged sweep
};
static BatchShape batch_shape(const pvsc_lattice* l0, int R, int prec) {
  BatchShape sh;
  const int C = R / vpt_for(R, prec);
  auto it = l0->tuning.find({R, prec});
  if (it != l0->tuning.end()) {
    const pvsc_tuning& t = it->second;
    if (t.threads >= 32 && t.threads <= kMaxThreads && t.threads % 32 == 0 && t.threads % C == 0)
      sh.threads = t.threads;
    if (t.zslab > 0) sh.zs = t.zslab;
    sh.bps = t.blocks_per_sm;
    if (t.kernel == kKernelTma) {
      sh.per_lattice = true;
      sh.threads = t.threads == 512 ? 512 : 256;
    }
  }
  return sh;
}

// ---------------------------------------------------------------- per-lattice mode
// Tuning kernel 7 on the batch: each lattice's KPM runs as its own chain of
// TMA-staged sweeps (kpm_enqueue), the chains spread over a few streams that
// fork from and join the caller's stream, all inside one captured graph; a
// large lattice's sweeps fill the GPU while the small lattices' short sweeps
// run beside them.  Work: per lattice the dot header and partials and its two
// recurrence vectors.  Sixteen streams: the 64-cube benchmark batch ran at 57.7,
// 62.0, 65.5 and 63.6 GLUP/s on 4, 8, 16 and 32.
constexpr int kBatchStreams = 16;

static bool per_lattice_possible(const pvsc_lattice* const* lats, int n, int R, int prec) {
  for (int i = 0; i < n; ++i)
    if (!lats[i] || !tma_sweep_possible(lats[i], R, prec)) return false;
  return true;
}

static size_t per_lattice_bytes(const pvsc_lattice* lat, int R, int prec) {
  return ((dots_work_bytes(lat, R) + 255) & ~size_t(255)) + 2 * vec_bytes(lat, R, prec);
}

static int kpm_per_lattice(const pvsc_lattice* const* lats, int n, int R, int prec, const uint64_t* seeds, int M,
                           const double* a, const double* b, double* mu, void* work, size_t work_bytes,
                           const BatchShape& bs, cudaStream_t st) {
  std::vector<size_t> off(n);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    off[i] = total;
    total += (per_lattice_bytes(lats[i], R, prec) + 255) & ~size_t(255);
  }
  if (work_bytes < total) return set_error(PVSC_ERR_ARG, "work buffer too small: %zu < %zu", work_bytes, total);
  static std::mutex mu_streams;
  static cudaStream_t pool[kBatchStreams];
  static cudaEvent_t fork_ev, join_ev[kBatchStreams];
  static bool ready = false;
  std::lock_guard<std::mutex> lk(mu_streams);
  if (!ready) {
    for (int k = 0; k < kBatchStreams; ++k) {
      PVSC_CUDA_TRY(cudaStreamCreateWithFlags(&pool[k], cudaStreamNonBlocking));
      PVSC_CUDA_TRY(cudaEventCreateWithFlags(&join_ev[k], cudaEventDisableTiming));
    }
    PVSC_CUDA_TRY(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    ready = true;
  }
  // the largest lattices first, each on the stream with the least work so far
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return lats[x]->g.n_sites > lats[y]->g.n_sites; });
  LaunchShape force;
  force.kernel = kKernelTma;
  force.threads = bs.threads;
  std::vector<uint64_t> uid = {6, (uint64_t)n, (uint64_t)R, (uint64_t)prec, (uint64_t)M,
                               (uint64_t)(uintptr_t)mu, (uint64_t)(uintptr_t)work, (uint64_t)bs.threads};
  for (int i = 0; i < n; ++i) {
    uint64_t ab[2];
    std::memcpy(&ab[0], &a[i], 8);
    std::memcpy(&ab[1], &b[i], 8);
    uid.insert(uid.end(), {(uint64_t)(uintptr_t)lats[i], lats[i]->generation, seeds[i], ab[0], ab[1]});
  }
  auto body = [&](cudaStream_t cs) -> int {
    PVSC_CUDA_TRY(cudaEventRecord(fork_ev, cs));
    for (int k = 0; k < kBatchStreams; ++k) PVSC_CUDA_TRY(cudaStreamWaitEvent(pool[k], fork_ev, 0));
    double load[kBatchStreams] = {};
    for (int i : order) {
      int k = 0;
      for (int j = 1; j < kBatchStreams; ++j)
        if (load[j] < load[k]) k = j;
      load[k] += (double)lats[i]->g.n_sites;
      if (int rc = kpm_enqueue(lats[i], R, prec, nullptr, seeds[i], M, a[i], b[i], mu + (size_t)i * R * M,
                               static_cast<char*>(work) + off[i], &force, pool[k]))
        return rc;
    }
    for (int k = 0; k < kBatchStreams; ++k) {
      PVSC_CUDA_TRY(cudaEventRecord(join_ev[k], pool[k]));
      PVSC_CUDA_TRY(cudaStreamWaitEvent(cs, join_ev[k], 0));
    }
    return PVSC_OK;
  };
  return run_graph(lats[0], uid, st, body);
}

static int batched_layout(const pvsc_lattice* const* lats, int n, int R, int prec, int M,
                          std::vector<BatchLat>& out, size_t* total, int threads, int zs) {
  const int C = R / vpt_for(R, prec);
  size_t off = batch_header_bytes(n);
  out.assign(n, BatchLat{});
  int64_t unit0 = 0;
  for (int i = 0; i < n; ++i) {
    const pvsc_lattice* lat = lats[i];
    if (!lat) return set_error(PVSC_ERR_ARG, "lattice %d is NULL", i);
    if (lat->g.model != PVSC_TI) return set_error(PVSC_ERR_UNSUPPORTED, "batched KPM takes TI lattices");
    if (lat->g.zhalo) return set_error(PVSC_ERR_UNSUPPORTED, "batched KPM does not take halo lattices");
    BatchLat& L = out[i];
    L.g = lat->g;
    const int64_t plane = lat->g.L[0] * lat->g.L[1], Lz = lat->g.L[2];
    L.nbx = (plane * C + threads - 1) / threads;
    L.zs = (int)(zs <= 0 || Lz < zs ? Lz : zs);
    L.units = L.nbx * ((Lz + L.zs - 1) / L.zs);
    L.unit0 = unit0;
    unit0 += L.units;
    L.wa = reinterpret_cast<void*>(off);  // offsets for now; rebased on the device pointer later
    off += vec_bytes(lat, R, prec);
    L.wb = reinterpret_cast<void*>(off);
    off += vec_bytes(lat, R, prec);
    L.partials = reinterpret_cast<double*>(off);
    off += ((size_t)L.units * 2 * R * sizeof(double) + 255) & ~size_t(255);
  }
  *total = off;
  return PVSC_OK;
}

}  // namespace pvsc

using namespace pvsc;

extern "C" {

int pvsc_debug_inject_stall(int enable) {
  g_inject_stall = enable ? 1 : 0;
  return PVSC_OK;
}

int pvsc_set_wait_limit(uint64_t spins) {
  if (spins == 0) return set_error(PVSC_ERR_ARG, "the wait limit must be at least 1");
  g_wait_limit = spins;
  return PVSC_OK;
}

size_t pvsc_batched_work_bytes(const pvsc_lattice* const* lats, int n, int R, int prec, int M) {
  if (!lats || n < 1 || n > kMaxBatch || !valid_R(R) || (prec != PVSC_C128 && prec != PVSC_C64) || M < 1) return 0;
  std::vector<BatchLat> L;
  size_t total = 0;
  if (!lats[0]) return 0;
  const BatchShape sh = batch_shape(lats[0], R, prec);
  if (sh.per_lattice && per_lattice_possible(lats, n, R, prec)) {
    for (int i = 0; i < n; ++i) total += (per_lattice_bytes(lats[i], R, prec) + 255) & ~size_t(255);
    return total;
  }
  if (batched_layout(lats, n, R, prec, M, L, &total, sh.threads, sh.zs) != PVSC_OK) return 0;
  return total;
}

int pvsc_kpm_moments_batched(const pvsc_lattice* const* lats, int n, int R, int prec,
                             const uint64_t* seeds, int M, const double* a, const double* b,
                             double* mu, void* work, size_t work_bytes, void* stream) {
  if (!lats || n < 1 || n > kMaxBatch)
    return set_error(PVSC_ERR_ARG, "need 1 to %d lattices, got %d", kMaxBatch, n);
  if (!valid_R(R)) return set_error(PVSC_ERR_ARG, "R = %d: must be 1, 2, 4, 8, 16, 32 or 64", R);
  if (prec != PVSC_C128 && prec != PVSC_C64) return set_error(PVSC_ERR_ARG, "unknown precision %d", prec);
  if (M < 1 || !seeds || !a || !b || !mu) return set_error(PVSC_ERR_ARG, "bad M, seeds, a, b or mu");
  for (int i = 0; i < n; ++i)
    if (!(std::isfinite(a[i]) && a[i] > 0) || !std::isfinite(b[i]))
      return set_error(PVSC_ERR_ARG, "scaling of lattice %d invalid", i);
  if (int rc = check_ptr(work, "work")) return rc;
  if (!lats[0]) return set_error(PVSC_ERR_ARG, "lattice 0 is NULL");
  const BatchShape sh = batch_shape(lats[0], R, prec);
  if (sh.per_lattice && per_lattice_possible(lats, n, R, prec)) {
    for (int i = 0; i < n; ++i)
      if (lats[i]->g.model != PVSC_TI || lats[i]->g.zhalo)
        return set_error(PVSC_ERR_UNSUPPORTED, "batched KPM takes TI lattices without halo planes");
    return kpm_per_lattice(lats, n, R, prec, seeds, M, a, b, mu, work, work_bytes, sh,
                           static_cast<cudaStream_t>(stream));
  }
  const int threads = sh.threads;
  std::vector<BatchLat> L;
  size_t total = 0;
  if (int rc = batched_layout(lats, n, R, prec, M, L, &total, threads, sh.zs)) return rc;
  if (work_bytes < total) return set_error(PVSC_ERR_ARG, "work buffer too small: %zu < %zu", work_bytes, total);
  char* base = static_cast<char*>(work);
  int* err = reinterpret_cast<int*>(base);
  unsigned* counters = reinterpret_cast<unsigned*>(base + kWorkHeader);
  for (int i = 0; i < n; ++i) {
    L[i].wa = base + reinterpret_cast<size_t>(L[i].wa);
    L[i].wb = base + reinterpret_cast<size_t>(L[i].wb);
    L[i].partials = reinterpret_cast<double*>(base + reinterpret_cast<size_t>(L[i].partials));
    L[i].arrive = counters + 2 * i;
    L[i].phase = counters + 2 * i + 1;
    L[i].mu = mu + (size_t)i * R * M;
    L[i].a_inv = 1.0 / a[i];
    L[i].b = b[i];
    L[i].key = hash_key(seeds[i], 1);
  }
  const int vpt = vpt_for(R, prec);
  void* fn = prec == PVSC_C128 ? reinterpret_cast<void*>(&kpm_batched_kernel<double, 1>)
             : (vpt == 1 ? reinterpret_cast<void*>(&kpm_batched_kernel<float, 1>)
                         : reinterpret_cast<void*>(&kpm_batched_kernel<float, 2>));
  int occ = 0;
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0));
  if (occ < 1) return set_error(PVSC_ERR_CUDA, "batched kernel cannot be resident");
  const pvsc_lattice* l0 = lats[0];
  int bps = occ;
  if (sh.bps > 0 && sh.bps < occ) bps = sh.bps;
  int64_t grid = (int64_t)l0->sm_count * bps;
  const int64_t total_units = L.back().unit0 + L.back().units;
  if (grid > total_units) grid = total_units;
  // ~30 KB: kept off the host stack; one block shared by all calls, so calls
  // from several host threads take turns from here to the launch (the launch
  // copies the parameters)
  static BatchArgs args;
  static std::mutex args_mu;
  static_assert(sizeof(BatchArgs) <= 32000, "kernel parameter block too large");
  std::lock_guard<std::mutex> args_lock(args_mu);
  std::memset(&args, 0, sizeof(args));
  for (int i = 0; i < n; ++i) args.lats[i] = L[i];
  args.nlat = n;
  args.total_units = total_units;
  args.R = R;
  args.C = R / vpt;
  args.M = M;
  args.nphases = 1 + (M + 1) / 2;
  args.err = err;
  args.wait_limit = g_wait_limit;
  args.inject_stall = g_inject_stall;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<uint64_t> key = {5, (uint64_t)n, (uint64_t)R, (uint64_t)prec, (uint64_t)M,
                               (uint64_t)(uintptr_t)mu, (uint64_t)(uintptr_t)work, g_wait_limit,
                               (uint64_t)grid, (uint64_t)g_inject_stall};
  for (int i = 0; i < n; ++i) {
    uint64_t ab[2];
    std::memcpy(&ab[0], &a[i], 8);
    std::memcpy(&ab[1], &b[i], 8);
    key.insert(key.end(), {(uint64_t)(uintptr_t)lats[i], lats[i]->generation, seeds[i], ab[0], ab[1]});
  }
  auto body = [&](cudaStream_t cs) -> int {
    PVSC_CUDA_TRY(cudaMemsetAsync(base, 0, batch_header_bytes(n), cs));
    void* kargs[] = {&args};
    PVSC_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(threads), kargs, 0, cs));
    return PVSC_OK;
  };
  if (int rc = run_graph(lats[0], key, st, body)) return rc;
  int herr = 0;
  PVSC_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PVSC_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr) return set_error(PVSC_ERR_TIMEOUT, "a batched-KPM wait exceeded %llu spins", g_wait_limit);
  return PVSC_OK;
}

// Launch-shape autotuner of the batched KPM over the whole batch: threads per
// block (and so the vectors per block), z-segment length of the units and
// blocks per SM are timed on the batch itself with a short moment count, and
// the fastest shape becomes the (R, prec) tuning entry of lats[0], which the
// batched calls read.
int pvsc_autotune_batched(pvsc_lattice* const* lats, int n, int R, int prec, const uint64_t* seeds,
                          int M, const double* a, const double* b, pvsc_tuning* best, void* stream) {
  if (!lats || n < 1 || n > kMaxBatch || !lats[0])
    return set_error(PVSC_ERR_ARG, "need 1 to %d lattices", kMaxBatch);
  if (!valid_R(R)) return set_error(PVSC_ERR_ARG, "R = %d: must be 1, 2, 4, 8, 16, 32 or 64", R);
  if (prec != PVSC_C128 && prec != PVSC_C64) return set_error(PVSC_ERR_ARG, "unknown precision %d", prec);
  if (M < 2 || !seeds || !a || !b) return set_error(PVSC_ERR_ARG, "need M >= 2, seeds, a and b");
  pvsc_lattice* l0 = lats[0];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int C = R / vpt_for(R, prec);
  int64_t Lzmax = 1;
  for (int i = 0; i < n; ++i) {
    if (!lats[i]) return set_error(PVSC_ERR_ARG, "lattice %d is NULL", i);
    Lzmax = std::max<int64_t>(Lzmax, lats[i]->g.L[2]);
  }
  std::vector<pvsc_tuning> cands;
  for (int th : {128, 256})
    if (th % C == 0)
      for (int zs : {0, 16, 24, 32, 48, 64})
        if (zs == 0 || zs < Lzmax)
          for (int bps : {0, 1}) cands.push_back(pvsc_tuning{th, bps, zs, 0.f, 0, 0, 0, 0});
  // every lattice's KPM on the TMA-staged sweep, in concurrent chains
  if (per_lattice_possible(lats, n, R, prec))
    for (int th : {256, 512}) cands.push_back(pvsc_tuning{th, 0, 0, 0.f, 0, 0, 0, kKernelTma});
  auto saved = l0->tuning.find({R, prec});
  const bool had = saved != l0->tuning.end();
  const pvsc_tuning old = had ? saved->second : pvsc_tuning{};
  size_t wmax = 0;
  for (const pvsc_tuning& c : cands) {
    l0->tuning[{R, prec}] = c;
    wmax = std::max(wmax, pvsc_batched_work_bytes(lats, n, R, prec, M));
  }
  void *work = nullptr, *mu = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(work);
    cudaFree(mu);
  };
  int rc = PVSC_OK;
  if (wmax == 0 || cudaMalloc(&work, wmax) != cudaSuccess ||
      cudaMalloc(&mu, sizeof(double) * (size_t)n * R * M) != cudaSuccess) {
    cleanup();
    if (had) l0->tuning[{R, prec}] = old; else l0->tuning.erase({R, prec});
    return set_error(PVSC_ERR_OOM, "batched autotune could not allocate its buffers");
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  pvsc_tuning win{256, 0, 0, 1e30f, 0, 0, 0, 0};
  for (const pvsc_tuning& c : cands) {
    l0->tuning[{R, prec}] = c;
    drop_graphs(l0);
    const size_t wb = pvsc_batched_work_bytes(lats, n, R, prec, M);
    double* mp = static_cast<double*>(mu);
    if ((rc = pvsc_kpm_moments_batched(lats, n, R, prec, seeds, M, a, b, mp, work, wb, stream)) != PVSC_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e0, st) != cudaSuccess) { rc = set_error(PVSC_ERR_CUDA, "event record failed"); break; }
    if ((rc = pvsc_kpm_moments_batched(lats, n, R, prec, seeds, M, a, b, mp, work, wb, stream)) != PVSC_OK) break;
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < win.time_ms) {
      win = c;
      win.time_ms = ms;
    }
  }
  cleanup();
  if (rc != PVSC_OK) {
    if (had) l0->tuning[{R, prec}] = old; else l0->tuning.erase({R, prec});
    drop_graphs(l0);
    return rc;
  }
  l0->tuning[{R, prec}] = win;
  drop_graphs(l0);
  if (best) *best = win;
  return PVSC_OK;
}

}  // extern "C"
