// Shared-memory staged TI sweep (2.5D blocking with the bulk-copy engine).
//
// Each block owns a tile of TX x TY columns of the cubic lattice and marches
// it through a z-slab.  Plane z of the tile, with its one-site halo in x and
// y (all 4 orbitals x R vectors of every site), lives in one slot of a 4-slot
// shared-memory ring; planes z-1, z, z+1 are resident while the cp.async.bulk
// (TMA engine) copies of planes z+2 and z+3 are in flight.  The y_in tile of
// plane z rides in the same copy group as x plane z+1 (a second 4-slot ring),
// and the potential of plane z+1 is prefetched into a 2-slot buffer while
// plane z is computed, so the compute loop issues no global load it waits on.
// Every site row of a tile is contiguous in global memory (sites are x-fast,
// the orbital x vector data of a site is contiguous), so one halo row is one
// bulk copy, plus one single-site copy where a periodic axis wraps.  Copy
// completion is tracked with one mbarrier per slot (expect_tx / complete_tx);
// every wait is bounded.
//
// Thread t updates vector r = t mod R of tile sites t / R, t / R + blockDim/R,
// ..., so a warp reads consecutive vectors of a site (conflict-free) and
// stores y_new with the coalescing of the input layout.  HBM sees each x
// element once per sweep (halo rows are shared with neighbouring tiles
// through L2).
#pragma once

#include "sweep.cuh"

namespace pvsc {

struct BulkSmem {
  static __host__ __device__ size_t plane_bytes(int TX, int TY, int R, int csize) {
    return (size_t)(TX + 2) * (TY + 2) * 4 * R * csize;
  }
  static __host__ __device__ size_t ytile_bytes(int TX, int TY, int R, int csize) {
    return (size_t)TX * TY * 4 * R * csize;
  }
  static __host__ __device__ size_t total(int TX, int TY, int R, int csize) {
    return 4 * plane_bytes(TX, TY, R, csize) + 4 * ytile_bytes(TX, TY, R, csize) +
           2 * (size_t)TX * TY * sizeof(double) + 64;
  }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait on one slot barrier; every thread polls.  Returns false (for
// the whole block) if the copy did not complete within `limit` polls.
__device__ __forceinline__ bool block_wait_slot(uint64_t* bar, unsigned parity, unsigned limit) {
  bool done = false;
  for (unsigned n = 0; n < limit && !done; ++n) done = mbar_try_wait(bar, parity);
  return __syncthreads_and(done) != 0;
}

constexpr unsigned kBulkWaitLimit = 1u << 24;

// Device error word of the staged sweep (one per translation unit): set if a
// copy wait ran out; read and cleared through pvsc_device_error.
static __device__ int g_bulk_sweep_error;

template <typename T, int FEAT>
__global__ void __launch_bounds__(256) ti_sweep_bulk(const __grid_constant__ Sweep p) {
  using C2 = typename CT<T>::c;
  extern __shared__ __align__(128) unsigned char smem[];
  const int TX = p.tile_x, TY = p.tile_y;
  const int R = p.R;
  const int64_t Lx = p.g.L[0], Ly = p.g.L[1], Lz = p.g.L[2];
  const int64_t plane = Lx * Ly;
  const int csize = 2 * (int)sizeof(T);
  const int SB = 4 * R * csize;  // bytes of one site (4 orbitals x R vectors)
  const size_t PB = BulkSmem::plane_bytes(TX, TY, R, csize);
  const size_t YB = BulkSmem::ytile_bytes(TX, TY, R, csize);
  unsigned char* slots = smem;
  unsigned char* yslots = smem + 4 * PB;
  double* vslots = reinterpret_cast<double*>(yslots + 4 * YB);
  uint64_t* bars = reinterpret_cast<uint64_t*>(vslots + 2 * TX * TY);
  const T* __restrict__ X = static_cast<const T*>(p.x);
  const T* __restrict__ Yin = static_cast<const T*>(p.yin);
  const int r = threadIdx.x % R;
  const int site_step = blockDim.x / R;
  if (threadIdx.x == 0)
    for (int s = 0; s < 4; ++s) mbar_init(&bars[s], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  const VecCoef<T, 1> cf = load_coef<T, 1>(p, r);
  DotAcc<T, 1> dacc;
  dacc.init();

  const int64_t ntx = (Lx + TX - 1) / TX, nty = (Ly + TY - 1) / TY;
  const int zs = p.zslab;
  const int64_t nzs = (Lz + zs - 1) / zs;
  const int64_t nunits = ntx * nty * nzs;
  unsigned phase_bits = 0;  // expected parity of each slot's next completion
  unsigned issued = 0;      // slots with a copy group in flight
  bool failed = false;

  for (int64_t u = blockIdx.x; u < nunits && !failed; u += gridDim.x) {
    const int64_t bz = u / (ntx * nty);
    const int64_t rem = u - bz * ntx * nty;
    const int64_t y0 = (rem / ntx) * TY, x0 = (rem % ntx) * TX;
    const int TXe = (int)min((int64_t)TX, Lx - x0), TYe = (int)min((int64_t)TY, Ly - y0);
    const int64_t z0 = bz * zs, z1 = min(z0 + (int64_t)zs, Lz);
    const int n = (int)(z1 - z0);
    const int nsite = TXe * TYe;
    // loaded plane j (0 .. n+1) is lattice plane z0 - 1 + j, wrapped or absent
    auto plane_of = [&](int j) -> int64_t {
      const int64_t zz = z0 - 1 + j;
      if (zz >= 0 && zz < Lz) return zz;
      if (!p.g.per[2]) return -1;
      return (zz + Lz) % Lz;
    };
    // copy group j: x plane j (with halo) and, for 2 <= j <= n+1, the y_in tile
    // of plane z0 + j - 2; issued by warp 0 into slot j % 4
    auto issue = [&](int j) {
      const int64_t pz = plane_of(j);
      const bool with_y = Yin != nullptr && j >= 2 && j <= n + 1;
      if (pz < 0 && !with_y) return;
      const int slot = j & 3;
      issued |= 1u << slot;
      if (threadIdx.x >= 32) return;
      const int lane = threadIdx.x;
      unsigned char* base = slots + slot * PB;
      unsigned char* ybase = yslots + slot * YB;
      const int64_t yz = z0 + j - 2;
      const int c_lo = x0 > 0 ? 0 : 1;
      const int c_hi = (x0 + TXe < Lx) ? TXe + 2 : TXe + 1;
      const bool wrap_lo = x0 == 0 && p.g.per[0], wrap_hi = x0 + TXe == Lx && p.g.per[0];
      for (int pass = 0; pass < 2; ++pass) {
        unsigned bytes = 0;
        if (pz >= 0)
          for (int jr = lane; jr < TYe + 2; jr += 32) {
            int64_t gy = y0 - 1 + jr;
            if (gy < 0 || gy >= Ly) {
              if (!p.g.per[1]) continue;
              gy = (gy + Ly) % Ly;
            }
            const char* grow = reinterpret_cast<const char*>(X) + ((pz * Ly + gy) * Lx) * (int64_t)SB;
            unsigned char* srow = base + (size_t)jr * (TX + 2) * SB;
            const unsigned run = (unsigned)(c_hi - c_lo) * SB;
            if (pass == 0) {
              bytes += run + (wrap_lo ? SB : 0) + (wrap_hi ? SB : 0);
            } else {
              bulk_g2s(srow + (size_t)c_lo * SB, grow + (x0 - 1 + c_lo) * (int64_t)SB, run, &bars[slot]);
              if (wrap_lo) bulk_g2s(srow, grow + (Lx - 1) * (int64_t)SB, SB, &bars[slot]);
              if (wrap_hi) bulk_g2s(srow + (size_t)(TXe + 1) * SB, grow, SB, &bars[slot]);
            }
          }
        if (with_y)
          for (int jr = lane; jr < TYe; jr += 32) {
            const char* grow = reinterpret_cast<const char*>(Yin) + ((yz * Ly + y0 + jr) * Lx + x0) * (int64_t)SB;
            if (pass == 0) bytes += (unsigned)TXe * SB;
            else bulk_g2s(ybase + (size_t)jr * TX * SB, grow, (unsigned)TXe * SB, &bars[slot]);
          }
        if (pass == 0) {
          // announce the group's bytes before any copy of it is issued
#pragma unroll
          for (int off = 16; off >= 1; off >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, off);
          if (lane == 0) mbar_arrive_expect_tx(&bars[slot], bytes);
          __syncwarp();
        }
      }
    };
    auto wait_slot = [&](int j) -> bool {
      const int slot = j & 3;
      if (!(issued & (1u << slot))) return true;  // nothing in this group
      const bool ok = block_wait_slot(&bars[slot], (phase_bits >> slot) & 1u, kBulkWaitLimit);
      if (ok) {
        phase_bits ^= 1u << slot;
        issued &= ~(1u << slot);
      }
      return ok;
    };
    const int prolog = min(n + 2, 4);
    for (int j = 0; j < prolog; ++j) issue(j);
    for (int t = threadIdx.x; t < nsite; t += blockDim.x)
      vslots[t] = site_potential(p.g, plane * z0 + (y0 + t / TXe) * Lx + x0 + t % TXe);
    if (!wait_slot(0) || !wait_slot(1)) { failed = true; break; }
    for (int i = 0; i < n; ++i) {
      if (!wait_slot(i + 2)) { failed = true; break; }
      const int64_t z = z0 + i;
      // prefetch the potential of plane z+1 (stored after the compute)
      double vnext[2] = {0.0, 0.0};
      if (i + 1 < n)
        for (int k = 0, t = threadIdx.x; k < 2 && t < nsite; ++k, t += blockDim.x)
          vnext[k] = site_potential(p.g, plane * (z + 1) + (y0 + t / TXe) * Lx + x0 + t % TXe);
      const unsigned char* Pm = slots + ((i) & 3) * PB;      // plane z-1
      const unsigned char* Pc = slots + ((i + 1) & 3) * PB;  // plane z
      const unsigned char* Pp = slots + ((i + 2) & 3) * PB;  // plane z+1
      const unsigned char* Yt = yslots + ((i + 2) & 3) * YB;  // y_in of plane z
      const double* Vt = vslots + (i & 1) * TX * TY;
      const bool hzm = plane_of(i) >= 0, hzp = plane_of(i + 2) >= 0;
      for (int ts = threadIdx.x / R; ts < nsite; ts += site_step) {
        const int tx = ts % TXe, ty = ts / TXe;
        const int64_t gx = x0 + tx, gy = y0 + ty;
        const int64_t s = plane * z + gy * Lx + gx;
        const bool hxm = gx > 0 || p.g.per[0], hxp = gx < Lx - 1 || p.g.per[0];
        const bool hym = gy > 0 || p.g.per[1], hyp = gy < Ly - 1 || p.g.per[1];
        const int cc = (ty + 1) * (TX + 2) + (tx + 1);  // cell of the site in a plane slot
        auto cell = [&](const unsigned char* P, int c, int o) -> cplx<T> {
          const C2 q = reinterpret_cast<const C2*>(P + (size_t)c * SB)[o * R + r];
          return {q.x, q.y};
        };
        const T Vs = T(Vt[ts]);
        Blk<T, 1> xc, S, D;
        cplx<T> am[4], ap[4];
        const cplx<T> zero{T(0), T(0)};
        // z axis
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          xc.v[o][0] = cell(Pc, cc, o);
          am[o] = hzm ? cell(Pm, cc, o) : zero;
          ap[o] = hzp ? cell(Pp, cc, o) : zero;
        }
        {
          cplx<T> d[4];
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            S.v[o][0] = cadd(am[o], ap[o]);
            d[o] = csub(am[o], ap[o]);
          }
          D.v[0][0] = d[1];
          D.v[1][0] = {-d[0].re, -d[0].im};
          D.v[2][0] = d[3];
          D.v[3][0] = {-d[2].re, -d[2].im};
        }
        // x axis
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          am[o] = hxm ? cell(Pc, cc - 1, o) : zero;
          ap[o] = hxp ? cell(Pc, cc + 1, o) : zero;
        }
        {
          cplx<T> d[4];
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            S.v[o][0] = cadd(S.v[o][0], cadd(am[o], ap[o]));
            d[o] = csub(am[o], ap[o]);
          }
          D.v[0][0] = cadd(D.v[0][0], d[3]);
          D.v[1][0] = cadd(D.v[1][0], d[2]);
          D.v[2][0] = csub(D.v[2][0], d[1]);
          D.v[3][0] = csub(D.v[3][0], d[0]);
        }
        // y axis: -i d = (d.im, -d.re)
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          am[o] = hym ? cell(Pc, cc - (TX + 2), o) : zero;
          ap[o] = hyp ? cell(Pc, cc + (TX + 2), o) : zero;
        }
        {
          cplx<T> d[4];
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            S.v[o][0] = cadd(S.v[o][0], cadd(am[o], ap[o]));
            d[o] = csub(am[o], ap[o]);
          }
          D.v[0][0] = cadd(D.v[0][0], cplx<T>{d[3].im, -d[3].re});
          D.v[1][0] = cadd(D.v[1][0], cplx<T>{d[2].im, -d[2].re});
          D.v[2][0] = cadd(D.v[2][0], cplx<T>{d[1].im, -d[1].re});
          D.v[3][0] = cadd(D.v[3][0], cplx<T>{d[0].im, -d[0].re});
        }
        Blk<T, 1> yn;
        {
          const T e = fma(cf.alpha[0], Vs, -cf.ab[0]);
          const T dp = e + cf.am[0], dm = e - cf.am[0];
          const int yc = ty * TX + tx;  // cell of the site in a y_in tile
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const T dd = (o & 1) ? dm : dp;
            const cplx<T> Tt = (o & 1) ? csub(D.v[o][0], S.v[o][0]) : cadd(D.v[o][0], S.v[o][0]);
            T re = fma(cf.kt[0], Tt.re, dd * xc.v[o][0].re);
            T im = fma(cf.kt[0], Tt.im, dd * xc.v[o][0].im);
            if (Yin != nullptr) {
              const cplx<T> yv = cell(Yt, yc, o);
              re = fma(cf.gamma[0], yv.re, re);
              im = fma(cf.gamma[0], yv.im, im);
            }
            yn.v[o][0] = {re, im};
          }
          if (p.g.has_delta) ti_add_delta(p.g, cf, xc, yn);
        }
        const int64_t sites[4] = {s, s, s, s};
        epilogue<T, 1, FEAT>(p, s, r, xc, yn, dacc, sites);
      }
      if (i + 1 < n) {
        double* Vn = vslots + ((i + 1) & 1) * TX * TY;
        for (int k = 0, t = threadIdx.x; k < 2 && t < nsite; ++k, t += blockDim.x) Vn[t] = vnext[k];
      }
      __syncthreads();  // slots of plane z-1 and y_in(z-... ) free; V of plane z+1 visible
      if (i + 4 < n + 2) issue(i + 4);
    }
    if (failed) break;
  }
  if (failed) {
    // drain: wait (bounded) for the copies this block still has in flight, then leave
    for (int slot = 0; slot < 4; ++slot) {
      if (!(issued & (1u << slot))) continue;
      for (unsigned k = 0; k < kBulkWaitLimit && !mbar_try_wait(&bars[slot], (phase_bits >> slot) & 1u); ++k) {
      }
    }
    if (threadIdx.x == 0) atomicExch(&g_bulk_sweep_error, 1);
    return;
  }
  if constexpr (has_dots(FEAT)) {
    dacc.flush();
    reduce_dots<1>(p, dacc.d);
  }
}

}  // namespace pvsc
