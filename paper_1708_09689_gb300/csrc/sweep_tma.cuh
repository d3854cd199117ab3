// TI sweep with tensor-memory-accelerator (TMA) staging of z-plane tiles
// (tuning kernel 7; kernel 8 marches the same tiles along x), complex64
// storage, R = 1 .. 64; the same kernel carries the Weyl-semimetal cells and
// the fixed-point (PVSC_Q64) KPM sweep.
//
// The stencil of Eq. TB_H_topi reads every x element of a plane seven times
// (the site itself and its six neighbours).  Here a block owns a tile of
// TX x TY columns and marches it along z.  Per plane, cp.async.bulk.tensor
// copies bring the tile of x with its four one-site halo strips (x-/x+
// columns, y-/y+ rows; no corners, the stencil has none) and, per updated
// plane, the tile of y_in and of the fp32 potential into shared memory: a ring
// of x planes and a ring of y_in planes, deep enough to keep three planes of
// copies (about 130 KB per SM) in flight.  Eight warps take all six neighbours
// and y_in from shared memory and keep only x(z-1) of their sites in
// registers, so no register waits on HBM.  Each slot has a full mbarrier
// (copy bytes) and a release count: the warp that releases a slot last issues
// the copy that refills it, so no thread ever blocks waiting for a free slot.
// Halo strips are taken with the wrapped coordinate on a periodic axis and read
// zeros past an open edge (the copy's out-of-range fill), so one code path
// serves every boundary mix and partial tiles.
//
// Shared-memory layout: the x and y_in tiles use the 128-byte swizzle (the
// 16-byte chunk index of every 128-byte row XORed with the row index modulo
// 8).  A thread owns two vectors (16 bytes per orbital) of one site; R/2
// threads share a site, and the sites of a warp are permuted so that the 8
// threads of every quarter-warp hit 8 distinct bank groups for the centre,
// x+-1, y+-1 and z+1 blocks alike (conflict-free 128-bit shared loads).
// R = 1, 2: a copied row is one 32- or 64-byte site under the 32- or 64-byte
// swizzle and one thread owns a site; R = 32, 64: slices of 16 vectors.
//
// Work units are (z-chunk, tile) pairs taken in wave order (tiles fastest),
// unit u on block u mod grid: the grid (one block per SM) works on adjacent
// tiles at the same depth, so halo strips that another tile also reads come
// from L2; the planes of the units after the last full wave are split evenly
// over the grid.  The arithmetic, its order and the epilogue are those of the
// register z-march (ti_axes / ti_combine / epilogue of sweep.cuh), so the
// vectors equal that sweep's bit for bit.
//
// Every mbarrier wait is bounded: a wait that runs out sets a device error
// word (read by pvsc_device_error) and a block-wide abort flag; every warp then
// leaves its loop, one thread waits (bounded) for the copies still in flight,
// and the block finishes without touching the output further.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <type_traits>

#include "fx_arith.cuh"
#include "internal.h"
#include "sweep_bulk.cuh"

namespace pvsc {

constexpr unsigned kTmaWaitLimit = 1u << 24;
constexpr int kTmaMaxUnits = 512;  // work units of one block (a table in shared memory)
constexpr int kTmaUnitsPerSm = kTmaMaxUnits - 4;  // whole-column units per SM the launch checks allow

// Tile of TX x TY sites per R: 256 (site, vector pair) items, one per thread,
// and NXS x-plane / NYS y_in-plane ring slots: three planes of copies in flight
// beyond the two x planes and the y_in plane being read (DEEP = true).
// DEEP = false: twice the tile (512 items, two per thread) with two planes of
// copies in flight.  R = 1, 2: one thread per site (sites of 32 and 64 bytes).
// R = 32, 64 run as slices of 16 vectors on the tiles of R = 16.
template <int R, bool DEEP> struct TmaTile;
template <> struct TmaTile<1, true> { static constexpr int TX = 32, TY = 16, NXS = 5, NYS = 4; };
template <> struct TmaTile<2, true> { static constexpr int TX = 32, TY = 8, NXS = 5, NYS = 4; };
template <> struct TmaTile<1, false> { static constexpr int TX = 32, TY = 32, NXS = 3, NYS = 2; };
template <> struct TmaTile<2, false> { static constexpr int TX = 32, TY = 16, NXS = 3, NYS = 2; };
template <> struct TmaTile<4, true> { static constexpr int TX = 16, TY = 8, NXS = 5, NYS = 4; };
template <> struct TmaTile<8, true> { static constexpr int TX = 16, TY = 4, NXS = 5, NYS = 4; };
template <> struct TmaTile<16, true> { static constexpr int TX = 8, TY = 4, NXS = 5, NYS = 4; };
template <> struct TmaTile<4, false> { static constexpr int TX = 16, TY = 16, NXS = 3, NYS = 2; };
template <> struct TmaTile<8, false> { static constexpr int TX = 16, TY = 8, NXS = 3, NYS = 2; };
template <> struct TmaTile<16, false> { static constexpr int TX = 8, TY = 8, NXS = 3, NYS = 2; };

constexpr int round_up_1k(int b) { return (b + 1023) & ~1023; }

// VF: 4-byte words of potential data per tile point that a y stage holds room
// for (two fp32 potentials of a Weyl cell; the fixed-point sweep's (d+, d-) pair
// of 64-bit coefficients takes four).
template <int R, bool DEEP, int NW, int VF = 2>
struct TmaLayout {
  static constexpr int NWARPS = NW;  // warps per block (8 or 16), one block per SM
  static constexpr int TX = TmaTile<R, DEEP>::TX, TY = TmaTile<R, DEEP>::TY;
  static constexpr int SITE_B = 32 * R;          // 4 orbitals x R complex64
  static constexpr int ROWB = SITE_B < 128 ? SITE_B : 128;  // bytes of a copied row (the swizzle span)
  static constexpr int ROWS = SITE_B / ROWB;     // rows per site
  static constexpr int CPS = R >= 2 ? R / 2 : 1;  // threads per site
  static constexpr int SPW = 32 / CPS;           // sites per warp
  static constexpr int ITEMS = TX * TY * CPS;
  static constexpr int IPT = ITEMS / (32 * NW);  // items per thread
  static constexpr int INT_B = TX * TY * SITE_B;  // interior tile
  static constexpr int XS_B = TY * SITE_B;        // x-/x+ halo column
  static constexpr int YS_B = TX * SITE_B;        // y-/y+ halo row
  static constexpr int OFF_XM = INT_B, OFF_XP = INT_B + XS_B;
  static constexpr int OFF_YM = INT_B + 2 * XS_B, OFF_YP = INT_B + 2 * XS_B + YS_B;
  static constexpr int X_BYTES = INT_B + 2 * XS_B + 2 * YS_B;  // copied per x plane
  static constexpr int XSTAGE = round_up_1k(X_BYTES);
  static constexpr int V_B = TX * TY * 4;                  // fp32 potential per tile point
  static constexpr int YSTAGE = INT_B + round_up_1k(VF * V_B);
  static constexpr int NXS = TmaTile<R, DEEP>::NXS, NYS = TmaTile<R, DEEP>::NYS;
  static constexpr int BAR_OFF = NXS * XSTAGE + NYS * YSTAGE;
  static constexpr int DOT_OFF = BAR_OFF + 128;  // fp64 dot partials [warp][dot][v][c]
  static constexpr int DOT_B = NW * 4 * 2 * CPS * 8;
  static constexpr int TAB_OFF = DOT_OFF + DOT_B;  // the block's units: (x0 | y0 << 16, z0 | n << 16)
  static constexpr int TAB_B = kTmaMaxUnits * 8;
  static constexpr size_t SMEM = 1024 + (size_t)TAB_OFF + TAB_B;  // + alignment slack
  static_assert(IPT >= 1 && ITEMS % (32 * NW) == 0, "tile items");
  static_assert(NXS >= 3 && NYS >= 2, "ring depth");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// The tensor maps of one launch (kernel parameter, 64-byte aligned entries).
struct TmaMaps {
  CUtensorMap xi;   // x: interior tile box {32, ROWS, TX, TY, 1}
  CUtensorMap xs;   // x: halo column box {32, ROWS, 1, TY, 1}
  CUtensorMap ys;   // x: halo row box {32, ROWS, TX, 1, 1}
  CUtensorMap yi;   // y_in: interior tile box
  CUtensorMap v;    // fp32 potential: box {TX, TY, 1}
  int has_yin;      // y_in present (gamma != 0)
  int v_tma;        // potential copied with the y_in tile (stored potential)
  int nch;          // z-chunks per column
  int ntx, nty;     // tiles along x and y
  long long nunits;
};

static __device__ int g_tma_sweep_error;

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// Shared-memory counter increment with acquire-release ordering at block
// scope: a warp's reads of a ring slot happen before its release count, and
// the warp that brings the count to completion sees all of them before it
// refills the slot.
__device__ __forceinline__ unsigned release_count(unsigned* ctr) {
  unsigned old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(smem_addr(ctr)) : "memory");
  return old;
}

// L2 prefetch of one global line (a hint; the address is a valid element).
__device__ __forceinline__ void prefetch_l2(const void* ptr) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Bounded wait for the phase of the given parity; false if it ran out or the
// block is aborting.
__device__ __forceinline__ bool tma_wait(uint64_t* bar, unsigned parity, volatile int* abort) {
  for (unsigned n = 0; n < kTmaWaitLimit; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 255u) == 255u && *abort) return false;
  }
  atomicExch(&g_tma_sweep_error, 1);
  *abort = 1;
  return false;
}

// Site of a tile owned by quarter-warp slot q of a warp: consecutive sites in
// one quarter-warp would meet the same bank group under the 128-byte swizzle
// whenever their rows agree modulo 8; this permutation spreads them.
template <int R>
__device__ __forceinline__ int tma_site_perm(int q) {
  if constexpr (R >= 16 || R <= 2) {
    return q;  // one site per quarter-warp, or consecutive sites under the 64 / 32-byte swizzle
  } else if constexpr (R == 8) {
    return (q & 4) | ((q & 1) << 1) | ((q >> 1) & 1);  // quarter-warp: sites a, a + 2
  } else {
    const int ph = q >> 2, i = q & 3;  // quarter-warp: sites a, a + 2, a + 4, a + 6
    return ((ph >> 1) << 3) + (ph & 1) + 2 * i;
  }
}

// Swizzled offset of the 16-byte chunk of vectors (2c, 2c+1), orbital 0, of the
// site at byte offset O (a multiple of 32 R) in a tile buffer: the logical
// offset L = O + 16 c with its chunk bits XORed with its row bits.  Orbital o
// then sits at (B ^ (K_o << 4)) + (its row offset) with the compile-time K of
// tma_lds_blk (the row offset of orbital o modulo 8 never carries into the row
// bits of L for R = 4 .. 64).  SWZ = false: tiles copied without swizzle
// (the logical offset itself).
template <int R, bool SWZ = true>
__device__ __forceinline__ uint32_t tma_swz(uint32_t O, int c) {
  const uint32_t L = O + 16u * (uint32_t)c;
  if constexpr (!SWZ) return L;
  // the swizzle of the copy: 128-byte (R >= 4), 64-byte (R = 2) or 32-byte (R = 1)
  // span, the 16-byte chunk bits XORed with the bits above bit 7
  constexpr uint32_t MASK = R >= 4 ? 7u : (R == 2 ? 3u : 1u);
  return L ^ (((L >> 7) & MASK) << 4);
}

// All four orbitals (two vectors each) of one site from a swizzled tile
// buffer: buf = the buffer (1024-byte aligned), B = tma_swz of the site.
// Plain shared-memory loads, so that the compiler schedules them; the
// mbarrier waits (asm volatile with a memory clobber) order them after the copies.
template <int R>
__device__ __forceinline__ void tma_lds_blk(const unsigned char* buf, uint32_t B, Blk<float, 2>& b) {
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int ao = o * 8 * R;                      // byte offset of orbital o in the site
    const int K1 = (ao >> 4) & 7, K2 = (ao >> 7) & 7;
    const float4 v = *reinterpret_cast<const float4*>(buf + ((B ^ (uint32_t)((K1 ^ K2) << 4)) + (uint32_t)(ao & ~127)));
    b.v[o][0] = {v.x, v.y};
    b.v[o][1] = {v.z, v.w};
  }
}

// One vector (R = 1): the 32-byte site is two chunks, orbitals (0, 1) and
// (2, 3); under the 32-byte swizzle chunk k sits at B ^ 16 k.
template <int R>
__device__ __forceinline__ void tma_lds_blk(const unsigned char* buf, uint32_t B, Blk<float, 1>& b) {
  static_assert(R == 1, "one vector per site");
  const float4 v0 = *reinterpret_cast<const float4*>(buf + B);
  const float4 v1 = *reinterpret_cast<const float4*>(buf + (B ^ 16u));
  b.v[0][0] = {v0.x, v0.y};
  b.v[1][0] = {v0.z, v0.w};
  b.v[2][0] = {v1.x, v1.y};
  b.v[3][0] = {v1.z, v1.w};
}

// The same four orbitals of a fixed-point block: a site of R/2 vectors of
// 16-byte (re, im) 64-bit pairs has the byte layout of a complex64 site of R
// vectors, and vector c is the 16-byte chunk c of every orbital.  SWZ = false
// (unswizzled tiles): orbital o at B + its offset, an immediate of the load.
template <int R, bool SWZ = true>
__device__ __forceinline__ void tma_lds_blk(const unsigned char* buf, uint32_t B, Blk<long long, 1>& b) {
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int ao = o * 8 * R;
    const int K1 = (ao >> 4) & 7, K2 = (ao >> 7) & 7;
    const uint32_t off = SWZ ? (B ^ (uint32_t)((K1 ^ K2) << 4)) + (uint32_t)(ao & ~127) : B + (uint32_t)ao;
    const longlong2 v = *reinterpret_cast<const longlong2*>(buf + off);
    b.v[o][0] = {v.x, v.y};
  }
}

// MODEL 1: TI sites; MODEL 3: Weyl-semimetal cells of two x-adjacent sites
// (Eq. TB_H_wsm), whose four components form the same block as a TI site, with
// the cell update of the Weyl sweeps and two potentials per cell;
// kModelTIFx: the TI KPM sweep of sweep_fx.cu on fixed-point vectors (R/2
// vectors in the byte layout of R complex64 vectors, one vector per thread,
// the per-site coefficient pair in place of the potential, exact dot sums).
// SL > 1: the block of R SL vectors is swept as SL slices of R vectors
// (R = 16, the layout of the 8 x 8 tiles): block b takes slice b mod SL
// (the grid is a multiple of SL), whose 128-byte rows the tensor maps select
// by their innermost coordinate, and the units b / SL + lu G / SL of that
// slice; the epilogue addresses the whole block.
// XM (TI sites or Weyl cells, complex64): march along the lattice's x axis: the kernel's tile axes
// (X, Y) and march axis Z are the lattice's (y, z) and x (the tensor maps take
// the permuted strides), for lattices whose z columns are short; the neighbour
// pairs are folded in the z-march's order (z, x, y), so the vectors stay equal
// to the z-march's bit for bit; the potential is read per site (its plane is
// not a tile of a contiguous row).
template <int R, bool DEEP, int NW, int FEAT, int MODEL, int SL = 1, bool XM = false>
__global__ void __launch_bounds__(32 * NW, 1)
    ti_sweep_tma(const __grid_constant__ Sweep p, const __grid_constant__ TmaMaps m) {
  static_assert(SL == 1 || R == 16, "vector slices of 16 complex64 (8 fixed-point) vectors");
  static_assert(!XM || MODEL == PVSC_TI || MODEL == PVSC_WSM, "marching along x: TI sites or Weyl cells");
  constexpr int RF = R * SL;  // vectors (complex64 layout) of the whole block
  constexpr int VP = R == 1 ? 1 : 2;  // complex64 vectors per thread (R = 1: one per site)
  constexpr bool WSM = MODEL == 3;
  constexpr bool FX = MODEL == kModelTIFx;
  // fixed point with R/2 >= 8 vectors: a quarter-warp reads one whole 128-byte
  // row of an orbital, conflict-free without the swizzle (no XOR per load)
  constexpr bool SWZ = !(FX && R >= 16);
  constexpr int VPC = WSM ? 2 : 1;               // sites per tile point
  constexpr int VF = WSM ? 2 : (FX ? 4 : 1);     // 4-byte words of potential data per tile point
  using L = TmaLayout<R, DEEP, NW, FX ? 4 : 2>;
  constexpr int NCW = NW, IPT = L::IPT, TX = L::TX, TY = L::TY;
  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_abort;
  __shared__ unsigned s_cnt[L::NXS + L::NYS];  // releases per slot (x slots, then y slots)
  __shared__ unsigned s_issued[2];             // x, y copies issued
  const uint32_t raw = smem_addr(smem_raw);
  unsigned char* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sbase = smem_addr(base);
  uint64_t* full_x = reinterpret_cast<uint64_t*>(base + L::BAR_OFF);
  uint64_t* full_y = full_x + L::NXS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Programmatic dependent launch (when the host launches with it): the next
  // sweep on the stream may start its blocks now, on SMs this grid leaves free
  // or frees; they set up their barriers and unit tables and then wait at
  // griddepcontrol.wait below for this grid to complete.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < L::NXS; ++s) mbar_init(&full_x[s], 1);
    for (int s = 0; s < L::NYS; ++s) mbar_init(&full_y[s], 1);
    for (int s = 0; s < L::NXS + L::NYS; ++s) s_cnt[s] = 0;
    s_issued[0] = s_issued[1] = 0;
    s_abort = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  const Geometry& g = p.g;
  // the kernel's tile axes X, Y and march axis Z: the lattice's (x, y, z) (x in
  // tile points), or (y, z, x) when marching along x
  const int LX = (int)(g.L[0] / VPC), LY = (int)g.L[1], LZ = (int)g.L[2];
  const int Lx = XM ? LY : LX, Ly = XM ? LZ : LY, Lz = XM ? LX : LZ;
  const int perX = XM ? g.per[1] : g.per[0], perY = XM ? g.per[2] : g.per[1], perZ = XM ? g.per[0] : g.per[2];
  const int64_t plane = XM ? 1 : (int64_t)Lx * Ly;  // site stride of one step along Z
  const int sl = SL > 1 ? (int)(blockIdx.x % SL) : 0;  // this block's vector slice
  const int vb = SL > 1 ? (int)(blockIdx.x / SL) : (int)blockIdx.x;
  const int G = gridDim.x / SL;  // blocks per slice
  const int c0 = 32 * sl;       // the slice's rows: innermost tensor-map coordinate
  volatile int* abort = &s_abort;
  // This block's units, decoded once into a shared table (x0 | y0 << 16, z0 |
  // planes << 16), so that the per-plane copy logic does no division: in the full
  // waves, units u = vb + lu G (lu < nfull) of the slice in wave order (tiles
  // fastest, so the grid works on adjacent tiles at one depth); the planes of the
  // units left after the last full wave, taken in wave order, are split evenly
  // over the G blocks, a block's share being pieces of one to three units.
  const int64_t ntiles = (int64_t)m.ntx * m.nty;
  const int nfull = (int)(m.nunits / G);
  const int64_t tail0 = (int64_t)nfull * G;  // first unit of the tail
  auto unit = [&](int64_t u, uint32_t& xy, uint32_t& z0, uint32_t& n) {
    const int64_t ch = u / ntiles, t = u - ch * ntiles, ty = t / m.ntx;
    xy = (uint32_t)((t - ty * m.ntx) * TX) | ((uint32_t)(ty * TY) << 16);
    z0 = (uint32_t)(ch * Lz / m.nch);
    n = (uint32_t)((ch + 1) * Lz / m.nch) - z0;
  };
  uint2* tab = reinterpret_cast<uint2*>(base + L::TAB_OFF);
  for (int i = threadIdx.x; i < nfull; i += blockDim.x) {
    uint32_t xy, z0, n;
    unit(vb + (int64_t)i * G, xy, z0, n);
    tab[i] = make_uint2(xy, z0 | (n << 16));
  }
  __shared__ int s_ntail;
  if (threadIdx.x == 0) {
    // the tail spans few chunks (units are chunk-major) and a chunk's units all
    // have its depth, so the walk goes chunk by chunk
    int nt = 0;
    if (tail0 < m.nunits) {
      const int64_t cha = tail0 / ntiles, chb = (m.nunits - 1) / ntiles;
      int64_t P = 0;  // planes of the tail
      for (int64_t ch = cha; ch <= chb; ++ch) {
        const int64_t ua = tail0 > ch * ntiles ? tail0 : ch * ntiles;
        const int64_t ub = m.nunits < (ch + 1) * ntiles ? m.nunits : (ch + 1) * ntiles;
        P += (ub - ua) * ((ch + 1) * Lz / m.nch - ch * Lz / m.nch);
      }
      const int64_t lo = P * vb / G, hi = P * (vb + 1) / G;  // this block's planes of the tail
      int64_t off = 0;
      for (int64_t ch = cha; ch <= chb && off < hi; ++ch) {
        const int64_t ua = tail0 > ch * ntiles ? tail0 : ch * ntiles;
        const int64_t ub = m.nunits < (ch + 1) * ntiles ? m.nunits : (ch + 1) * ntiles;
        const int64_t z0 = ch * Lz / m.nch, n = (ch + 1) * Lz / m.nch - z0;  // n >= 1
        for (int64_t k = lo > off ? (lo - off) / n : 0; ua + k < ub && off + k * n < hi; ++k) {
          const int64_t uo = off + k * n;
          const int64_t a = lo > uo ? lo : uo, b = hi < uo + n ? hi : uo + n;
          if (a < b) {
            uint32_t xy, zu, nu;
            unit(ua + k, xy, zu, nu);
            tab[nfull + nt++] = make_uint2(xy, (zu + (uint32_t)(a - uo)) | ((uint32_t)(b - a) << 16));
          }
        }
        off += (ub - ua) * n;
      }
    }
    s_ntail = nt;
  }
  __syncthreads();
  const int nlu = nfull + s_ntail;
  auto planes_of = [&](int lu) { return (int)(tab[lu].y >> 16); };
  // The copies of a block, in the order they are consumed: per unit (of n
  // planes z0 .. z0+n-1) the x planes z0-1 .. z0+n (positions j = -1 .. n) and
  // the y_in / potential planes z0 .. z0+n-1 (positions j = 0 .. n-1).  Copy k
  // of a ring goes to slot k mod (ring size); when the last warp releases copy
  // k, that warp issues copy k + ring size into the freed slot.  Positions
  // k steps further along the sequence:
  auto ahead_x = [&](int& lu, int& j, int steps) -> bool {
    j += steps;
    while (lu < nlu) {
      const int n = planes_of(lu);
      if (j <= n) return true;
      j -= n + 2;
      ++lu;
    }
    return false;
  };
  auto ahead_y = [&](int& lu, int& j, int steps) -> bool {
    j += steps;
    while (lu < nlu) {
      const int n = planes_of(lu);
      if (j < n) return true;
      j -= n;
      ++lu;
    }
    return false;
  };
  auto issue_x = [&](int lu, int j, uint32_t k) {
    const uint2 e = tab[lu];
    const int x0 = (int)(e.x & 0xffffu), y0 = (int)(e.x >> 16), z0 = (int)(e.y & 0xffffu);
    const int TXe = min(TX, Lx - x0), TYe = min(TY, Ly - y0);
    // halo coordinates: wrapped on a periodic axis, out of range (zeros) past an open edge
    const int hxm = x0 > 0 ? x0 - 1 : (perX ? Lx - 1 : -1);
    const int hxp = x0 + TXe < Lx ? x0 + TXe : (perX ? 0 : Lx);
    const int hym = y0 > 0 ? y0 - 1 : (perY ? Ly - 1 : -1);
    const int hyp = y0 + TYe < Ly ? y0 + TYe : (perY ? 0 : Ly);
    int zx = z0 + j;
    if (perZ) zx = zx < 0 ? zx + Lz : (zx >= Lz ? zx - Lz : zx);
    const uint32_t slot = k % L::NXS;
    const uint32_t dst = sbase + slot * L::XSTAGE;
    mbar_arrive_expect_tx(&full_x[slot], L::X_BYTES);
    tma_load_5d(dst, &m.xi, c0, 0, x0, y0, zx, &full_x[slot]);
    tma_load_5d(dst + L::OFF_XM, &m.xs, c0, 0, hxm, y0, zx, &full_x[slot]);
    tma_load_5d(dst + L::OFF_XP, &m.xs, c0, 0, hxp, y0, zx, &full_x[slot]);
    tma_load_5d(dst + L::OFF_YM, &m.ys, c0, 0, x0, hym, zx, &full_x[slot]);
    tma_load_5d(dst + L::OFF_YP, &m.ys, c0, 0, x0, hyp, zx, &full_x[slot]);
    atomicMax(&s_issued[0], k + 1);
  };
  const unsigned ybytes = (m.has_yin ? L::INT_B : 0) + (m.v_tma ? VF * L::V_B : 0);
  auto issue_y = [&](int lu, int j, uint32_t k) {
    const uint2 e = tab[lu];
    const int x0 = (int)(e.x & 0xffffu), y0 = (int)(e.x >> 16), z0 = (int)(e.y & 0xffffu);
    const uint32_t slot = k % L::NYS;
    const uint32_t dst = sbase + L::NXS * L::XSTAGE + slot * L::YSTAGE;
    if (ybytes) {
      mbar_arrive_expect_tx(&full_y[slot], ybytes);
      if (m.has_yin) tma_load_5d(dst, &m.yi, c0, 0, x0, y0, z0 + j, &full_y[slot]);
      if (m.v_tma) tma_load_3d(dst + L::INT_B, &m.v, VF * x0, y0, z0 + j, &full_y[slot]);
    } else {
      mbar_arrive(&full_y[slot]);
    }
    atomicMax(&s_issued[1], k + 1);
  };
  // release copy k (unit lu, position j) of a ring by this warp; the last warp refills
  auto release_x = [&](uint32_t k, int lu, int j) {
    __syncwarp();
    if (lane == 0 && release_count(&s_cnt[k % L::NXS]) % NCW == NCW - 1)
      if (ahead_x(lu, j, L::NXS)) issue_x(lu, j, k + L::NXS);
  };
  auto release_y = [&](uint32_t k, int lu, int j) {
    __syncwarp();
    if (lane == 0 && release_count(&s_cnt[L::NXS + k % L::NYS]) % NCW == NCW - 1)
      if (ahead_y(lu, j, L::NYS)) issue_y(lu, j, k + L::NYS);
  };

  // Everything above used kernel parameters only.  Before the first access to
  // global memory, wait for the grid this one depends on (the previous sweep,
  // whose outputs it reads and whose inputs it may overwrite) to complete; a
  // no-op without programmatic dependent launch.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // a block without a plane of work (more blocks than planes) issues no copy:
  // its unit table is empty
  if (threadIdx.x == 0 && nlu > 0) {
    prefetch_map(&m.xi);
    prefetch_map(&m.xs);
    prefetch_map(&m.ys);
    if (m.has_yin) prefetch_map(&m.yi);
    if (m.v_tma) prefetch_map(&m.v);
    // the first copies of both rings
    int lu = 0, j = -1;
    for (uint32_t k = 0; k < (uint32_t)L::NXS; ++k) {
      if (k > 0 && !ahead_x(lu, j, 1)) break;
      issue_x(lu, j, k);
    }
    lu = 0;
    j = 0;
    for (uint32_t k = 0; k < (uint32_t)L::NYS; ++k) {
      if (k > 0 && !ahead_y(lu, j, 1)) break;
      issue_y(lu, j, k);
    }
  }

  const int c = lane % L::CPS;
  const int q = lane / L::CPS;
  const int cg = c + sl * L::CPS;  // the chunk (complex64) or vector (fixed point) in the block
  VecCoef<float, VP> cf;
  if constexpr (!FX) cf = load_coef<float, VP>(p, cg);
  DotAcc<float, VP> dacc;  // compensated fp32 sums; their fp64 part lives in shared memory
  dacc.init();
  // fixed point: exact per-unit dot sums of this thread's vector c, the
  // coefficient limbs and the fp64 value of one dot unit
  FxAcc fxx, fxy;
  fx_acc_zero(fxx);
  fx_acc_zero(fxy);
  const FxLimbs fkt = fx_split(FX ? p.fx_kt : 0);
  const int fdshift = p.fx_dshift ? 1 : 0;  // alpha = 2/a: coefficients doubled
  const double fvs = FX ? p.vscale[cg] : 0.0;
  double* wdots = reinterpret_cast<double*>(base + L::DOT_OFF) + warp * kNumDots * 2 * L::CPS;
  if constexpr (has_dots(FEAT)) {
    if (lane < L::CPS)
      for (int k = 0; k < kNumDots * 2; ++k) wdots[k * L::CPS + lane] = 0.0;
  }
  // flush a unit's compensated fp32 sums into this warp's fp64 partials (fixed order)
  auto flush_dots = [&]() {
    if constexpr (FX) {
      double t0 = fx_acc_value(fxx, fvs), t1 = fx_acc_value(fxy, fvs);
      fx_acc_zero(fxx);
      fx_acc_zero(fxy);
      for (int off = 16; off >= L::CPS; off >>= 1) {
        t0 += __shfl_xor_sync(0xffffffffu, t0, off);
        t1 += __shfl_xor_sync(0xffffffffu, t1, off);
      }
      if (lane < L::CPS) {
        wdots[lane] += t0;
        wdots[L::CPS + lane] += t1;
      }
      return;
    }
#pragma unroll
    for (int d = 0; d < kNumDots; ++d)
#pragma unroll
      for (int v = 0; v < VP; ++v) {
        double t = widen(dacc.s[d][v]) + widen(dacc.c[d][v]);
        dacc.s[d][v] = 0.f;
        dacc.c[d][v] = 0.f;
        for (int off = 16; off >= L::CPS; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane < L::CPS) wdots[(d * 2 + v) * L::CPS + lane] += t;
      }
  };
  using XBlk = typename std::conditional<FX, Blk<long long, 1>, Blk<float, VP>>::type;
  XBlk xmr[IPT];
  uint32_t kx = 0, ky = 0;
  const unsigned char* ybase = base + L::NXS * L::XSTAGE;
  bool alive = true;
  for (int lu = 0; lu < nlu && alive; ++lu) {
    const uint2 e = tab[lu];
    const int x0 = (int)(e.x & 0xffffu), y0 = (int)(e.x >> 16), z0 = (int)(e.y & 0xffffu);
    const int n = (int)(e.y >> 16);
    const int TXe = min(TX, Lx - x0), TYe = min(TY, Ly - y0);
    uint32_t Bc[IPT], Bxm[IPT], Bxp[IPT], Bym[IPT], Byp[IPT], Vo[IPT];
    bool ok[IPT];
    int64_t col[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const int li = (i * NCW + warp) * L::SPW + tma_site_perm<R>(q);
      const int ly = li / TX, lx = li - ly * TX;
      ok[i] = lx < TXe && ly < TYe;
      const uint32_t SB = L::SITE_B;
      Bc[i] = tma_swz<R, SWZ>(li * SB, c);
      Bxm[i] = tma_swz<R, SWZ>(lx > 0 ? (li - 1) * SB : L::OFF_XM + ly * SB, c);
      Bxp[i] = tma_swz<R, SWZ>(lx + 1 < TXe ? (li + 1) * SB : L::OFF_XP + ly * SB, c);
      Bym[i] = tma_swz<R, SWZ>(ly > 0 ? (li - TX) * SB : L::OFF_YM + lx * SB, c);
      Byp[i] = tma_swz<R, SWZ>(ly + 1 < TYe ? (li + TX) * SB : L::OFF_YP + lx * SB, c);
      Vo[i] = L::INT_B + 4 * VF * li;
      col[i] = XM ? (int64_t)LX * ((x0 + lx) + (int64_t)LY * (y0 + ly)) : (int64_t)(x0 + lx) + (int64_t)Lx * (y0 + ly);
    }
    // plane z0 - 1: x(z-1) of every site into registers
    if (!tma_wait(&full_x[kx % L::NXS], (kx / L::NXS) & 1, abort)) {
      alive = false;
      break;
    }
    {
      const unsigned char* s0 = base + (kx % L::NXS) * L::XSTAGE;
#pragma unroll
      for (int i = 0; i < IPT; ++i)
        if (ok[i]) {
          if constexpr (FX)
            tma_lds_blk<R, SWZ>(s0, Bc[i], xmr[i]);
          else
            tma_lds_blk<R>(s0, Bc[i], xmr[i]);
        }
    }
    release_x(kx, lu, -1);
    ++kx;
    if (!tma_wait(&full_x[kx % L::NXS], (kx / L::NXS) & 1, abort)) {
      alive = false;
      break;
    }
    for (int j = 0; j < n; ++j) {
      if (!tma_wait(&full_x[(kx + 1) % L::NXS], ((kx + 1) / L::NXS) & 1, abort) ||
          !tma_wait(&full_y[ky % L::NYS], (ky / L::NYS) & 1, abort)) {
        alive = false;
        break;
      }
      const int z = z0 + j;
      const unsigned char* s0 = base + (kx % L::NXS) * L::XSTAGE;
      const unsigned char* s1 = base + ((kx + 1) % L::NXS) * L::XSTAGE;
      const unsigned char* sy = ybase + (ky % L::NYS) * L::YSTAGE;
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        if (!ok[i]) continue;
        const int64_t s = col[i] + plane * z;
        if constexpr ((FEAT & F_ACC) != 0) {
          // the accumulator (and source) lines of this site two planes ahead into
          // L2, so that the epilogue's fp64 reads do not wait on HBM; one thread
          // per 128-byte line of its chunks
          if (z + 2 < Lz && (cg & 3) == 0) {
            const int64_t s2 = s + 2 * plane;
            const bool rd = !(p.acc_mode & ACC_INIT), rs = (p.acc_mode & ACC_XSRC) != 0;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
              if (rd) prefetch_l2(acc_ptr(p.acc, s2, o, RF, 2 * cg));
              if (rs) prefetch_l2(acc_ptr(const_cast<double2*>(p.src), s2, o, RF, 2 * cg));
            }
          }
        }
        if constexpr (FX) {
          // the fixed-point update of sweep_fx.cu: y = d x + kt T (- y_in), exact
          // with one rounding, then the exact dot sums of the site
          Blk<long long, 1> T, yn;
          {
            Blk<long long, 1> xp;
            tma_lds_blk<R, SWZ>(s1, Bc[i], xp);
            fx_axis_T<0, true>(xmr[i], xp, T);
          }
          {
            Blk<long long, 1> ax, bx;
            tma_lds_blk<R, SWZ>(s0, Bxm[i], ax);
            tma_lds_blk<R, SWZ>(s0, Bxp[i], bx);
            fx_axis_T<1, false>(ax, bx, T);
          }
          {
            Blk<long long, 1> ay, by;
            tma_lds_blk<R, SWZ>(s0, Bym[i], ay);
            tma_lds_blk<R, SWZ>(s0, Byp[i], by);
            fx_axis_T<2, false>(ay, by, T);
          }
          Blk<long long, 1> xc, yi;
          tma_lds_blk<R, SWZ>(s0, Bc[i], xc);
          if (m.has_yin) tma_lds_blk<R, SWZ>(sy, Bc[i], yi);
          const longlong2 dv = *reinterpret_cast<const longlong2*>(sy + Vo[i]);
          const FxLimbs dp = fx_split((long long)((unsigned long long)dv.x << fdshift)),
                        dm = fx_split((long long)((unsigned long long)dv.y << fdshift));
          FxLimbs xs[8], ys[8];
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const FxLimbs d = (o & 1) ? dm : dp;
            xs[2 * o] = fx_split(xc.v[o][0].re);
            xs[2 * o + 1] = fx_split(xc.v[o][0].im);
            long long re = fx_mul2(d, xs[2 * o], fkt, fx_split(T.v[o][0].re));
            long long im = fx_mul2(d, xs[2 * o + 1], fkt, fx_split(T.v[o][0].im));
            if (m.has_yin) {
              re -= yi.v[o][0].re;
              im -= yi.v[o][0].im;
            }
            yn.v[o][0] = {re, im};
            ys[2 * o] = fx_split(re);
            ys[2 * o + 1] = fx_split(im);
          }
          store_blk<long long, 1>(static_cast<long long*>(p.yout), s, RF / 2, cg, yn);
          fx_dot_item(xs, ys, fxx, fxy);
          xmr[i] = xc;
        } else {
          if constexpr (WSM) {
            // the Weyl cell update of the Weyl sweeps, on the cell blocks around the cell
            Blk<float, VP> xp, ax, bx, ay, by, xc, yi, yn;
            tma_lds_blk<R>(s1, Bc[i], xp);
            tma_lds_blk<R>(s0, Bxm[i], ax);
            tma_lds_blk<R>(s0, Bxp[i], bx);
            tma_lds_blk<R>(s0, Bym[i], ay);
            tma_lds_blk<R>(s0, Byp[i], by);
            tma_lds_blk<R>(s0, Bc[i], xc);
            if (m.has_yin) tma_lds_blk<R>(sy, Bc[i], yi);
            const float V0 = m.v_tma ? *reinterpret_cast<const float*>(sy + Vo[i])
                                     : site_potential_t<float>(g, 2 * s);
            const float V1 = m.v_tma ? *reinterpret_cast<const float*>(sy + Vo[i] + 4)
                                     : site_potential_t<float>(g, 2 * s + 1);
            if constexpr (XM)  // lattice z = the Y halos, x cells = the march, y = the X halos
              wsm_cell_update(cf, V0, V1, ay, xc, by, xmr[i], xp, ax, bx, m.has_yin ? &yi : nullptr, yn);
            else
              wsm_cell_update(cf, V0, V1, xmr[i], xc, xp, ax, bx, ay, by, m.has_yin ? &yi : nullptr, yn);
            const int64_t sites[4] = {2 * s, 2 * s, 2 * s + 1, 2 * s + 1};
            epilogue<float, VP, FEAT>(p, s, cg, xc, yn, dacc, sites, yi);
            xmr[i] = xc;
            continue;
          }
          // the axes in ti_axes' order (z pair, x pair, y pair), each pair loaded
          // just before it is folded in, so that few blocks are live at a time
          Blk<float, VP> S, D, yn;
          if constexpr (XM) {  // lattice z = the Y halos, x = the march, y = the X halos
            {
              Blk<float, VP> zm, zp;
              tma_lds_blk<R>(s0, Bym[i], zm);
              tma_lds_blk<R>(s0, Byp[i], zp);
              axis_z_init(zm, zp, S, D);
            }
            {
              Blk<float, VP> xp;
              tma_lds_blk<R>(s1, Bc[i], xp);
              axis_x_add(xmr[i], xp, S, D);
            }
            {
              Blk<float, VP> ay, by;
              tma_lds_blk<R>(s0, Bxm[i], ay);
              tma_lds_blk<R>(s0, Bxp[i], by);
              axis_y_add(ay, by, S, D);
            }
          } else {
            {
              Blk<float, VP> xp;
              tma_lds_blk<R>(s1, Bc[i], xp);
              axis_z_init(xmr[i], xp, S, D);
            }
            {
              Blk<float, VP> ax, bx;
              tma_lds_blk<R>(s0, Bxm[i], ax);
              tma_lds_blk<R>(s0, Bxp[i], bx);
              axis_x_add(ax, bx, S, D);
            }
            {
              Blk<float, VP> ay, by;
              tma_lds_blk<R>(s0, Bym[i], ay);
              tma_lds_blk<R>(s0, Byp[i], by);
              axis_y_add(ay, by, S, D);
            }
          }
          Blk<float, VP> xc, yi;
          tma_lds_blk<R>(s0, Bc[i], xc);
          if (m.has_yin) tma_lds_blk<R>(sy, Bc[i], yi);
          const float Vs = m.v_tma ? *reinterpret_cast<const float*>(sy + Vo[i]) : site_potential_t<float>(g, s);
          ti_combine(cf, Vs, xc, S, D, m.has_yin ? &yi : nullptr, yn, g);
          const int64_t sites[4] = {s, s, s, s};
          epilogue<float, VP, FEAT>(p, s, cg, xc, yn, dacc, sites, yi);
          xmr[i] = xc;
        }
      }
      release_x(kx, lu, j);
      release_y(ky, lu, j);
      ++kx;
      ++ky;
    }
    if (!alive) break;
    // plane z1 (waited on as z + 1 by the last plane) is no longer needed
    release_x(kx, lu, n);
    ++kx;
    if constexpr (has_dots(FEAT)) flush_dots();  // once per unit
  }
  __syncthreads();  // every warp has left the rings: no copy is issued after this
  if (threadIdx.x == 0) {
    // drain: wait (bounded) for the last copy issued into every slot, so that no
    // copy is in flight when the block reuses its shared memory or exits (after
    // an abort some of them were never waited for)
    const uint32_t nx = s_issued[0], ny = s_issued[1];
    for (uint32_t k = nx > (uint32_t)L::NXS ? nx - L::NXS : 0; k < nx; ++k)
      for (unsigned t = 0; t < kTmaWaitLimit && !mbar_try_wait(&full_x[k % L::NXS], (k / L::NXS) & 1); ++t) {
      }
    for (uint32_t k = ny > (uint32_t)L::NYS ? ny - L::NYS : 0; k < ny; ++k)
      for (unsigned t = 0; t < kTmaWaitLimit && !mbar_try_wait(&full_y[k % L::NYS], (k / L::NYS) & 1); ++t) {
      }
  }
  __syncthreads();
  if constexpr (has_dots(FEAT)) {
    // fixed-order reduction: the warps' partials in index order, then the
    // blocks in finish_dots (after an abort the values are garbage, but the
    // arrival counter stays consistent)
    const double* wd = reinterpret_cast<const double*>(base + L::DOT_OFF);
    constexpr int RV = FX ? R / 2 : R;  // vectors of a slice
    constexpr int RVF = RV * SL;        // of the block (zeros outside this block's slice)
    double* row = p.partials + (size_t)blockIdx.x * kNumDots * RVF;
    for (int t = threadIdx.x; t < kNumDots * RVF; t += blockDim.x) {
      const int d = t / RVF, r = t - d * RVF - sl * RV;
      double sum = 0.0;
      if (r >= 0 && r < RV) {
        if constexpr (FX) {
          if (d < 2)
            for (int w = 0; w < NCW; ++w) sum += wd[w * kNumDots * 2 * L::CPS + d * L::CPS + r];
        } else {
          for (int w = 0; w < NCW; ++w) sum += wd[((w * kNumDots + d) * 2 + (r & 1)) * L::CPS + (r >> 1)];
        }
      }
      row[t] = sum;
    }
    finish_dots(p);
  }
}

// ------------------------------------------------------------------ host side
inline PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

template <int R, bool DEEP, int MODEL = PVSC_TI, int SL = 1, bool XM = false>
static int encode_maps(const pvsc_lattice* lat, const Sweep& p, TmaMaps& m) {
  using L = TmaLayout<R, DEEP, 8>;
  auto enc = encode_tiled();
  if (!enc) return set_error(PVSC_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
  const int vpc = lat->g.model == PVSC_WSM ? 2 : 1;  // Weyl cells: two sites each
  // 4-byte words of potential data per tile point: fp32 potentials, or the
  // fixed-point sweep's per-site (d+, d-) pair of 64-bit coefficients
  const int vf = MODEL == kModelTIFx ? 4 : vpc;
  const cuuint64_t Lx = lat->g.L[0] / vpc, Ly = lat->g.L[1], Lz = lat->g.L[2];
  // rows of ROWB bytes (128; a whole 64- or 32-byte site for R = 2, 1); with SL
  // slices a row of the block holds SL slice rows side by side (the innermost
  // coordinate selects one) and a site SL times the slice's bytes
  const cuuint64_t SB = (cuuint64_t)L::SITE_B * SL;
  const cuuint64_t RW = (cuuint64_t)L::ROWB / 4;  // floats of a row
  // the kernel's axes (X, Y, Z): (x, y, z), or (y, z, x) when marching along x
  const cuuint64_t dims[5] = {RW * SL, (cuuint64_t)L::ROWS, XM ? Ly : Lx, XM ? Lz : Ly, XM ? Lx : Lz};
  const cuuint64_t strides[4] = {(cuuint64_t)L::ROWB * SL, XM ? SB * Lx : SB, XM ? SB * Lx * Ly : SB * Lx,
                                 XM ? SB : SB * Lx * Ly};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  // the kernel's addressing: the swizzle spanning a row (128, 64 or 32 bytes);
  // unswizzled tiles for fixed point with R/2 >= 8 vectors
  const CUtensorMapSwizzle swz = (MODEL == kModelTIFx && R >= 16) ? CU_TENSOR_MAP_SWIZZLE_NONE
                                 : L::ROWB == 128                 ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : L::ROWB == 64                  ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                  : CU_TENSOR_MAP_SWIZZLE_32B;
  auto tile5 = [&](CUtensorMap* map, const void* ptr, cuuint32_t bx, cuuint32_t by) -> int {
    const cuuint32_t box[5] = {(cuuint32_t)RW, (cuuint32_t)L::ROWS, bx, by, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(ptr), dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PVSC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PVSC_OK;
  };
  std::memset(&m, 0, sizeof(m));
  if (int rc = tile5(&m.xi, p.x, L::TX, L::TY)) return rc;
  if (int rc = tile5(&m.xs, p.x, 1, L::TY)) return rc;
  if (int rc = tile5(&m.ys, p.x, L::TX, 1)) return rc;
  m.has_yin = p.yin != nullptr;
  if (m.has_yin)
    if (int rc = tile5(&m.yi, p.yin, L::TX, L::TY)) return rc;
  m.v_tma = MODEL == kModelTIFx ? 1 : (!XM && lat->g.v_mode == 1);
  if (m.v_tma) {
    const cuuint64_t vd[3] = {vf * Lx, Ly, Lz};  // per site
    const cuuint64_t vs[2] = {4 * vf * Lx, 4 * vf * Lx * Ly};
    const cuuint32_t vb[3] = {(cuuint32_t)(vf * L::TX), (cuuint32_t)L::TY, 1};
    void* vptr = MODEL == kModelTIFx ? const_cast<void*>(p.fx_d) : static_cast<void*>(const_cast<float*>(lat->g.V32));
    const CUresult r = enc(&m.v, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, vptr, vd, vs, vb,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PVSC_ERR_CUDA, "cuTensorMapEncodeTiled (potential) failed (%d)", (int)r);
  }
  return PVSC_OK;
}

template <int R, bool DEEP, int NW, int MODEL, int SL = 1, bool XM = false>
static void* tma_kernel(int feat) {
  if constexpr (MODEL == kModelTIFx) {  // KPM sweeps only
    return feat == F_DOTS ? reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, F_DOTS, MODEL, SL>) : nullptr;
  } else if constexpr (XM) {  // the KPM, series and plain sweeps
    switch (feat) {
      case 0: return reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, 0, MODEL, SL, true>);
      case F_DOTS: return reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, F_DOTS, MODEL, SL, true>);
      case F_ACC: return reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, F_ACC, MODEL, SL, true>);
      default: return nullptr;
    }
  } else {
    switch (feat) {
      case 0: return reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, 0, MODEL, SL>);
      case F_DOTS: return reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, F_DOTS, MODEL, SL>);
      case F_Z: return reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, F_Z, MODEL, SL>);
      case F_DOTS | F_Z: return reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, F_DOTS | F_Z, MODEL, SL>);
      case F_ACC: return reinterpret_cast<void*>(&ti_sweep_tma<R, DEEP, NW, F_ACC, MODEL, SL>);
      default: return nullptr;
    }
  }
}

// z-chunks per column: the count whose wave quantisation and per-unit halo
// planes (two extra x planes, about a third of a plane's traffic each) cost least.
static int auto_chunks(int64_t ntiles, int64_t Lz, int64_t grid) {
  int best = 1;
  double best_cost = 1e300;
  for (int64_t nch = 1; nch <= Lz; ++nch) {
    // full waves of whole units, then the tail's planes spread evenly over the grid
    const int64_t units = ntiles * nch, full = units / grid, tail = units - full * grid;
    const double depth = (double)((Lz + nch - 1) / nch) + 0.7;
    const double cost = (double)full * depth + (tail ? (double)tail * Lz / nch / grid + 1.4 : 0.0);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = (int)nch;
    }
  }
  return best;
}


// SL > 1: the block of R SL vectors in SL slices of R (one slice per block; the
// grid a multiple of SL, each slice's units spread over grid / SL blocks).
// XM: marching along x (tiles over (y, z)); a feature set it has no kernel for
// returns PVSC_ERR_UNSUPPORTED with nothing launched.
template <int R, bool DEEP, int NW, int MODEL = PVSC_TI, int SL = 1, bool XM = false>
static int launch_tma_r(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st) {
  using L = TmaLayout<R, DEEP, NW, MODEL == kModelTIFx ? 4 : 2>;
  void* fn = tma_kernel<R, DEEP, NW, MODEL, SL, XM>(feat);
  if (!fn) return set_error(PVSC_ERR_UNSUPPORTED, "no TMA-staged sweep for feature set %d", feat);
  if (int rc = allow_max_smem(fn)) return rc;
  int occ = 0;
  PVSC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * NW, L::SMEM));
  if (occ < 1) return set_error(PVSC_ERR_CUDA, "the TMA-staged sweep does not fit an SM");
  p.C = L::CPS;
  p.tile_x = L::TX;
  p.tile_y = L::TY;
  TmaMaps m;
  if (int rc = encode_maps<R, DEEP, MODEL, SL, XM>(lat, p, m)) return rc;
  const int64_t LX = lat->g.L[0] / (MODEL == PVSC_WSM ? 2 : 1), LY = lat->g.L[1], LZ = lat->g.L[2];
  const int64_t Lx = XM ? LY : LX, Ly = XM ? LZ : LY, Lz = XM ? LX : LZ;  // the kernel's axes
  m.ntx = (int)((Lx + L::TX - 1) / L::TX);
  m.nty = (int)((Ly + L::TY - 1) / L::TY);
  const int64_t ntiles = (int64_t)m.ntx * m.nty;
  int64_t grid_max = (int64_t)lat->sm_count * occ / SL;  // blocks per slice
  if (grid_max < 1) grid_max = 1;
  int nch = sh.zslab > 0 ? (int)((Lz + sh.zslab - 1) / sh.zslab) : auto_chunks(ntiles, Lz, grid_max);
  if (nch < 1) nch = 1;
  if (nch > Lz) nch = (int)Lz;
  // unit table: the full waves plus at most two pieces of the tail (a margin of four)
  while (nch > 1 && ntiles * nch / grid_max + 4 > kTmaMaxUnits) --nch;
  if (ntiles * nch / grid_max + 4 > kTmaMaxUnits)
    return set_error(PVSC_ERR_UNSUPPORTED, "the TMA-staged sweep's unit table cannot hold %lld tiles per block",
                     (long long)(ntiles / grid_max));
  m.nch = nch;
  m.nunits = ntiles * nch;  // per slice
  p.zslab = (int)((Lz + nch - 1) / nch);
  // no more blocks than units, unless the shape asks to spread (blocks_per_sm
  // = 1): with fewer units than SMs, splitting the columns' planes over all SMs
  // was measured slower on the Weyl cuboid (77.9 -> 72.2 GLUP/s: pieces at
  // staggered depths lose the halo strips' L2 reuse) and is left to the
  // autotuner; blocks left without a plane issue no copy
  const bool spread = sh.blocks_per_sm == 1;
  const int grid = (int)(SL * (m.nunits < grid_max && !spread ? m.nunits : grid_max));
  void* args[] = {&p, &m};
  // with programmatic dependent launch: all of a sweep's blocks are resident at
  // once (grid <= SMs x occupancy), so the next sweep's blocks, which wait for
  // this grid to complete, only take SMs this one leaves free or has finished with
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32 * NW);
  cfg.dynamicSmemBytes = L::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  PVSC_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, args));
  return PVSC_OK;
}

// The two tiles of kernel 7 per R, as (tile_x, tile_y): {large, deep}.
}  // namespace pvsc
