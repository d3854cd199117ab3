// Fused stencil sweeps: one pass of H over a block of R vectors, fused with
// the Chebyshev-recurrence update, the series accumulation, the adjoint
// source/gradient terms and the partial dot products (the loop fusion of
// Listing graphenec, Sec. 3.2).
//
// Layout: element (site, orbital, r) at complex offset ((site*4 + orbital)*R + r)
// (TI) or ((4*cell + nu)*R + r) (graphene).  A thread owns one site (TI) or
// one 4-site cell (graphene) and VPT consecutive vectors of it, so every load
// and store is a 16-byte vector access: complex128 one value, complex64 two
// vectors of one orbital (or, for R = 1, two orbitals).
//
// TI sweeps march along z (2.5D blocking): a thread keeps planes z-1, z, z+1
// of its own column in registers and reads the four in-plane neighbours,
// which its neighbours in the block have just loaded, from L1/L2.  Each
// vector element is then read from HBM once per sweep; the paper's layer
// condition (Sec. 3.1) becomes "one plane of the block in L1/L2".
#pragma once

#include "common.cuh"

namespace pvsc {

// F_DOTS: the dot products selected at run time by Sweep::dot_flags.
enum Feat { F_DOTS = 1, F_Z = 2, F_ACC = 4, F_ADJ = 8 };
__host__ __device__ constexpr bool has_dots(int feat) { return (feat & F_DOTS) != 0; }

// 16-byte vector of two 8-byte elements: complex128 (re, im) or the fixed-point pair
template <typename T> struct Pair16 { using type = double2; };
template <> struct Pair16<long long> { using type = longlong2; };

template <typename T, int VPT>
struct Blk {
  cplx<T> v[4][VPT];
};

template <typename T, int VPT>
__device__ __forceinline__ void zero_blk(Blk<T, VPT>& b) {
#pragma unroll
  for (int o = 0; o < 4; ++o)
#pragma unroll
    for (int v = 0; v < VPT; ++v) b.v[o][v] = {T(0), T(0)};
}

// Load the 4 orbitals (TI site) or 4 sites (graphene cell) `s` of chunk rc.
template <typename T, int VPT, bool RO>
__device__ __forceinline__ void load_blk(const T* __restrict__ base, int64_t s, int R, int rc,
                                         Blk<T, VPT>& b) {
  const T* p = base + 2 * ((s * 4) * (int64_t)R + rc * VPT);
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const double2* q = reinterpret_cast<const double2*>(p + 2 * o * R);
      double2 a = RO ? __ldg(q) : *q;
      b.v[o][0] = {a.x, a.y};
    }
  } else if constexpr (VPT == 1) {
    if (R == 1) {  // complex64, R == 1: 32 contiguous bytes
      const float4* q = reinterpret_cast<const float4*>(p);
      float4 a = RO ? __ldg(q) : q[0];
      float4 c = RO ? __ldg(q + 1) : q[1];
      b.v[0][0] = {a.x, a.y};
      b.v[1][0] = {a.z, a.w};
      b.v[2][0] = {c.x, c.y};
      b.v[3][0] = {c.z, c.w};
    } else {  // complex64, one vector per thread: 8 bytes per orbital, coalesced across r
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const float2* q = reinterpret_cast<const float2*>(p + 2 * o * R);
        float2 a = RO ? __ldg(q) : *q;
        b.v[o][0] = {a.x, a.y};
      }
    }
  } else {  // complex64, two vectors per 16 bytes
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const float4* q = reinterpret_cast<const float4*>(p + 2 * o * R);
      float4 a = RO ? __ldg(q) : *q;
      b.v[o][0] = {a.x, a.y};
      b.v[o][1] = {a.z, a.w};
    }
  }
}

template <typename T, int VPT>
__device__ __forceinline__ void store_blk(T* __restrict__ base, int64_t s, int R, int rc,
                                          const Blk<T, VPT>& b) {
  T* p = base + 2 * ((s * 4) * (int64_t)R + rc * VPT);
  if constexpr (sizeof(T) == 8) {
    using P2 = typename Pair16<T>::type;
#pragma unroll
    for (int o = 0; o < 4; ++o) *reinterpret_cast<P2*>(p + 2 * o * R) = P2{b.v[o][0].re, b.v[o][0].im};
  } else if constexpr (VPT == 1) {
    if (R == 1) {
      float4* q = reinterpret_cast<float4*>(p);
      q[0] = make_float4(b.v[0][0].re, b.v[0][0].im, b.v[1][0].re, b.v[1][0].im);
      q[1] = make_float4(b.v[2][0].re, b.v[2][0].im, b.v[3][0].re, b.v[3][0].im);
    } else {
#pragma unroll
      for (int o = 0; o < 4; ++o)
        *reinterpret_cast<float2*>(p + 2 * o * R) = make_float2(b.v[o][0].re, b.v[o][0].im);
    }
  } else {
#pragma unroll
    for (int o = 0; o < 4; ++o)
      *reinterpret_cast<float4*>(p + 2 * o * R) =
          make_float4(b.v[o][0].re, b.v[o][0].im, b.v[o][1].re, b.v[o][1].im);
  }
}

// As load_blk, from a precomputed pointer to the block's first element
// (p = base + 2 ((s * 4) R + rc VPT)); orbital o sits 2 o R reals further.
template <typename T, int VPT, bool RO>
__device__ __forceinline__ void load_at(const T* __restrict__ p, int R, Blk<T, VPT>& b) {
  if constexpr (sizeof(T) == 8) {
    using P2 = typename Pair16<T>::type;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const P2* q = reinterpret_cast<const P2*>(p + 2 * o * R);
      P2 a = RO ? __ldg(q) : *q;
      b.v[o][0] = {a.x, a.y};
    }
  } else if constexpr (VPT == 1) {
    if (R == 1) {
      const float4* q = reinterpret_cast<const float4*>(p);
      float4 a = RO ? __ldg(q) : q[0];
      float4 c = RO ? __ldg(q + 1) : q[1];
      b.v[0][0] = {a.x, a.y};
      b.v[1][0] = {a.z, a.w};
      b.v[2][0] = {c.x, c.y};
      b.v[3][0] = {c.z, c.w};
    } else {
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const float2* q = reinterpret_cast<const float2*>(p + 2 * o * R);
        float2 a = RO ? __ldg(q) : *q;
        b.v[o][0] = {a.x, a.y};
      }
    }
  } else {
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const float4* q = reinterpret_cast<const float4*>(p + 2 * o * R);
      float4 a = RO ? __ldg(q) : *q;
      b.v[o][0] = {a.x, a.y};
      b.v[o][1] = {a.z, a.w};
    }
  }
}

// One value (all VPT vectors) of orbital/site o of block s.
template <typename T, int VPT>
__device__ __forceinline__ void load_one(const T* __restrict__ base, int64_t s, int o, int R,
                                         int rc, cplx<T> (&out)[VPT]) {
  const T* p = base + 2 * ((s * 4 + o) * (int64_t)R + rc * VPT);
  if constexpr (sizeof(T) == 8) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    out[0] = {a.x, a.y};
  } else if constexpr (VPT == 1) {
    float2 a = __ldg(reinterpret_cast<const float2*>(p));
    out[0] = {a.x, a.y};
  } else {
    float4 a = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = {a.x, a.y};
    out[1] = {a.z, a.w};
  }
}

// complex128 accumulator element of (block s, orbital o, vector r)
__device__ __forceinline__ double2* acc_ptr(double2* base, int64_t s, int o, int R, int r) {
  return base + ((s * 4 + o) * (int64_t)R + r);
}

// ---------------------------------------------------------------- per-thread constants
template <typename T, int VPT>
struct VecCoef {
  T alpha[VPT], ab[VPT], am[VPT], kt[VPT], gamma[VPT], delta[VPT];
};

template <typename T, int VPT>
__device__ __forceinline__ VecCoef<T, VPT> load_coef(const Sweep& p, int rc) {
  VecCoef<T, VPT> c;
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int r = rc * VPT + v;
    const double a = p.coef[0][r], b = p.coef[1][r];
    c.alpha[v] = T(a);
    c.ab[v] = T(a * b);
    c.am[v] = T(a * p.g.m);
    c.kt[v] = T(-0.5 * a * p.g.t);
    c.gamma[v] = T(p.coef[2][r]);
    c.delta[v] = T(p.coef[3][r]);
  }
  return c;
}

// ---------------------------------------------------------------- dot-product accumulators
// Per-thread partial sums of the fused dot products.  fp64 storage adds the
// per-site fp64 products straight into fp64.  complex64 storage forms each
// site's products in fp32 and accumulates them in a compensated fp32 pair
// (Knuth's TwoSum keeps the exact rounding error of every addition), flushed
// into fp64 once per column segment: the fp64 pipe, 1/64 of the fp32 rate on
// GB300, is then not touched per site.
template <typename T, int VPT>
struct DotAcc {
  double d[kNumDots][VPT];
  T s[kNumDots][VPT], c[kNumDots][VPT];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int k = 0; k < kNumDots; ++k)
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        d[k][v] = 0.0;
        s[k][v] = T(0);
        c[k][v] = T(0);
      }
  }
  __device__ __forceinline__ void add(int k, int v, T x) {
    if constexpr (sizeof(T) == 8) {
      d[k][v] += x;
    } else {
      const T t = s[k][v] + x;
      const T bp = t - s[k][v];
      c[k][v] += (s[k][v] - (t - bp)) + (x - bp);
      s[k][v] = t;
    }
  }
  __device__ __forceinline__ void flush() {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int k = 0; k < kNumDots; ++k)
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          d[k][v] += (double)s[k][v] + (double)c[k][v];
          s[k][v] = T(0);
          c[k][v] = T(0);
        }
    }
  }
};

// ---------------------------------------------------------------- fp64 accumulation helpers
// binary32 -> binary64 by rebuilding the IEEE 754 bit fields with integer
// operations (sign kept, exponent rebiased by 1023 - 127 = 896, mantissa
// shifted up by 29 bits).  Exact, like the hardware conversion, which on this
// part issues on the narrow fp64 pipe; zero, subnormal, infinite and NaN
// inputs take the hardware conversion.
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)u, 0);
  return (double)f;
}

// (ar, ai) += (cr + i ci)(xr + i xi); kind (set on the host): 1 ci == 0,
// 2 cr == 0, 3 both zero, 0 general.  The Bessel weights of the propagation
// alternate between real and imaginary, so one half of the products is skipped.
__device__ __forceinline__ void cfma_acc(double cr, double ci, int kind, double xr, double xi,
                                         double& ar, double& ai) {
  if (kind == 1) {
    ar = fma(cr, xr, ar);
    ai = fma(cr, xi, ai);
  } else if (kind == 2) {
    ar = fma(-ci, xi, ar);
    ai = fma(ci, xr, ai);
  } else if (kind == 0) {
    ar = fma(cr, xr, fma(-ci, xi, ar));
    ai = fma(cr, xi, fma(ci, xr, ai));
  }
}

// A compensated fp32 sum of products: the value is S + E, where every product
// a b = p + q exactly (q by FMA) and every addition S + p = s + e exactly
// (Knuth's TwoSum) keep their errors in E; S + E is rounded once at the end.
// The round-off of an uncompensated chain of partial sums is correlated with
// the recurring series weights and the terms they multiply, which biases the
// result; the compensated sum is rounded like the exact one.  The _rn
// intrinsics keep the compiler from contracting these steps into FMAs.
struct CSum {
  float S, E;
};

__device__ __forceinline__ void csum_add(CSum& c, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float q = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(c.S, p);
  const float bb = __fsub_rn(s, c.S);
  const float e = __fadd_rn(__fsub_rn(c.S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  c.S = s;
  c.E = __fadd_rn(c.E, __fadd_rn(q, e));
}

// (sr, si) += w (xr + i xi) with the weight w = (re, im) given as fp32 pairs
// hi + lo (w[part][0] hi, w[part][1] lo), so that the product carries the
// weight to about 2^-48 instead of repeating one fp32 rounding of it on every
// series evaluation: the hi products enter compensated, the lo products
// (about 2^-24 of them) go straight into E.  kind as cfma_acc.
__device__ __forceinline__ void csum_cfma(const float (&w)[2][2], int kind, float xr, float xi, CSum& sr,
                                          CSum& si) {
  if (kind == 1 || kind == 0) {
    csum_add(sr, w[0][0], xr);
    sr.E = __fmaf_rn(w[0][1], xr, sr.E);
    csum_add(si, w[0][0], xi);
    si.E = __fmaf_rn(w[0][1], xi, si.E);
  }
  if (kind == 2 || kind == 0) {
    csum_add(sr, -w[1][0], xi);
    sr.E = __fmaf_rn(-w[1][1], xi, sr.E);
    csum_add(si, w[1][0], xr);
    si.E = __fmaf_rn(w[1][1], xr, si.E);
  }
}

// The same with the weight's kind fixed at compile time (KIND 0, 1 or 2);
// FIRST: the sums start with this term, exactly (S = p, E = q).
template <int KIND, bool FIRST>
__device__ __forceinline__ void csum_term(const float (&w)[2][2], float xr, float xi, CSum& sr, CSum& si) {
  static_assert(KIND >= 0 && KIND <= 2, "a nonzero weight");
  if constexpr (KIND != 2) {
    if constexpr (FIRST) {
      sr.S = __fmul_rn(w[0][0], xr);
      sr.E = __fmaf_rn(w[0][0], xr, -sr.S);
      si.S = __fmul_rn(w[0][0], xi);
      si.E = __fmaf_rn(w[0][0], xi, -si.S);
    } else {
      csum_add(sr, w[0][0], xr);
      csum_add(si, w[0][0], xi);
    }
    sr.E = __fmaf_rn(w[0][1], xr, sr.E);
    si.E = __fmaf_rn(w[0][1], xi, si.E);
  }
  if constexpr (KIND != 1) {
    if constexpr (FIRST && KIND == 2) {
      sr.S = __fmul_rn(-w[1][0], xi);
      sr.E = __fmaf_rn(-w[1][0], xi, -sr.S);
      si.S = __fmul_rn(w[1][0], xr);
      si.E = __fmaf_rn(w[1][0], xr, -si.S);
    } else {
      csum_add(sr, -w[1][0], xi);
      csum_add(si, w[1][0], xr);
    }
    sr.E = __fmaf_rn(-w[1][1], xi, sr.E);
    si.E = __fmaf_rn(w[1][1], xr, si.E);
  }
}

// acc (+)= cz y_in + cx x + cy y_new for the complex64 values of one block:
// the one to three terms of each value as a compensated fp32 sum (weights in
// p.fc: [0] x, [1] y_new, [2] y_in), rounded once and added to the fp64
// accumulator with one fp64 add per part.  KZ, KX, KY: the kinds of the y_in,
// x and y_new weights, or -1 for all three taken at run time from p.acc_kind
// (kind 3: no such term).
template <int KZ, int KX, int KY, int VPT>
__device__ __forceinline__ void acc_c64(const Sweep& p, int64_t s, int rc, const Blk<float, VPT>& yi,
                                        const Blk<float, VPT>& xc, const Blk<float, VPT>& yn) {
  const int R = p.R, mode = p.acc_mode;
  // all of the block's accumulator loads first: the stores below are at offsets
  // scaled by the run-time R, which the compiler cannot tell apart from later
  // loads, so a load after a store would wait for a full round trip each time
  double2 av[4][VPT];
#pragma unroll
  for (int o = 0; o < 4; ++o)
#pragma unroll
    for (int v = 0; v < VPT; ++v)
      av[o][v] = (mode & ACC_INIT) ? make_double2(0.0, 0.0) : *acc_ptr(p.acc, s, o, R, rc * VPT + v);
#pragma unroll
  for (int o = 0; o < 4; ++o)
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int r = rc * VPT + v;
      double ar = av[o][v].x, ai = av[o][v].y;
      CSum cr{0.f, 0.f}, ci{0.f, 0.f};
      if constexpr (KZ < 0) {
        const int kx = p.acc_kind & 3, ky = (p.acc_kind >> 2) & 3, kz = (p.acc_kind >> 4) & 3;
        csum_cfma(p.fc[2], kz, yi.v[o][v].re, yi.v[o][v].im, cr, ci);
        csum_cfma(p.fc[0], kx, xc.v[o][v].re, xc.v[o][v].im, cr, ci);
        csum_cfma(p.fc[1], ky, yn.v[o][v].re, yn.v[o][v].im, cr, ci);
      } else {
        static_assert(KZ != 3 && KX != 3 && KY != 3, "compiled for three terms");
        csum_term<KZ, true>(p.fc[2], yi.v[o][v].re, yi.v[o][v].im, cr, ci);
        csum_term<KX, false>(p.fc[0], xc.v[o][v].re, xc.v[o][v].im, cr, ci);
        csum_term<KY, false>(p.fc[1], yn.v[o][v].re, yn.v[o][v].im, cr, ci);
      }
      const float sr = __fadd_rn(cr.S, cr.E), si = __fadd_rn(ci.S, ci.E);
      if (mode & ACC_INIT) {
        ar = widen(sr);
        ai = widen(si);
      } else {
        ar += widen(sr);
        ai += widen(si);
      }
      if (mode & ACC_FINAL) {
        *acc_ptr(p.acc_out, s, o, R, r) = make_double2(p.ph_re * ar - p.ph_im * ai, p.ph_re * ai + p.ph_im * ar);
      } else {
        *acc_ptr(p.acc, s, o, R, r) = make_double2(ar, ai);
      }
    }
}

constexpr int acc_key(int kx, int ky, int kz) { return kx | (ky << 2) | (kz << 4); }

// ---------------------------------------------------------------- the shared epilogue
// Everything a sweep does after y_new of one block is known.  yi: the block's
// y_in as the sweep read it (read only by an accumulating sweep that takes the
// y_in term, which the driver runs with y_in only).
template <typename T, int VPT, int FEAT>
__device__ __forceinline__ void epilogue(const Sweep& p, int64_t s, int rc, const Blk<T, VPT>& xc,
                                         Blk<T, VPT>& yn, DotAcc<T, VPT>& dacc,
                                         const int64_t* site_of /* 4 sites of the block */,
                                         const Blk<T, VPT>& yi) {
  const int R = p.R;
  if constexpr ((FEAT & F_ADJ) != 0) {
    // y_new += sigma * src (complex128 source)
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const double2 h = *acc_ptr(const_cast<double2*>(p.src), s, o, R, rc * VPT + v);
        yn.v[o][v].re += T(p.sg_re * h.x - p.sg_im * h.y);
        yn.v[o][v].im += T(p.sg_re * h.y + p.sg_im * h.x);
      }
  }
  if (p.yout != nullptr) store_blk<T, VPT>(static_cast<T*>(p.yout), s, R, rc, yn);
  if constexpr ((FEAT & F_Z) != 0) {
    Blk<T, VPT> zb;
    load_blk<T, VPT, false>(static_cast<const T*>(p.z), s, R, rc, zb);
    const VecCoef<T, VPT> c = load_coef<T, VPT>(p, rc);
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        zb.v[o][v].re += c.delta[v] * yn.v[o][v].re;
        zb.v[o][v].im += c.delta[v] * yn.v[o][v].im;
      }
    store_blk<T, VPT>(static_cast<T*>(p.z), s, R, rc, zb);
  }
  if constexpr ((FEAT & F_ACC) != 0) {
    // acc (+)= cz y_in + cx x + cy y_new, where x is this sweep's input (or
    // the complex128 source), y_in the vector y_new replaces and y_new its
    // output: with three terms per sweep the driver touches the accumulator on
    // every third sweep only.
    const int mode = p.acc_mode;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      // complex64 vectors (the complex128 source aside): compensated fp32 sums
      // of the one to three terms (a plain fp32 chain of three terms is biased
      // for the recurring weights of a propagation: the norm of the state
      // drifts by ~1e-8 per time step), compiled for the kinds of the
      // three-term touches of real series (filters) and of propagations
      // (weights alternating between real and imaginary); other touches take
      // the kinds at run time.
      if (!(mode & ACC_XSRC)) {
        switch (p.acc_kind) {
          case acc_key(1, 1, 1): acc_c64<1, 1, 1, VPT>(p, s, rc, yi, xc, yn); break;
          case acc_key(2, 1, 1): acc_c64<1, 2, 1, VPT>(p, s, rc, yi, xc, yn); break;
          case acc_key(1, 2, 2): acc_c64<2, 1, 2, VPT>(p, s, rc, yi, xc, yn); break;
          default: acc_c64<-1, -1, -1, VPT>(p, s, rc, yi, xc, yn);
        }
        done = true;
      }
    }
    if (!done) {
      const int kx = p.acc_kind & 3, ky = (p.acc_kind >> 2) & 3, kz = (p.acc_kind >> 4) & 3;
#pragma unroll
      for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const int r = rc * VPT + v;
          double ar = 0.0, ai = 0.0;
          if (!(mode & ACC_INIT)) {
            const double2 a = *acc_ptr(p.acc, s, o, R, r);
            ar = a.x;
            ai = a.y;
          }
          if constexpr (sizeof(T) == 4) {  // the first touch: x exact from the complex128 source
            const double2 h = *acc_ptr(const_cast<double2*>(p.src), s, o, R, r);
            cfma_acc(p.cx_re, p.cx_im, kx, h.x, h.y, ar, ai);
            cfma_acc(p.cy_re, p.cy_im, ky, widen(yn.v[o][v].re), widen(yn.v[o][v].im), ar, ai);
          } else {
            if (mode & ACC_YIN) cfma_acc(p.cz_re, p.cz_im, kz, yi.v[o][v].re, yi.v[o][v].im, ar, ai);
            if (mode & ACC_X) {
              double xr = xc.v[o][v].re, xi = xc.v[o][v].im;
              if (mode & ACC_XSRC) {
                const double2 h = *acc_ptr(const_cast<double2*>(p.src), s, o, R, r);
                xr = h.x;
                xi = h.y;
              }
              cfma_acc(p.cx_re, p.cx_im, kx, xr, xi, ar, ai);
            }
            cfma_acc(p.cy_re, p.cy_im, ky, yn.v[o][v].re, yn.v[o][v].im, ar, ai);
          }
          if (mode & ACC_FINAL) {
            *acc_ptr(p.acc_out, s, o, R, r) =
                make_double2(p.ph_re * ar - p.ph_im * ai, p.ph_re * ai + p.ph_im * ar);
          } else {
            *acc_ptr(p.acc, s, o, R, r) = make_double2(ar, ai);
          }
        }
    }
  }
  if constexpr ((FEAT & F_ADJ) != 0) {
    if (p.grad != nullptr) {
      // gradient partner w: one value per orbital/site, summed per site over vectors
      Blk<T, VPT> wb;
      load_blk<T, VPT, false>(static_cast<const T*>(p.wg), s, R, rc, wb);
      if (p.g.model == 1) {
        double gsum = 0.0;
#pragma unroll
        for (int o = 0; o < 4; ++o)
#pragma unroll
          for (int v = 0; v < VPT; ++v)
            gsum += (double)yn.v[o][v].re * (double)wb.v[o][v].re +
                    (double)yn.v[o][v].im * (double)wb.v[o][v].im;
        p.grad[site_of[0]] += p.gscale * gsum;
      } else {
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          double gsum = 0.0;
#pragma unroll
          for (int v = 0; v < VPT; ++v)
            gsum += (double)yn.v[o][v].re * (double)wb.v[o][v].re +
                    (double)yn.v[o][v].im * (double)wb.v[o][v].im;
          p.grad[site_of[o]] += p.gscale * gsum;
        }
      }
    }
  }
  if constexpr (has_dots(FEAT)) {
    // per-site products in T, accumulated per thread (compensated for fp32)
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      T xx = 0, xyr = 0, xyi = 0, yy = 0;
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const cplx<T> a = xc.v[o][v], b = yn.v[o][v];
        xx = fma(a.re, a.re, fma(a.im, a.im, xx));
        xyr = fma(b.re, a.re, fma(b.im, a.im, xyr));
        if (p.dot_flags & 2) xyi = fma(b.re, a.im, fma(-b.im, a.re, xyi));
        if (p.dot_flags & 4) yy = fma(b.re, b.re, fma(b.im, b.im, yy));
      }
      dacc.add(0, v, xx);
      dacc.add(1, v, xyr);
      if (p.dot_flags & 2) dacc.add(2, v, xyi);
      if (p.dot_flags & 4) dacc.add(3, v, yy);
    }
  }
}

// The epilogue for a sweep that keeps no y_in block: an accumulating sweep
// that takes the y_in term reads it here, before y_new is stored over it.
template <typename T, int VPT, int FEAT>
__device__ __forceinline__ void epilogue(const Sweep& p, int64_t s, int rc, const Blk<T, VPT>& xc,
                                         Blk<T, VPT>& yn, DotAcc<T, VPT>& dacc, const int64_t* site_of) {
  Blk<T, VPT> yi;
  if constexpr ((FEAT & F_ACC) != 0) {
    if (p.acc_mode & ACC_YIN) load_blk<T, VPT, false>(static_cast<const T*>(p.yin), s, p.R, rc, yi);
  }
  epilogue<T, VPT, FEAT>(p, s, rc, xc, yn, dacc, site_of, yi);
}

// ---------------------------------------------------------------- TI sweep
// y_new = alpha (H - beta) x + gamma y_in with H of Eq. TB_H_topi:
//   (H x)_n = (m Gamma^1 + V_n) x_n + sum_j [A_j x_{n-e_j} + A_j^+ x_{n+e_j}],
//   A_j = -(t/2)(Gamma^1 - i Gamma^{j+1}).
// With s_j = x_{n-e_j} + x_{n+e_j} and d_j = x_{n-e_j} - x_{n+e_j}:
//   sum_j [...] = -(t/2) [Gamma^1 S - i sum_j Gamma^{j+1} d_j],  S = sum_j s_j,
// and -i Gamma^{j+1} d is a signed permutation of d's components:
//   j=x: ( d3,  d2, -d1, -d0)   j=y: -i (d3, d2, d1, d0)   j=z: (d1, -d0, d3, -d2).
// Gamma^1 = diag(1,-1,1,-1) is a sign flip, so no multiply is spent on it.
//
// ti_march runs this along one column (x, y) of the lattice for planes
// z0 <= z < z1 and vector chunk rc, handing every updated site to emit(s, xc,
// yn).  NC selects the read-only (non-coherent) load path for x, valid only
// when x is not written anywhere during the kernel.
//
// With DEPTH > 0 the HBM stream of the column (plane z+1 of x and y_in of
// plane z) is prefetched DEPTH planes ahead with cp.async into a per-thread
// shared-memory ring of DEPTH+1 slots, so every thread keeps DEPTH planes of
// loads in flight without holding them in registers.  Each thread only reads
// the slots it filled itself, so the ring needs no block barrier.  Ring layout:
// 16-byte granule k of slot q, buffer b (0 x, 1 y_in) of thread t at
// ((((q * 2 + b) * 4 + k) * nthr) + t) * 16 bytes (conflict-free).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Ring slots hold NBUF buffers: 2 (x(z+1), y_in(z): the HBM streams) or 6
// (plus the four in-plane neighbours, which otherwise come from L1/L2).

// Issue the 16-byte granules of one block (4 orbitals x VPT vectors) whose
// first element is at p (p as for load_at).
template <typename T, int VPT>
__device__ __forceinline__ void ring_issue(unsigned char* buf, int nthr, const T* p, int R) {
  if constexpr (sizeof(T) == 4 && VPT == 1) {  // complex64, R == 1: 2 granules
    cp_async16(buf, p);
    cp_async16(buf + (size_t)nthr * 16, p + 4);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) cp_async16(buf + (size_t)k * nthr * 16, p + 2 * k * R);
  }
}

template <typename T, int VPT>
__device__ __forceinline__ void ring_read(const unsigned char* buf, int nthr, Blk<T, VPT>& b) {
  if constexpr (sizeof(T) == 8) {
    using P2 = typename Pair16<T>::type;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const P2 a = *reinterpret_cast<const P2*>(buf + (size_t)o * nthr * 16);
      b.v[o][0] = {a.x, a.y};
    }
  } else if constexpr (VPT == 2) {
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const float4 a = *reinterpret_cast<const float4*>(buf + (size_t)o * nthr * 16);
      b.v[o][0] = {a.x, a.y};
      b.v[o][1] = {a.z, a.w};
    }
  } else {
    const float4 a = *reinterpret_cast<const float4*>(buf);
    const float4 c = *reinterpret_cast<const float4*>(buf + (size_t)nthr * 16);
    b.v[0][0] = {a.x, a.y};
    b.v[1][0] = {a.z, a.w};
    b.v[2][0] = {c.x, c.y};
    b.v[3][0] = {c.z, c.w};
  }
}

// ---------------------------------------------------------------- TI stencil arithmetic
// With S = sum over the two neighbours of an axis and d = x(n - e_j) - x(n + e_j),
// the hopping part of Eq. TB_H_topi is -(t/2) (Gamma^1 S_total + sum_j (-i Gamma^{j+1}) d_j);
// the -i Gamma^{j+1} are signed permutations: x axis (d3, d2, -d1, -d0),
// y axis -i (d3, d2, d1, d0), z axis (d1, -d0, d3, -d2).
template <typename T, int VPT>
__device__ __forceinline__ void axis_z_init(const Blk<T, VPT>& a, const Blk<T, VPT>& b, Blk<T, VPT>& S,
                                            Blk<T, VPT>& D) {
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    cplx<T> d[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      S.v[o][v] = cadd(a.v[o][v], b.v[o][v]);
      d[o] = csub(a.v[o][v], b.v[o][v]);
    }
    D.v[0][v] = d[1];
    D.v[1][v] = {-d[0].re, -d[0].im};
    D.v[2][v] = d[3];
    D.v[3][v] = {-d[2].re, -d[2].im};
  }
}

template <typename T, int VPT>
__device__ __forceinline__ void axis_x_add(const Blk<T, VPT>& a, const Blk<T, VPT>& b, Blk<T, VPT>& S,
                                           Blk<T, VPT>& D) {
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    cplx<T> d[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      S.v[o][v] = cadd(S.v[o][v], cadd(a.v[o][v], b.v[o][v]));
      d[o] = csub(a.v[o][v], b.v[o][v]);
    }
    D.v[0][v] = cadd(D.v[0][v], d[3]);
    D.v[1][v] = cadd(D.v[1][v], d[2]);
    D.v[2][v] = csub(D.v[2][v], d[1]);
    D.v[3][v] = csub(D.v[3][v], d[0]);
  }
}

template <typename T, int VPT>
__device__ __forceinline__ void axis_y_add(const Blk<T, VPT>& a, const Blk<T, VPT>& b, Blk<T, VPT>& S,
                                           Blk<T, VPT>& D) {
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    cplx<T> d[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      S.v[o][v] = cadd(S.v[o][v], cadd(a.v[o][v], b.v[o][v]));
      d[o] = csub(a.v[o][v], b.v[o][v]);
    }
    // -i d = (d.im, -d.re)
    D.v[0][v] = cadd(D.v[0][v], cplx<T>{d[3].im, -d[3].re});
    D.v[1][v] = cadd(D.v[1][v], cplx<T>{d[2].im, -d[2].re});
    D.v[2][v] = cadd(D.v[2][v], cplx<T>{d[1].im, -d[1].re});
    D.v[3][v] = cadd(D.v[3][v], cplx<T>{d[0].im, -d[0].re});
  }
}

// S and D of all three axes from the six neighbour blocks (z-, z+, x-, x+, y-, y+).
template <typename T, int VPT>
__device__ __forceinline__ void ti_axes(const Blk<T, VPT>& zm, const Blk<T, VPT>& zp, const Blk<T, VPT>& xm,
                                        const Blk<T, VPT>& xp, const Blk<T, VPT>& ym, const Blk<T, VPT>& yp,
                                        Blk<T, VPT>& S, Blk<T, VPT>& D) {
  axis_z_init(zm, zp, S, D);
  axis_x_add(xm, xp, S, D);
  axis_y_add(ym, yp, S, D);
}

// y += alpha (Delta_1 Gamma^5 + Delta_2 Gamma^15) x, the on-site Delta terms of
// Eq. TB_H_topi.  Gamma^5 = sigma_z (x) s_x and Gamma^15 = [Gamma^1, Gamma^5]/2i =
// sigma_z (x) s_y, so orbital 0 takes (D1 - i D2) x_1, orbital 1 (D1 + i D2) x_0,
// orbital 2 -(D1 - i D2) x_3 and orbital 3 -(D1 + i D2) x_2.
// The Delta values are read from the geometry (kernel parameter space) where
// they are used, so the common Delta = 0 sweep holds no registers for them.
template <typename T, int VPT>
__device__ __forceinline__ void ti_add_delta(const Geometry& g, const VecCoef<T, VPT>& cf,
                                             const Blk<T, VPT>& x, Blk<T, VPT>& y) {
  const T d1 = sizeof(T) == 4 ? T(g.d1f) : T(g.d1), d2 = sizeof(T) == 4 ? T(g.d2f) : T(g.d2);
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const T a1 = cf.alpha[v] * d1, a2 = cf.alpha[v] * d2;
    const cplx<T> x0 = x.v[0][v], x1 = x.v[1][v], x2 = x.v[2][v], x3 = x.v[3][v];
    y.v[0][v].re += fma(a1, x1.re, a2 * x1.im);
    y.v[0][v].im += fma(a1, x1.im, -a2 * x1.re);
    y.v[1][v].re += fma(a1, x0.re, -a2 * x0.im);
    y.v[1][v].im += fma(a1, x0.im, a2 * x0.re);
    y.v[2][v].re -= fma(a1, x3.re, a2 * x3.im);
    y.v[2][v].im -= fma(a1, x3.im, -a2 * x3.re);
    y.v[3][v].re -= fma(a1, x2.re, -a2 * x2.im);
    y.v[3][v].im -= fma(a1, x2.im, a2 * x2.re);
  }
}

// y_new = d_o x_o + kt (Gamma^1 S + D)_o + gamma y_in,  d_o = alpha (V - beta) +- alpha m
// (ti_combine adds the Delta terms when the geometry has them)
template <typename T, int VPT>
__device__ __forceinline__ void ti_combine_core(const VecCoef<T, VPT>& cf, T Vs, const Blk<T, VPT>& xc,
                                                const Blk<T, VPT>& S, const Blk<T, VPT>& D,
                                                const Blk<T, VPT>* yi, Blk<T, VPT>& yn) {
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const T e = fma(cf.alpha[v], Vs, -cf.ab[v]);
    const T dp = e + cf.am[v], dm = e - cf.am[v];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const T dd = (o & 1) ? dm : dp;
      const cplx<T> Tt = (o & 1) ? csub(D.v[o][v], S.v[o][v]) : cadd(D.v[o][v], S.v[o][v]);
      T re = fma(cf.kt[v], Tt.re, dd * xc.v[o][v].re);
      T im = fma(cf.kt[v], Tt.im, dd * xc.v[o][v].im);
      if (yi != nullptr) {
        re = fma(cf.gamma[v], yi->v[o][v].re, re);
        im = fma(cf.gamma[v], yi->v[o][v].im, im);
      }
      yn.v[o][v] = {re, im};
    }
  }
}

template <typename T, int VPT>
__device__ __forceinline__ void ti_combine(const VecCoef<T, VPT>& cf, T Vs, const Blk<T, VPT>& xc,
                                           const Blk<T, VPT>& S, const Blk<T, VPT>& D,
                                           const Blk<T, VPT>* yi, Blk<T, VPT>& yn, const Geometry& g) {
  ti_combine_core(cf, Vs, xc, S, D, yi, yn);
  if (g.has_delta) ti_add_delta(g, cf, xc, yn);
}

template <typename T, int VPT, bool NC, int DEPTH, int NBUF, class Site, class Combine, class Emit>
__device__ __forceinline__ void ti_march(const Geometry& g, const T* __restrict__ X,
                                         const T* __restrict__ Yin, int R, int rc, int64_t col,
                                         int64_t z0, int64_t z1, unsigned char* ring,
                                         Site&& site, Combine&& combine, Emit&& emit) {
  const int64_t Lx = g.L[0], Ly = g.L[1], Lz = g.L[2];
  const int64_t plane = Lx * Ly;
  const int64_t y = udiv64(col, Lx), x = col - y * Lx;
  // in-plane neighbour columns (-1: absent)
  const int64_t cxm = nbr_minus(col, x, Lx, g.per[0], 1);
  const int64_t cxp = nbr_plus(col, x, Lx, g.per[0], 1);
  const int64_t cym = nbr_minus(col, y, Ly, g.per[1], Lx);
  const int64_t cyp = nbr_plus(col, y, Ly, g.per[1], Lx);
  // column base pointers (plane 0) and the plane stride, in reals: the loop
  // then steps pointers instead of recomputing 64-bit element offsets
  const int64_t SS = (int64_t)8 * R;  // reals per site: 4 orbitals x R complex
  const int64_t PS = plane * SS;      // reals per plane
  const int64_t cofs = 2 * rc * VPT;
  const T* Pc = X + col * SS + cofs;
  const T* Pxm = X + (cxm >= 0 ? cxm : 0) * SS + cofs;
  const T* Pxp = X + (cxp >= 0 ? cxp : 0) * SS + cofs;
  const T* Pym = X + (cym >= 0 ? cym : 0) * SS + cofs;
  const T* Pyp = X + (cyp >= 0 ? cyp : 0) * SS + cofs;
  const T* Py = Yin != nullptr ? Yin + col * SS + cofs : nullptr;
  Blk<T, VPT> xm, xc, xp;
  load_at<T, VPT, NC>(Pc + z0 * PS, R, xc);
  {
    const int64_t zm = nbr_minus(z0, z0, Lz, g.per[2], 1);
    if (zm >= 0) load_at<T, VPT, NC>(Pc + zm * PS, R, xm);
    else zero_blk(xm);
  }
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  // prefetch group i (plane z = z0+i) into slot i % (DEPTH+1), buffers:
  // 0 x(z+1) own column, 1 y_in(z), 2..5 the x-/x+/y-/y+ neighbours at plane z
  auto slot_of = [&](int64_t i) {
    return ring + ((size_t)((i % (DEPTH + 1)) * NBUF) * 4 * nthr + tid) * 16;
  };
  auto buf = [&](unsigned char* sl, int b) { return sl + (size_t)b * 4 * nthr * 16; };
  auto ring_group = [&](int64_t i) {
    if constexpr (DEPTH > 0) {
      if (z0 + i < z1) {
        unsigned char* sl = slot_of(i);
        const int64_t zz = z0 + i;
        const int64_t zq = nbr_plus(zz, zz, Lz, g.per[2], 1);
        if (zq >= 0) ring_issue<T, VPT>(buf(sl, 0), nthr, Pc + zq * PS, R);
        if (Yin != nullptr) ring_issue<T, VPT>(buf(sl, 1), nthr, Py + zz * PS, R);
        if constexpr (NBUF == 6) {
          if (cxm >= 0) ring_issue<T, VPT>(buf(sl, 2), nthr, Pxm + zz * PS, R);
          if (cxp >= 0) ring_issue<T, VPT>(buf(sl, 3), nthr, Pxp + zz * PS, R);
          if (cym >= 0) ring_issue<T, VPT>(buf(sl, 4), nthr, Pym + zz * PS, R);
          if (cyp >= 0) ring_issue<T, VPT>(buf(sl, 5), nthr, Pyp + zz * PS, R);
        }
      }
      cp_async_commit();
    }
  };
  if constexpr (DEPTH > 0)
    for (int i = 0; i < DEPTH; ++i) ring_group(i);
  for (int64_t z = z0; z < z1; ++z) {
    const int64_t s = col + plane * z;
    const int64_t zp = nbr_plus(z, z, Lz, g.per[2], 1);
    Blk<T, VPT> yi, ax, bx, ay, by;
    if constexpr (DEPTH > 0) {
      const int64_t i = z - z0;
      ring_group(i + DEPTH);
      cp_async_wait<DEPTH>();  // group i has landed (own slots only: no barrier)
      unsigned char* sl = slot_of(i);
      if (zp >= 0) ring_read<T, VPT>(buf(sl, 0), nthr, xp); else zero_blk(xp);
      if (Yin != nullptr) ring_read<T, VPT>(buf(sl, 1), nthr, yi);
      if constexpr (NBUF == 6) {
        if (cxm >= 0) ring_read<T, VPT>(buf(sl, 2), nthr, ax); else zero_blk(ax);
        if (cxp >= 0) ring_read<T, VPT>(buf(sl, 3), nthr, bx); else zero_blk(bx);
        if (cym >= 0) ring_read<T, VPT>(buf(sl, 4), nthr, ay); else zero_blk(ay);
        if (cyp >= 0) ring_read<T, VPT>(buf(sl, 5), nthr, by); else zero_blk(by);
      } else {  // in-plane neighbours from L1/L2, issued together
        const int64_t zoff = z * PS;
        if (cxm >= 0) load_at<T, VPT, NC>(Pxm + zoff, R, ax); else zero_blk(ax);
        if (cxp >= 0) load_at<T, VPT, NC>(Pxp + zoff, R, bx); else zero_blk(bx);
        if (cym >= 0) load_at<T, VPT, NC>(Pym + zoff, R, ay); else zero_blk(ay);
        if (cyp >= 0) load_at<T, VPT, NC>(Pyp + zoff, R, by); else zero_blk(by);
      }
    } else {
      if (zp >= 0) load_at<T, VPT, NC>(Pc + zp * PS, R, xp);
      else zero_blk(xp);
      if (Yin != nullptr) load_at<T, VPT, false>(Py + z * PS, R, yi);
      // issue the four in-plane neighbour loads together (one L1/L2 round trip)
      const int64_t zoff = z * PS;
      if (cxm >= 0) load_at<T, VPT, NC>(Pxm + zoff, R, ax); else zero_blk(ax);
      if (cxp >= 0) load_at<T, VPT, NC>(Pxp + zoff, R, bx); else zero_blk(bx);
      if (cym >= 0) load_at<T, VPT, NC>(Pym + zoff, R, ay); else zero_blk(ay);
      if (cyp >= 0) load_at<T, VPT, NC>(Pyp + zoff, R, by); else zero_blk(by);
    }
    const auto sv = site(s);  // per-site data (potential), issued with the loads above
    Blk<T, VPT> yn;
    combine(sv, xm, xc, xp, ax, bx, ay, by, Yin != nullptr ? &yi : nullptr, yn);
    emit(s, xc, yn);
    xm = xc;
    xc = xp;
  }
}

// complex64 with one vector per thread holds half the state of two: capped at
// 128 registers, two 256-thread blocks (16 warps) share an SM.
template <typename T, int VPT, int FEAT, int DEPTH = 0, int NBUF = 2>
__global__ void __launch_bounds__(256, (VPT == 1 && sizeof(T) == 4) ? 2 : 1) ti_sweep(const __grid_constant__ Sweep p) {
  extern __shared__ __align__(16) unsigned char ring[];  // DEPTH > 0: cp.async prefetch ring
  const int64_t plane = p.g.L[0] * p.g.L[1], Lz = p.g.L[2];
  const int R = p.R, C = p.C;
  const int rc = threadIdx.x % C;
  const int cshift = __ffs(C) - 1;  // C = R / VPT is a power of two
  const VecCoef<T, VPT> cf = load_coef<T, VPT>(p, rc);
  const T* __restrict__ X = static_cast<const T*>(p.x);
  const T* __restrict__ Yin = static_cast<const T*>(p.yin);
  DotAcc<T, VPT> dacc;
  dacc.init();

  // column groups: runs of blockDim / C consecutive columns, or with
  // p.tile_x > 0 tiles of tile_x x tile_y columns (in-plane y neighbours then
  // mostly inside the block, loaded one plane earlier by their own threads)
  const int64_t ncolthr = plane * C;
  const int TX = p.tile_x, TY = p.tile_y;
  const int64_t ntx = TX > 0 ? (p.g.L[0] + TX - 1) / TX : 0;
  const int64_t nbx = TX > 0 ? ntx * ((p.g.L[1] + TY - 1) / TY) : (ncolthr + blockDim.x - 1) / blockDim.x;
  const int zs = p.zslab;
  // planes updated: all, or on a lattice with halo planes those between them
  // (the halo planes are read as z-neighbours only)
  const int64_t zlo = p.g.zhalo & 1, zn = Lz - (p.g.zhalo & 1) - (p.g.zhalo >> 1);
  const int64_t nzs = (zn + zs - 1) / zs;
  const int64_t nunits = nbx * nzs;
  const int sl = threadIdx.x >> cshift;  // column of this thread within a tile
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t bz = udiv64(u, nbx), bx = u - bz * nbx;
    int64_t col;
    if (TX > 0) {
      if (sl >= TX * TY) continue;
      const int64_t ty = udiv64(bx, ntx), tx = bx - ty * ntx;
      const int64_t x = tx * TX + sl % TX, y = ty * TY + sl / TX;
      if (x >= p.g.L[0] || y >= p.g.L[1]) continue;
      col = x + p.g.L[0] * y;
    } else {
      const int64_t tid = bx * blockDim.x + threadIdx.x;
      if (tid >= ncolthr) continue;
      col = tid >> cshift;
    }
    const int64_t z0 = zlo + bz * zs, z1 = min(z0 + (int64_t)zs, zlo + zn);
    ti_march<T, VPT, true, DEPTH, NBUF>(p.g, X, Yin, R, rc, col, z0, z1, ring,
                           [&](int64_t s) { return site_potential_t<T>(p.g, s); },
                           [&](T Vs, const Blk<T, VPT>& xm, const Blk<T, VPT>& xc,
                               const Blk<T, VPT>& xp, const Blk<T, VPT>& ax, const Blk<T, VPT>& bx,
                               const Blk<T, VPT>& ay, const Blk<T, VPT>& by, const Blk<T, VPT>* yi,
                               Blk<T, VPT>& yn) {
                             Blk<T, VPT> S, D;
                             ti_axes(xm, xp, ax, bx, ay, by, S, D);
                             ti_combine(cf, Vs, xc, S, D, yi, yn, p.g);
                           },
                           [&](int64_t s, const Blk<T, VPT>& xc, Blk<T, VPT>& yn) {
                             const int64_t sites[4] = {s, s, s, s};
                             epilogue<T, VPT, FEAT>(p, s, rc, xc, yn, dacc, sites);
                           });
    if constexpr (has_dots(FEAT)) dacc.flush();  // one fp64 add per column segment
  }
  if constexpr (has_dots(FEAT)) {
    dacc.flush();
    reduce_dots<VPT>(p, dacc.d);
  }
}

// TI sweep marching along x (for lattices whose z extent is short): a thread
// keeps sites x-1, x, x+1 of its line (y, z) in registers and reads the y and
// z neighbours, which the threads of neighbouring lines load, from L1/L2.  The
// neighbours enter ti_axes in the same order as in the z-march (z pair, x
// pair, y pair), so the result equals the z-marching sweep's bit for bit.
// Units: groups of blockDim / C lines (y fastest) times x-segments of p.zslab
// sites (whole lines when p.zslab >= Lx).
template <typename T, int VPT, int FEAT>
__global__ void __launch_bounds__(256) ti_sweep_xmarch(const __grid_constant__ Sweep p) {
  const Geometry& g = p.g;
  const int64_t Lx = g.L[0], Ly = g.L[1], Lz = g.L[2];
  const int R = p.R, C = p.C;
  const int rc = threadIdx.x % C;
  const int cshift = __ffs(C) - 1;
  const VecCoef<T, VPT> cf = load_coef<T, VPT>(p, rc);
  const T* __restrict__ X = static_cast<const T*>(p.x);
  const T* __restrict__ Yin = static_cast<const T*>(p.yin);
  DotAcc<T, VPT> dacc;
  dacc.init();
  const int64_t nlines = Ly * Lz, nthr_lines = nlines * C;
  const int64_t nbx = (nthr_lines + blockDim.x - 1) / blockDim.x;
  const int64_t xs = p.zslab, nxs = (Lx + xs - 1) / xs;
  const int64_t nunits = nbx * nxs;
  const int64_t SS = (int64_t)8 * R, cofs = 2 * rc * VPT;
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t bxs = udiv64(u, nbx), bl = u - bxs * nbx;
    const int64_t tid = bl * blockDim.x + threadIdx.x;
    if (tid >= nthr_lines) continue;
    const int64_t line = tid >> cshift;
    const int64_t z = udiv64(line, Ly), y = line - z * Ly;
    const int64_t x0 = bxs * xs, x1 = min(x0 + xs, Lx);
    const int64_t base = Lx * (y + Ly * z);  // site of x = 0 on this line
    // neighbour lines (site offsets), -1: absent
    const int64_t lym = nbr_minus(base, y, Ly, g.per[1], Lx), lyp = nbr_plus(base, y, Ly, g.per[1], Lx);
    const int64_t lzm = nbr_minus(base, z, Lz, g.per[2], Lx * Ly), lzp = nbr_plus(base, z, Lz, g.per[2], Lx * Ly);
    auto at = [&](int64_t site) { return X + site * SS + cofs; };
    Blk<T, VPT> xm, xc, xp;
    load_at<T, VPT, true>(at(base + x0), R, xc);
    {
      const int64_t q = nbr_minus(x0, x0, Lx, g.per[0], 1);
      if (q >= 0) load_at<T, VPT, true>(at(base + q), R, xm); else zero_blk(xm);
    }
    for (int64_t x = x0; x < x1; ++x) {
      const int64_t s = base + x;
      const int64_t q = nbr_plus(x, x, Lx, g.per[0], 1);
      if (q >= 0) load_at<T, VPT, true>(at(base + q), R, xp); else zero_blk(xp);
      Blk<T, VPT> yi, za, zb, ya, yb, S, D, yn;
      if (Yin != nullptr) load_at<T, VPT, false>(Yin + s * SS + cofs, R, yi);
      if (lzm >= 0) load_at<T, VPT, true>(at(lzm + x), R, za); else zero_blk(za);
      if (lzp >= 0) load_at<T, VPT, true>(at(lzp + x), R, zb); else zero_blk(zb);
      if (lym >= 0) load_at<T, VPT, true>(at(lym + x), R, ya); else zero_blk(ya);
      if (lyp >= 0) load_at<T, VPT, true>(at(lyp + x), R, yb); else zero_blk(yb);
      const T Vs = site_potential_t<T>(g, s);
      ti_axes(za, zb, xm, xp, ya, yb, S, D);
      ti_combine(cf, Vs, xc, S, D, Yin != nullptr ? &yi : nullptr, yn, g);
      const int64_t sites[4] = {s, s, s, s};
      epilogue<T, VPT, FEAT>(p, s, rc, xc, yn, dacc, sites, yi);
      xm = xc;
      xc = xp;
    }
    if constexpr (has_dots(FEAT)) dacc.flush();
  }
  if constexpr (has_dots(FEAT)) {
    dacc.flush();
    reduce_dots<VPT>(p, dacc.d);
  }
}

// Flat TI sweep: one (site, vector chunk) per thread and pass, no state
// carried between planes.  The six neighbours are folded into S and D one at
// a time (each load consumed at once), which keeps the register footprint
// small enough for several blocks per SM; neighbour reuse comes from L1 (x)
// and L2 (y, z).
template <typename T, int VPT, int FEAT>
__global__ void __launch_bounds__(256, 2) ti_sweep_flat(const __grid_constant__ Sweep p) {
  const int64_t Lx = p.g.L[0], Ly = p.g.L[1], Lz = p.g.L[2];
  const int64_t plane = Lx * Ly;
  const int R = p.R, C = p.C;
  const int rc = threadIdx.x % C;
  const VecCoef<T, VPT> cf = load_coef<T, VPT>(p, rc);
  const T* __restrict__ X = static_cast<const T*>(p.x);
  const T* __restrict__ Yin = static_cast<const T*>(p.yin);
  DotAcc<T, VPT> dacc;
  dacc.init();
  const int64_t nthr = p.g.n_sites * C;
  for (int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; tid < nthr;
       tid += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = tid / C;
    const int64_t col = s % plane, z = s / plane, x = col % Lx, y = col / Lx;
    Blk<T, VPT> xc, S, D, a;
    load_blk<T, VPT, true>(X, s, R, rc, xc);
    zero_blk(S);
    zero_blk(D);
    // fold one neighbour: S += a, D += sg * P_axis(a)
    auto fold = [&](int axis, T sg) {
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
#pragma unroll
        for (int o = 0; o < 4; ++o) S.v[o][v] = cadd(S.v[o][v], a.v[o][v]);
        if (axis == 2) {  // z: (d1, -d0, d3, -d2)
          D.v[0][v].re += sg * a.v[1][v].re; D.v[0][v].im += sg * a.v[1][v].im;
          D.v[1][v].re -= sg * a.v[0][v].re; D.v[1][v].im -= sg * a.v[0][v].im;
          D.v[2][v].re += sg * a.v[3][v].re; D.v[2][v].im += sg * a.v[3][v].im;
          D.v[3][v].re -= sg * a.v[2][v].re; D.v[3][v].im -= sg * a.v[2][v].im;
        } else if (axis == 0) {  // x: (d3, d2, -d1, -d0)
          D.v[0][v].re += sg * a.v[3][v].re; D.v[0][v].im += sg * a.v[3][v].im;
          D.v[1][v].re += sg * a.v[2][v].re; D.v[1][v].im += sg * a.v[2][v].im;
          D.v[2][v].re -= sg * a.v[1][v].re; D.v[2][v].im -= sg * a.v[1][v].im;
          D.v[3][v].re -= sg * a.v[0][v].re; D.v[3][v].im -= sg * a.v[0][v].im;
        } else {  // y: -i (d3, d2, d1, d0), -i d = (d.im, -d.re)
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            D.v[o][v].re += sg * a.v[3 - o][v].im;
            D.v[o][v].im -= sg * a.v[3 - o][v].re;
          }
        }
      }
    };
    const int64_t nb[6] = {nbr_minus(s, z, Lz, p.g.per[2], plane), nbr_plus(s, z, Lz, p.g.per[2], plane),
                           nbr_minus(s, x, Lx, p.g.per[0], 1),     nbr_plus(s, x, Lx, p.g.per[0], 1),
                           nbr_minus(s, y, Ly, p.g.per[1], Lx),    nbr_plus(s, y, Ly, p.g.per[1], Lx)};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (nb[k] < 0) continue;
      load_blk<T, VPT, true>(X, nb[k], R, rc, a);
      fold(k < 2 ? 2 : (k < 4 ? 0 : 1), (k & 1) ? T(-1) : T(1));
    }
    Blk<T, VPT> yi;
    if (Yin != nullptr) load_blk<T, VPT, false>(Yin, s, R, rc, yi);
    const T Vs = site_potential_t<T>(p.g, s);
    Blk<T, VPT> yn;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const T e = fma(cf.alpha[v], Vs, -cf.ab[v]);
      const T dp = e + cf.am[v], dm = e - cf.am[v];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const T dd = (o & 1) ? dm : dp;
        const cplx<T> Tt = (o & 1) ? csub(D.v[o][v], S.v[o][v]) : cadd(D.v[o][v], S.v[o][v]);
        T re = fma(cf.kt[v], Tt.re, dd * xc.v[o][v].re);
        T im = fma(cf.kt[v], Tt.im, dd * xc.v[o][v].im);
        if (Yin != nullptr) {
          re = fma(cf.gamma[v], yi.v[o][v].re, re);
          im = fma(cf.gamma[v], yi.v[o][v].im, im);
        }
        yn.v[o][v] = {re, im};
      }
    }
    if (p.g.has_delta) ti_add_delta(p.g, cf, xc, yn);
    const int64_t sites[4] = {s, s, s, s};
    epilogue<T, VPT, FEAT>(p, s, rc, xc, yn, dacc, sites, yi);
  }
  if constexpr (has_dots(FEAT)) {
    dacc.flush();
    reduce_dots<VPT>(p, dacc.d);
  }
}

// ---------------------------------------------------------------- graphene sweep
// H of Eq. graphene_model per 4-site cell c (x + Nx y), hopping -t:
//   (Hx)_{c,0} = v0 x_{c,0} - t (x_{c,1} + x_{c+x,1} + x_{c-y,3})
//   (Hx)_{c,1} = v1 x_{c,1} - t (x_{c,0} + x_{c,2} + x_{c-x,0})
//   (Hx)_{c,2} = v2 x_{c,2} - t (x_{c,1} + x_{c,3} + x_{c-x,3})
//   (Hx)_{c,3} = v3 x_{c,3} - t (x_{c,2} + x_{c+x,2} + x_{c+y,0})
// (T_x couples site 0 to site 1 of cell c + x and site 3 to site 2; T_y site 0
// to site 3 of cell c - y; T_n is the chain 0-1-2-3.)
// QD: the potential is the quantum-dot array of Eq. qdotarray, evaluated per
// site from the carried cell coordinates (v_mode 3).
template <typename T, int VPT, int FEAT, bool QD = false>
__global__ void __launch_bounds__(256) gr_sweep(const __grid_constant__ Sweep p) {
  const int64_t Nx = p.g.L[0], Ny = p.g.L[1];
  const int64_t ncell = Nx * Ny;
  const int R = p.R, C = p.C;
  const int rc = threadIdx.x % C;
  const VecCoef<T, VPT> cf = load_coef<T, VPT>(p, rc);
  const T* __restrict__ X = static_cast<const T*>(p.x);
  const T tt = T(p.g.t);
  DotAcc<T, VPT> dacc;
  dacc.init();
  // Grid-stride loop over cells with (x, y) carried along: C is a power of
  // two and divides blockDim, so a thread keeps its chunk rc and the only
  // 64-bit divisions are the two below, once per thread.
  const int cshift = __ffs(C) - 1;
  const int64_t cstride = ((int64_t)gridDim.x * blockDim.x) >> cshift;
  const int64_t sy = cstride / Nx, sx = cstride - sy * Nx;
  int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> cshift;
  int64_t y = c / Nx, x = c - y * Nx;
  for (; c < ncell; c += cstride, x += sx, y += sy) {
    if (x >= Nx) {
      x -= Nx;
      ++y;
    }
    const int64_t cxm = nbr_minus(c, x, Nx, p.g.per[0], 1);
    const int64_t cxp = nbr_plus(c, x, Nx, p.g.per[0], 1);
    const int64_t cym = nbr_minus(c, y, Ny, p.g.per[1], Nx);
    const int64_t cyp = nbr_plus(c, y, Ny, p.g.per[1], Nx);
    // the potentials first: loads issued early, and a regenerated quantum-dot
    // array evaluated while few registers are live
    T Vs[4];
    if constexpr (QD) {
      qd_cell_potentials<T>(p.qds, x, y, Vs);
    } else {
#pragma unroll
      for (int o = 0; o < 4; ++o) Vs[o] = site_potential_t<T>(p.g, 4 * c + o);
    }
    Blk<T, VPT> xc, yi;
    load_blk<T, VPT, true>(X, c, R, rc, xc);
    if (p.yin != nullptr) load_blk<T, VPT, false>(static_cast<const T*>(p.yin), c, R, rc, yi);
    cplx<T> n0[VPT], n1[VPT], n2[VPT], n3[VPT];  // neighbour sums of sites 0..3
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      n0[v] = xc.v[1][v];
      n1[v] = cadd(xc.v[0][v], xc.v[2][v]);
      n2[v] = cadd(xc.v[1][v], xc.v[3][v]);
      n3[v] = xc.v[2][v];
    }
    cplx<T> a[VPT];
    if (cxp >= 0) {
      load_one<T, VPT>(X, cxp, 1, R, rc, a);
#pragma unroll
      for (int v = 0; v < VPT; ++v) n0[v] = cadd(n0[v], a[v]);
      load_one<T, VPT>(X, cxp, 2, R, rc, a);
#pragma unroll
      for (int v = 0; v < VPT; ++v) n3[v] = cadd(n3[v], a[v]);
    }
    if (cxm >= 0) {
      load_one<T, VPT>(X, cxm, 0, R, rc, a);
#pragma unroll
      for (int v = 0; v < VPT; ++v) n1[v] = cadd(n1[v], a[v]);
      load_one<T, VPT>(X, cxm, 3, R, rc, a);
#pragma unroll
      for (int v = 0; v < VPT; ++v) n2[v] = cadd(n2[v], a[v]);
    }
    if (cym >= 0) {
      load_one<T, VPT>(X, cym, 3, R, rc, a);
#pragma unroll
      for (int v = 0; v < VPT; ++v) n0[v] = cadd(n0[v], a[v]);
    }
    if (cyp >= 0) {
      load_one<T, VPT>(X, cyp, 0, R, rc, a);
#pragma unroll
      for (int v = 0; v < VPT; ++v) n3[v] = cadd(n3[v], a[v]);
    }
    Blk<T, VPT> yn;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const T kt = -cf.alpha[v] * tt;
      const cplx<T>* ns[4] = {&n0[v], &n1[v], &n2[v], &n3[v]};
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const T dd = fma(cf.alpha[v], Vs[o], -cf.ab[v]);
        T re = fma(kt, ns[o]->re, dd * xc.v[o][v].re);
        T im = fma(kt, ns[o]->im, dd * xc.v[o][v].im);
        if (p.yin != nullptr) {
          re = fma(cf.gamma[v], yi.v[o][v].re, re);
          im = fma(cf.gamma[v], yi.v[o][v].im, im);
        }
        yn.v[o][v] = {re, im};
      }
    }
    const int64_t sites[4] = {4 * c, 4 * c + 1, 4 * c + 2, 4 * c + 3};
    epilogue<T, VPT, FEAT>(p, c, rc, xc, yn, dacc, sites);
  }
  if constexpr (has_dots(FEAT)) {
    dacc.flush();
    reduce_dots<VPT>(p, dacc.d);
  }
}

// ---------------------------------------------------------------- Weyl semimetal sweeps
// Eq. TB_H_wsm: two orbitals (a, b) per site, bonds n -> n + e_x with
// sigma_x/2 and n -> n + e_j (j = y, z) with (sigma_x + i sigma_j)/2, each with
// its Hermitian conjugate, on-site V_n - c0 sigma_x, c0 = 2 + cos k0 (kept in
// g.m).  Acting on a site:
//   (H x)_a = V a - c0 b + (b_x- + b_x+)/2 + b_y- + (b_z- + b_z+)/2 + i (a_z- - a_z+)/2
//   (H x)_b = V b - c0 a + (a_x- + a_x+)/2 + a_y+ + (a_z- + a_z+)/2 + i (b_z+ - b_z-)/2
// A thread owns a cell of two x-adjacent sites (2X, 2X+1): its four
// components (site 2X: a, b; site 2X+1: a, b) are the four consecutive block
// components of the layout, so cell c = X + (Lx/2)(y + Ly z) is loaded and
// stored like a 4-orbital block and shares the epilogue of the other sweeps.

// y_new of one cell from the cell blocks around it (absent neighbours zero):
// zm, zp the cells at z -+ 1, xm, xp at X -+ 1, ym, yp at y -+ 1; V0, V1 the
// potentials of the two sites; y_new = alpha (H - beta) x + gamma y_in.
template <typename T, int VPT>
__device__ __forceinline__ void wsm_cell_update(const VecCoef<T, VPT>& cf, T V0, T V1,
                                                const Blk<T, VPT>& zm, const Blk<T, VPT>& xc,
                                                const Blk<T, VPT>& zp, const Blk<T, VPT>& xm,
                                                const Blk<T, VPT>& xp, const Blk<T, VPT>& ym,
                                                const Blk<T, VPT>& yp, const Blk<T, VPT>* yi,
                                                Blk<T, VPT>& yn) {
  const T half = T(0.5);
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const cplx<T> a0 = xc.v[0][v], b0 = xc.v[1][v], a1 = xc.v[2][v], b1 = xc.v[3][v];
    cplx<T> T4[4];  // hopping part of each component, before the alpha scaling
    {  // site 0: x- is site 1 of cell X-1, x+ is site 1 of this cell; y- b, y+ a of site 0
      const cplx<T> Sb = cadd(cadd(xm.v[3][v], b1), cadd(zm.v[1][v], zp.v[1][v]));
      const cplx<T> Da = csub(zm.v[0][v], zp.v[0][v]);  // a_z- - a_z+
      T4[0] = {fma(half, Sb.re, ym.v[1][v].re) - half * Da.im, fma(half, Sb.im, ym.v[1][v].im) + half * Da.re};
      const cplx<T> Sa = cadd(cadd(xm.v[2][v], a1), cadd(zm.v[0][v], zp.v[0][v]));
      const cplx<T> Db = csub(zp.v[1][v], zm.v[1][v]);  // b_z+ - b_z-
      T4[1] = {fma(half, Sa.re, yp.v[0][v].re) - half * Db.im, fma(half, Sa.im, yp.v[0][v].im) + half * Db.re};
    }
    {  // site 1: x- is site 0 of this cell, x+ is site 0 of cell X+1
      const cplx<T> Sb = cadd(cadd(b0, xp.v[1][v]), cadd(zm.v[3][v], zp.v[3][v]));
      const cplx<T> Da = csub(zm.v[2][v], zp.v[2][v]);
      T4[2] = {fma(half, Sb.re, ym.v[3][v].re) - half * Da.im, fma(half, Sb.im, ym.v[3][v].im) + half * Da.re};
      const cplx<T> Sa = cadd(cadd(a0, xp.v[0][v]), cadd(zm.v[2][v], zp.v[2][v]));
      const cplx<T> Db = csub(zp.v[3][v], zm.v[3][v]);
      T4[3] = {fma(half, Sa.re, yp.v[2][v].re) - half * Db.im, fma(half, Sa.im, yp.v[2][v].im) + half * Db.re};
    }
    const T e0 = fma(cf.alpha[v], V0, -cf.ab[v]), e1 = fma(cf.alpha[v], V1, -cf.ab[v]);
    const T ac0 = cf.am[v];  // alpha c0
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const T dd = o < 2 ? e0 : e1;
      const cplx<T> partner = xc.v[o ^ 1][v];  // sigma_x: a <-> b of the same site
      T re = fma(cf.alpha[v], T4[o].re, fma(dd, xc.v[o][v].re, -ac0 * partner.re));
      T im = fma(cf.alpha[v], T4[o].im, fma(dd, xc.v[o][v].im, -ac0 * partner.im));
      if (yi != nullptr) {
        re = fma(cf.gamma[v], yi->v[o][v].re, re);
        im = fma(cf.gamma[v], yi->v[o][v].im, im);
      }
      yn.v[o][v] = {re, im};
    }
  }
}

// Flat cell sweep: one cell per thread and pass; of the in-plane neighbour
// cells only the components the update reads are loaded (x-: site 1, x+: site
// 0, y-: the b components, y+: the a components).
template <typename T, int VPT, int FEAT>
__global__ void __launch_bounds__(256, 2) wsm_sweep(const __grid_constant__ Sweep p) {
  const int64_t NX = p.g.L[0] / 2, Ly = p.g.L[1], Lz = p.g.L[2];
  const int64_t ncell = NX * Ly * Lz;
  const int64_t plane = NX * Ly;  // cells per z plane
  const int R = p.R, C = p.C;
  const int rc = threadIdx.x % C;
  const VecCoef<T, VPT> cf = load_coef<T, VPT>(p, rc);
  const T* __restrict__ X = static_cast<const T*>(p.x);
  DotAcc<T, VPT> dacc;
  dacc.init();
  const int cshift = __ffs(C) - 1;  // C = R / VPT is a power of two
  const int64_t cstride = ((int64_t)gridDim.x * blockDim.x) >> cshift;
  const int64_t szs = cstride / plane, rem = cstride - szs * plane;
  const int64_t sys = rem / NX, sxs = rem - sys * NX;
  int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> cshift;
  int64_t z = c / plane, xy = c - z * plane;
  int64_t y = xy / NX, x = xy - y * NX;
  for (; c < ncell; c += cstride, x += sxs, y += sys, z += szs) {
    if (x >= NX) {
      x -= NX;
      ++y;
    }
    if (y >= Ly) {
      y -= Ly;
      ++z;
    }
    const int64_t nb[6] = {nbr_minus(c, z, Lz, p.g.per[2], plane), nbr_plus(c, z, Lz, p.g.per[2], plane),
                           nbr_minus(c, x, NX, p.g.per[0], 1),     nbr_plus(c, x, NX, p.g.per[0], 1),
                           nbr_minus(c, y, Ly, p.g.per[1], NX),    nbr_plus(c, y, Ly, p.g.per[1], NX)};
    Blk<T, VPT> xc, yi, n[6];
    load_blk<T, VPT, true>(X, c, R, rc, xc);
    if (p.yin != nullptr) load_blk<T, VPT, false>(static_cast<const T*>(p.yin), c, R, rc, yi);
#pragma unroll
    for (int k = 0; k < 6; ++k) zero_blk(n[k]);
    if (nb[0] >= 0) load_blk<T, VPT, true>(X, nb[0], R, rc, n[0]);
    if (nb[1] >= 0) load_blk<T, VPT, true>(X, nb[1], R, rc, n[1]);
    const int want[4][2] = {{2, 3}, {0, 1}, {1, 3}, {0, 2}};  // x-, x+, y-, y+
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (nb[2 + k] >= 0) {
        load_one<T, VPT>(X, nb[2 + k], want[k][0], R, rc, n[2 + k].v[want[k][0]]);
        load_one<T, VPT>(X, nb[2 + k], want[k][1], R, rc, n[2 + k].v[want[k][1]]);
      }
    const T V0 = site_potential_t<T>(p.g, 2 * c), V1 = site_potential_t<T>(p.g, 2 * c + 1);
    Blk<T, VPT> yn;
    wsm_cell_update(cf, V0, V1, n[0], xc, n[1], n[2], n[3], n[4], n[5], p.yin != nullptr ? &yi : nullptr,
                    yn);
    const int64_t sites[4] = {2 * c, 2 * c, 2 * c + 1, 2 * c + 1};
    epilogue<T, VPT, FEAT>(p, c, rc, xc, yn, dacc, sites, yi);
  }
  if constexpr (has_dots(FEAT)) {
    dacc.flush();
    reduce_dots<VPT>(p, dacc.d);
  }
}

// z-marching cell sweep: the cells form columns along z like the TI sites, so
// ti_march runs on the cell geometry (Lx/2 cells along x) with the Weyl update.
template <typename T, int VPT, int FEAT>
__global__ void __launch_bounds__(256) wsm_march_sweep(const __grid_constant__ Sweep p) {
  Geometry gc = p.g;
  gc.L[0] = p.g.L[0] / 2;
  const int64_t plane = gc.L[0] * gc.L[1], Lz = gc.L[2];
  const int R = p.R, C = p.C;
  const int rc = threadIdx.x % C;
  const int cshift = __ffs(C) - 1;
  const VecCoef<T, VPT> cf = load_coef<T, VPT>(p, rc);
  const T* __restrict__ X = static_cast<const T*>(p.x);
  const T* __restrict__ Yin = static_cast<const T*>(p.yin);
  DotAcc<T, VPT> dacc;
  dacc.init();
  const int64_t ncolthr = plane * C;
  const int64_t nbx = (ncolthr + blockDim.x - 1) / blockDim.x;
  const int zs = p.zslab;
  const int64_t nunits = nbx * ((Lz + zs - 1) / zs);
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t bz = udiv64(u, nbx), bx = u - bz * nbx;
    const int64_t tid = bx * blockDim.x + threadIdx.x;
    if (tid >= ncolthr) continue;
    const int64_t z0 = bz * zs, z1 = min(z0 + (int64_t)zs, Lz);
    ti_march<T, VPT, true, 0, 2>(
        gc, X, Yin, R, rc, tid >> cshift, z0, z1, nullptr,
        [&](int64_t c) {
          return cplx<T>{site_potential_t<T>(p.g, 2 * c), site_potential_t<T>(p.g, 2 * c + 1)};
        },
        [&](cplx<T> V, const Blk<T, VPT>& zm, const Blk<T, VPT>& xc, const Blk<T, VPT>& zp,
            const Blk<T, VPT>& xm, const Blk<T, VPT>& xp, const Blk<T, VPT>& ym, const Blk<T, VPT>& yp,
            const Blk<T, VPT>* yi, Blk<T, VPT>& yn) {
          wsm_cell_update(cf, V.re, V.im, zm, xc, zp, xm, xp, ym, yp, yi, yn);
        },
        [&](int64_t c, const Blk<T, VPT>& xc, Blk<T, VPT>& yn) {
          const int64_t sites[4] = {2 * c, 2 * c, 2 * c + 1, 2 * c + 1};
          epilogue<T, VPT, FEAT>(p, c, rc, xc, yn, dacc, sites);
        });
    if constexpr (has_dots(FEAT)) dacc.flush();
  }
  if constexpr (has_dots(FEAT)) {
    dacc.flush();
    reduce_dots<VPT>(p, dacc.d);
  }
}

}  // namespace pvsc
