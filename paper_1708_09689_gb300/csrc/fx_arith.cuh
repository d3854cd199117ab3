// Integer arithmetic of the fixed-point (PVSC_Q64) KPM sweeps on 32-bit limbs.
//
// Values are Q4.59 vector entries and Q3.60 coefficients held in 64-bit
// integers (sweep_fx.cu gives the format).  Every 64 x 64-bit product the
// sweep needs is assembled from 32 x 32 -> 64-bit products (one wide
// multiply-add each) of the limbs v = v_h 2^31 + v_l, v_l in [0, 2^31),
// v_h = v >> 31, with the partial sums kept exact in 64 bits by the bounds
// below; no 128-bit product is ever formed.
//
// Bounds (they follow from the checks the driver makes before a fixed-point
// run: [b - a, b + a] holds the Gershgorin interval, a >= |t| / 2, and the
// start block has 2-norm <= 1 per vector):
//   * a vector entry |x| <= 1 (||w_k|| <= ||w_0|| <= 1 since ||T_k(H~)|| <= 1),
//     so |x_h| <= 2^28;
//   * a neighbour combination T of the stencil (a signed sum of at most twelve
//     entries of one vector, or six copies of one entry on a one-site periodic
//     axis) has |T| <= 6, so |T_h| < 1.5 2^30;
//   * a coefficient (d_+-, possibly doubled for alpha = 2/a, and kt) has
//     |c| <= 2, so |c_h| <= 2^30.
// With these, the partial sums in fx_mul2 and fx_dot_item stay below 2^63 in
// magnitude (worked out at each sum).
#pragma once

#include "sweep.cuh"

namespace pvsc {

using i64 = long long;
using u64 = unsigned long long;

constexpr int kFxVal = 59;   // fraction bits of vector values
constexpr int kFxCoef = 60;  // fraction bits of coefficients

struct FxLimbs {
  int h;  // v >> 31 (arithmetic)
  int l;  // v mod 2^31, in [0, 2^31)
};

__device__ __forceinline__ FxLimbs fx_split(i64 v) {
  return FxLimbs{(int)(v >> 31), (int)(v & 0x7fffffff)};
}

__device__ __forceinline__ i64 wmul32(int a, int b) { return (i64)a * (i64)b; }

// c + a b as one wide multiply-add (32 x 32 -> 64 bits, 64-bit addend)
__device__ __forceinline__ i64 wmad32(int a, int b, i64 c) {
  i64 d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

__device__ __forceinline__ u64 wmad32u(unsigned a, unsigned b, u64 c) {
  u64 d;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// round((c1 x1 + c2 x2) 2^-60), half up: Q3.60 x Q4.59 -> Q4.59.
// With P = c1 x1 + c2 x2 + 2^59 = H 2^62 + M 2^31 + L:
//   H = c1_h x1_h + c2_h x2_h               (|H| < 2^61)
//   M = c1_h x1_l + c1_l x1_h + c2_h x2_l + c2_l x2_h + 2^28
//       (|M| <= 2^61 + 2^59 + 2^61 + 1.5 2^61 + 2^28 < 2^63)
//   L = c1_l x1_l + c2_l x2_l               (0 <= L < 2^63)
// and, with N = M + floor(L / 2^31), floor(P / 2^60) = 4 H + floor(N / 2^29)
// (the remainder L mod 2^31 < 2^31 cannot carry across a multiple of 2^60).
__device__ __forceinline__ i64 fx_mul2(FxLimbs c1, FxLimbs x1, FxLimbs c2, FxLimbs x2) {
  const i64 H = wmad32(c2.h, x2.h, wmul32(c1.h, x1.h));
  const i64 M = wmad32(c2.l, x2.h, wmad32(c2.h, x2.l, wmad32(c1.l, x1.h, wmad32(c1.h, x1.l, (i64)1 << (kFxVal - 31)))));
  const i64 L = wmad32(c2.l, x2.l, wmul32(c1.l, x1.l));
  const i64 N = M + (i64)(unsigned)((u64)L >> 31);  // L >= 0: floor(L / 2^31) < 2^32
  return H * 4 + (N >> 29);
}

// The neighbour combination of the TI stencil (Eq. TB_H_topi) per orbital o:
// with S_o the sum of the six neighbours and D_o the signed, permuted axis
// differences d_j = x(n - e_j) - x(n + e_j) of the -i Gamma^{j+1} terms, the
// hopping part of the update is kt T_o, T_o = D_o + S_o for even o and
// D_o - S_o for odd o (the Gamma^1 sign).  T is accumulated axis by axis from
// the two neighbour blocks a = x(n - e_j), b = x(n + e_j): per value four
// terms, sigma_o (a_o + b_o) + (the axis's permuted difference of orbital
// p(o)), summed as two three-operand additions.  Integer sums are exact, so
// the order is free.  AXIS 0: z (d-permutation (d1, -d0, d3, -d2)), 1: x
// ((d3, d2, -d1, -d0)), 2: y (-i (d3, d2, d1, d0)).
template <int AXIS, bool INIT>
__device__ __forceinline__ void fx_axis_T(const Blk<i64, 1>& a, const Blk<i64, 1>& b, Blk<i64, 1>& T) {
  constexpr int P[3][4] = {{1, 0, 3, 2}, {3, 2, 1, 0}, {3, 2, 1, 0}};
  constexpr int SGN[2][4] = {{1, -1, 1, -1}, {1, 1, -1, -1}};  // z, x: sign of the difference
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const bool even = (o & 1) == 0;
    const int p = P[AXIS][o];
    const cplx<i64> ao = a.v[o][0], bo = b.v[o][0], ap = a.v[p][0], bp = b.v[p][0];
    // the permuted difference (dr, di) as (plus - minus) pairs
    i64 dr_p, dr_m, di_p, di_m;
    if constexpr (AXIS == 2) {  // -i (ap - bp) = (ap.im - bp.im, bp.re - ap.re)
      dr_p = ap.im;
      dr_m = bp.im;
      di_p = bp.re;
      di_m = ap.re;
    } else {
      const bool pos = SGN[AXIS][o] > 0;
      dr_p = pos ? ap.re : bp.re;
      dr_m = pos ? bp.re : ap.re;
      di_p = pos ? ap.im : bp.im;
      di_m = pos ? bp.im : ap.im;
    }
    if constexpr (INIT) {
      const i64 re = even ? (ao.re + bo.re + dr_p) : (dr_p - ao.re - bo.re);
      const i64 im = even ? (ao.im + bo.im + di_p) : (di_p - ao.im - bo.im);
      T.v[o][0] = {re - dr_m, im - di_m};
    } else {
      const i64 re = even ? (T.v[o][0].re + ao.re + bo.re) : (T.v[o][0].re - ao.re - bo.re);
      const i64 im = even ? (T.v[o][0].im + ao.im + bo.im) : (T.v[o][0].im - ao.im - bo.im);
      T.v[o][0] = {re + dr_p - dr_m, im + di_p - di_m};
    }
  }
}

// An exact dot-product sum: V = u 2^62 + (hi 2^64 + lo) (two's complement,
// u and hi signed).  u collects the products of the high limbs, whose sum over
// a vector is bounded by its norm, so it needs no carry handling.
struct FxAcc {
  i64 u;
  u64 lo;
  i64 hi;
};

__device__ __forceinline__ void fx_acc_zero(FxAcc& a) {
  a.u = 0;
  a.lo = 0;
  a.hi = 0;
}

// (hi, lo) += v (unsigned 64-bit)
__device__ __forceinline__ void fx_acc_add(FxAcc& a, u64 v) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.s64 %1, %1, 0;" : "+l"(a.lo), "+l"(a.hi) : "l"(v));
}

// (hi, lo) += v 2^s for a signed v and 0 < s < 64
template <int S>
__device__ __forceinline__ void fx_acc_add_shl(FxAcc& a, i64 v) {
  const u64 l = (u64)v << S;
  const i64 h = v >> (64 - S);
  asm("add.cc.u64 %0, %0, %2;\n\taddc.s64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(l), "l"(h));
}

// The value of an accumulator times `unit` (the fp64 weight of one unit),
// rounded once per term: the high-limb part u 2^62 is folded in exactly first.
__device__ __forceinline__ double fx_acc_value(FxAcc a, double unit) {
  fx_acc_add_shl<62>(a, a.u);
  return fma((double)a.hi, 0x1p64, (double)a.lo) * unit;
}

// The dot products of one site block (four orbitals, real and imaginary
// parts: eight entries) added to the accumulators:
//   xx += sum x^2   = sum x_h^2 2^62 + (sum x_h x_l) 2^32 + sum x_l^2
//   xy += sum y x   = sum y_h x_h 2^62 + (sum y_h x_l + y_l x_h) 2^31 + sum y_l x_l
// Per block: |sum x_h x_l| <= 2^31 sum |x_h| <= 2^31 sqrt(8) 2^28 < 2^62;
// |sum (y_h x_l + y_l x_h)| <= 2^31 (sum |y_h| + sum |x_h|) < 2^63; the low
// products (< 2^62 each) are summed four at a time as unsigned numbers.
__device__ __forceinline__ void fx_dot_item(const FxLimbs (&x)[8], const FxLimbs (&y)[8], FxAcc& xx, FxAcc& xy) {
  i64 ah = 0, am = 0, bh = 0, bm = 0;
  u64 al0 = 0, al1 = 0, bl0 = 0, bl1 = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const unsigned xl = (unsigned)x[k].l, yl = (unsigned)y[k].l;
    ah = wmad32(x[k].h, x[k].h, ah);
    am = wmad32(x[k].h, x[k].l, am);
    bh = wmad32(y[k].h, x[k].h, bh);
    bm = wmad32(y[k].l, x[k].h, wmad32(y[k].h, x[k].l, bm));
    if (k < 4) {
      al0 = wmad32u(xl, xl, al0);
      bl0 = wmad32u(yl, xl, bl0);
    } else {
      al1 = wmad32u(xl, xl, al1);
      bl1 = wmad32u(yl, xl, bl1);
    }
  }
  xx.u += ah;
  fx_acc_add_shl<32>(xx, am);
  fx_acc_add(xx, al0);
  fx_acc_add(xx, al1);
  xy.u += bh;
  fx_acc_add_shl<31>(xy, bm);
  fx_acc_add(xy, bl0);
  fx_acc_add(xy, bl1);
}

}  // namespace pvsc
