// Double-float refinement residual r = S - mu_W - L (p0 + q) at the two grid
// points (2m, 2m+1) that form one packed complex input of the x transform,
// with every floating-point step done on both points by one packed 2 x FP32
// instruction (add/mul/fma .f32x2, sm_100 and later).
//
// Same arithmetic as residual_value (residual.cuh), point for point: exact
// neighbour sums and differences by TwoSum (the vertical differences of q
// included), products with the double-float coefficient splits by FMA-based
// TwoProduct, one double-float accumulation;
// the x-, y- and z-parts are the 7-point stencil of the cell-centred operator.
// The source S is split into a float pair by integer operations (truncated high
// part, 23 further bits below it).
#pragma once
#include "kernels.cuh"

namespace pgb {

__device__ __forceinline__ float2 f2bc(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b rounded once: fma(b, -1, a)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// TwoSum / TwoDiff on both lanes: s + e == a + b (a - b) exactly.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2& s, float2& e) {
  s = sub2(a, b);
  const float2 bb = sub2(s, a);   // ~ -b
  e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}

// double -> (h, l): h = x truncated to float, l = the next 23 bits of x below h
// (|x - h - l| < 2^-46 |x|).  |x| < 2^-126 gives h = 0; |x| < 2^-80 gives l = 0.
// Finite x with |x| < 2^128 only.
__device__ __forceinline__ void d2ff_trunc(double x, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  // bits 60..29 of x: low 9 exponent bits and 23 mantissa bits; rebias 1023 -> 127
  const uint32_t hb = __funnelshift_r(lo, hi, 29) - (896u << 23);
  h = __uint_as_float(e > 896 ? (hb | sign) : sign);
  // remaining 29 mantissa bits, top 23 of them as an exact float, times 2^(e - 1075 + 6)
  const float m = __uint_as_float(0x4B000000u | ((lo >> 6) & 0x7FFFFFu)) - 8388608.0f;
  const int se = e - 942;
  const float sc = __uint_as_float((uint32_t)(se > 0 ? se : 0) << 23);
  l = __uint_as_float(__float_as_uint(m * sc) ^ sign);
}

// The double iterate p = p0 + q of two points (exact float sum, then to double).
__device__ __forceinline__ double2 finalize_pair(float2 a, float2 b) {
  float sx, ex, sy, ey;
  two_sum(a.x, b.x, sx, ex);
  two_sum(a.y, b.y, sy, ey);
  return make_double2(ff2d_int(sx, ex), ff2d_int(sy, ey));
}
// The correction q = p - p0 of two points to float accuracy, from the double iterate p ((h, l) = p
// split into floats; h - p0 is exact when h and p0 are within a factor 2, and rounds at 2^-24 |q|
// otherwise).
__device__ __forceinline__ float2 q_rebuild_pair(double2 pv, float2 a) {
  float hx, lx, hy, ly;
  d2ff_trunc(pv.x, hx, lx);
  d2ff_trunc(pv.y, hy, ly);
  return make_float2(__fadd_rn(__fsub_rn(hx, a.x), lx), __fadd_rn(__fsub_rn(hy, a.y), ly));
}

// Coefficients of one level, as lane-broadcast pairs (h = high part, l = low
// part of the double-float split; n* = negated high part).
struct ResCoef {
  float2 cxh, cxl, ncxh, cyh, cyl, ncyh, ah, al, nah, ch, cl, nch, muh, mul;
};
__device__ __forceinline__ ResCoef res_coef(float2 cx, float2 cy, float2 A, float2 Cc, float2 mu) {
  ResCoef k;
  k.cxh = f2bc(cx.x); k.cxl = f2bc(cx.y); k.ncxh = f2bc(-cx.x);
  k.cyh = f2bc(cy.x); k.cyl = f2bc(cy.y); k.ncyh = f2bc(-cy.x);
  k.ah = f2bc(A.x); k.al = f2bc(A.y); k.nah = f2bc(-A.x);
  k.ch = f2bc(Cc.x); k.cl = f2bc(Cc.y); k.nch = f2bc(-Cc.x);
  k.muh = f2bc(mu.x); k.mul = f2bc(mu.y);
  return k;
}

// r at the two points.  pc, pe, pw, pn, ps, pd, pu: p0 at the points and at their
// east, west, north, south, lower and upper neighbours (pd = pc at the bottom,
// pu = 0 above the top level); likewise for q when HAS_Q.  Sh, Sl: the split of S.
// Adds the correction's stencil sum qa + qb (+ qc2 + qd2) - m qc to the double-float pair (s, dl) of
// p0's, error-free up to the pair's own rounding: the neighbour sums by TwoSum, the (small) second
// difference rounded once by FMA, then TwoSum into s.  In plain FP32 the sum of q's neighbours (a few
// 1e-7 of |p|) rounds at 6e-8 of itself; on grids whose solution is dominated by weak horizontal
// modes (|p| ~ 1e5 |S|) that left a fixed 1e-12 relative bias in every sweep.
__device__ __forceinline__ void add_q_sum(float2& s, float2& dl, float2 x, float2 ex, float2 qc, float2 m) {
  const float2 qh = fma2(qc, m, x);        // (neighbour sum) + m qc, rounded once: error eps |second difference|
  float2 t, et;
  two_sum2(s, qh, t, et);
  s = t;
  dl = add2(dl, add2(et, ex));
}

// ISO: dx == dy (cx == cy as double-float pairs).  The x and y second differences are then
// summed first, pe + pw + pn + ps - 4 pc exactly as a double-float pair (four TwoSums; -4 pc is
// exact), and multiplied by 1/dx^2 once: one product chain and one TwoSum fewer than the
// general form, with the same double-float accuracy.
template <bool HAS_Q, bool ISO = false>
__device__ __forceinline__ float2 residual_value2(float2 pc, float2 pe, float2 pw, float2 pn, float2 ps, float2 pd,
                                                  float2 pu, float2 qc, float2 qe, float2 qw, float2 qn, float2 qs,
                                                  float2 qd, float2 qu, float2 Sh, float2 Sl, const ResCoef& k) {
  if constexpr (ISO) {
    float2 s1, e1, s2, e2, s3, e3, s4, e4;
    two_sum2(pe, pw, s1, e1);
    two_sum2(pn, ps, s2, e2);
    two_sum2(s1, s2, s3, e3);
    two_sum2(s3, mul2(pc, make_float2(-4.f, -4.f)), s4, e4);
    float2 dl = add2(add2(e1, e2), add2(e3, e4));
    if (HAS_Q) {
      float2 a1, f1, a2, f2, a3, f3;
      two_sum2(qe, qw, a1, f1);
      two_sum2(qn, qs, a2, f2);
      two_sum2(a1, a2, a3, f3);
      add_q_sum(s4, dl, a3, add2(add2(f1, f2), f3), qc, make_float2(-4.f, -4.f));
    }
    const float2 nthh = mul2(k.ncxh, s4);                      // -(cx s4) rounded
    const float2 thl = fma2(k.cxh, dl, fma2(k.cxl, s4, fma2(k.cxh, s4, nthh)));
    // z: a (pd - pc) + c (pu - pc), differences first, q's exactly as well
    float2 dd, ed, du, eu;
    two_diff2(pd, pc, dd, ed);
    two_diff2(pu, pc, du, eu);
    if (HAS_Q) {
      float2 dq, eq, t, et;
      two_diff2(qd, qc, dq, eq);
      two_sum2(dd, dq, t, et);
      dd = t;
      ed = add2(ed, add2(eq, et));
      two_diff2(qu, qc, dq, eq);
      two_sum2(du, dq, t, et);
      du = t;
      eu = add2(eu, add2(eq, et));
    }
    const float2 np1 = mul2(k.nah, dd);
    const float2 l1 = fma2(k.ah, ed, fma2(k.al, dd, fma2(k.ah, dd, np1)));
    const float2 np2 = mul2(k.nch, du);
    const float2 l2 = fma2(k.ch, eu, fma2(k.cl, du, fma2(k.ch, du, np2)));
    float2 b, eb, c, ec;
    two_sum2(np1, np2, b, eb);
    two_sum2(nthh, b, c, ec);                                  // -Lp high, exact with eb + ec
    const float2 lp_lo = sub2(add2(thl, add2(l1, l2)), add2(eb, ec));   // Lp low
    float2 t, et, r, er;
    two_diff2(Sh, k.muh, t, et);
    two_sum2(t, c, r, er);
    return add2(r, add2(er, sub2(add2(et, sub2(Sl, k.mul)), lp_lo)));
  }
  const float2 m2 = make_float2(-2.f, -2.f);
  const float2 m2pc = mul2(pc, m2);
  float2 s1, e1, s2, e2;
  // x: cx (pe + pw - 2 pc), the neighbour sum exact as s2 + dl
  two_sum2(pe, pw, s1, e1);
  two_sum2(s1, m2pc, s2, e2);
  float2 dl = add2(e1, e2);
  if (HAS_Q) {
    float2 a1, f1;
    two_sum2(qe, qw, a1, f1);
    add_q_sum(s2, dl, a1, f1, qc, m2);
  }
  const float2 ntxh = mul2(k.ncxh, s2);                       // -(cx s2) rounded
  const float2 txl = fma2(k.cxh, dl, fma2(k.cxl, s2, fma2(k.cxh, s2, ntxh)));
  // y: cy (pn + ps - 2 pc)
  two_sum2(pn, ps, s1, e1);
  two_sum2(s1, m2pc, s2, e2);
  dl = add2(e1, e2);
  if (HAS_Q) {
    float2 a1, f1;
    two_sum2(qn, qs, a1, f1);
    add_q_sum(s2, dl, a1, f1, qc, m2);
  }
  const float2 ntyh = mul2(k.ncyh, s2);
  const float2 tyl = fma2(k.cyh, dl, fma2(k.cyl, s2, fma2(k.cyh, s2, ntyh)));
  // z: a (pd - pc) + c (pu - pc), differences first (exact for a constant field)
  // (the q differences exactly as well: a_k (q_d - q_c) is far above the converged residual, so an FP32
  // rounding there would bias every sweep alike and stall the refinement)
  float2 dd, ed, du, eu;
  two_diff2(pd, pc, dd, ed);
  two_diff2(pu, pc, du, eu);
  if (HAS_Q) {
    float2 dq, eq, t, et;
    two_diff2(qd, qc, dq, eq);
    two_sum2(dd, dq, t, et);
    dd = t;
    ed = add2(ed, add2(eq, et));
    two_diff2(qu, qc, dq, eq);
    two_sum2(du, dq, t, et);
    du = t;
    eu = add2(eu, add2(eq, et));
  }
  const float2 np1 = mul2(k.nah, dd);
  const float2 l1 = fma2(k.ah, ed, fma2(k.al, dd, fma2(k.ah, dd, np1)));
  const float2 np2 = mul2(k.nch, du);
  const float2 l2 = fma2(k.ch, eu, fma2(k.cl, du, fma2(k.ch, du, np2)));
  // -Lp high parts: ntxh + ntyh + np1 + np2, low parts: txl + tyl + l1 + l2
  float2 a, ea, b, eb, c, ec;
  two_sum2(ntxh, ntyh, a, ea);
  two_sum2(np1, np2, b, eb);
  two_sum2(a, b, c, ec);                                       // -Lp high, exact with ea + eb + ec
  const float2 lp_lo = sub2(add2(add2(txl, tyl), add2(l1, l2)), add2(add2(ea, eb), ec));   // Lp low
  // S - mu - Lp
  float2 t, et, r, er;
  two_diff2(Sh, k.muh, t, et);
  two_sum2(t, c, r, er);
  return add2(r, add2(er, sub2(add2(et, sub2(Sl, k.mul)), lp_lo)));
}

// r = r0 - L q at the two points, from sweep 1's residual r0 of the iterate p0 (stored in FP32) and the
// correction q: the residual of p0 + q, with q's stencil as in residual_value2 (exact neighbour sums and
// differences, products with the coefficient splits by FMA-based TwoProduct) and one double-float
// accumulation onto r0.  r0's own FP32 rounding (at most 2^-24 |r0| per point) is the one error added
// to the residual_value2 form; the verification's bound accounts for it.
template <bool ISO>
__device__ __forceinline__ float2 residual_from_r0(float2 r0, float2 qc, float2 qe, float2 qw, float2 qn, float2 qs,
                                                   float2 qd, float2 qu, const ResCoef& k) {
  float2 nth, thl;   // -(horizontal part of L q) high, + low
  if constexpr (ISO) {
    float2 a1, f1, a2, f2, a3, f3;
    two_sum2(qe, qw, a1, f1);
    two_sum2(qn, qs, a2, f2);
    two_sum2(a1, a2, a3, f3);
    const float2 h = fma2(qc, make_float2(-4.f, -4.f), a3);   // neighbour sum - 4 qc, rounded once
    const float2 dl = add2(add2(f1, f2), f3);
    nth = mul2(k.ncxh, h);
    thl = fma2(k.cxh, dl, fma2(k.cxl, h, fma2(k.cxh, h, nth)));
  } else {
    const float2 m2 = make_float2(-2.f, -2.f);
    float2 a1, f1, a2, f2;
    two_sum2(qe, qw, a1, f1);
    const float2 hx = fma2(qc, m2, a1);
    const float2 ntx = mul2(k.ncxh, hx);
    const float2 txl = fma2(k.cxh, f1, fma2(k.cxl, hx, fma2(k.cxh, hx, ntx)));
    two_sum2(qn, qs, a2, f2);
    const float2 hy = fma2(qc, m2, a2);
    const float2 nty = mul2(k.ncyh, hy);
    const float2 tyl = fma2(k.cyh, f2, fma2(k.cyl, hy, fma2(k.cyh, hy, nty)));
    float2 ea;
    two_sum2(ntx, nty, nth, ea);
    thl = sub2(add2(txl, tyl), ea);
  }
  // z: a (qd - qc) + c (qu - qc), the differences exact
  float2 dd, ed, du, eu;
  two_diff2(qd, qc, dd, ed);
  two_diff2(qu, qc, du, eu);
  const float2 np1 = mul2(k.nah, dd);
  const float2 l1 = fma2(k.ah, ed, fma2(k.al, dd, fma2(k.ah, dd, np1)));
  const float2 np2 = mul2(k.nch, du);
  const float2 l2 = fma2(k.ch, eu, fma2(k.cl, du, fma2(k.ch, du, np2)));
  float2 b, eb, c, ec;
  two_sum2(np1, np2, b, eb);
  two_sum2(nth, b, c, ec);                                     // -Lq high, exact with eb + ec
  const float2 lq_lo = sub2(add2(thl, add2(l1, l2)), add2(eb, ec));   // Lq low
  float2 r, er;
  two_sum2(r0, c, r, er);
  return add2(r, sub2(er, lq_lo));
}

}  // namespace pgb
