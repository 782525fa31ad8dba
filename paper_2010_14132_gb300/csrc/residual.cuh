// Double-float residual of the mixed refinement at one grid point:
//   r = S - mu_W - L (p0 + q).
//
// mu_W (the weighted mean of S, found by the first solve) is removed here: it is
// outside the range of L, and left in r it would dominate r's dynamic range, so
// that the float rounding of r and of its transform would swamp the small
// compatible part (most visibly in the kx = 0 columns, whose y-transform carries
// the constant).  The correction solve removes what little constant remains.
//
// The refinement needs r to about 2^-44 of |L||p| (the 7-point sum cancels by
// orders of magnitude for the smooth, large pressure field), which FP32 alone
// cannot give and FP64 instructions make ALU bound on GB300.  Every product and
// sum of p0 (exact floats) with the double-float coefficients is formed with
// error-free transformations.  The vertical differences of the correction q are
// formed exactly too and folded into those of p0: a_k (q_{k-1} - q_k) is a few
// 1e-5 of |S| while the converged residual is near 1e-12 of it, so an FP32
// rounding there (6e-8 relative) would leave the same bias in every sweep and
// stall the refinement near 1e-12 relative error.  The horizontal q sums are
// formed error-free for the same reason: on grids dominated by weak horizontal
// modes |p| reaches 1e5 |S|, and their FP32 rounding became a 1e-12 bias too.
// S (double) is split into hi + lo floats with integer operations.
#pragma once
#include "kernels.cuh"

namespace pgb {

struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return FF{s, e + a.l + b.l};
}

// Residual at one point from its 7-point stencil values of p0 and q (the q
// values enter in plain FP32), the double source S, the vertical coefficient
// splits A = a_k, Cc = c_k, the horizontal ones cx, cy and mu = mu_W.
// At the bottom level pass pd = pc (a_0 = 0); at the top level pass pu = 0: the
// Dirichlet ghost value, and with zero flux c_{nz-1} = 0 makes the term vanish.
__device__ __forceinline__ float residual_value(float pc, float pe, float pw, float pn, float ps, float pd, float pu,
                                                float qc, float qe, float qw, float qn, float qs, float qd, float qu,
                                                double S, float2 A, float2 Cc, float2 cx, float2 cy, float2 mu) {
  // x: cx (pe + pw - 2 pc)
  float s1, e1, s2, e2;
  two_sum(pe, pw, s1, e1);
  two_sum(s1, -2.f * pc, s2, e2);
  float dl = e1 + e2;
  {   // q's stencil sum error-free, folded into (s2, dl) (see add_q_sum in residual2.cuh)
    float a1, f1, t, et;
    two_sum(qe, qw, a1, f1);
    two_sum(s2, __fmaf_rn(qc, -2.f, a1), t, et);
    s2 = t;
    dl += et + f1;
  }
  FF tx;
  two_prod(cx.x, s2, tx.h, tx.l);
  tx.l = __fmaf_rn(cx.x, dl, __fmaf_rn(cx.y, s2, tx.l));
  // y: cy (pn + ps - 2 pc)
  two_sum(pn, ps, s1, e1);
  two_sum(s1, -2.f * pc, s2, e2);
  dl = e1 + e2;
  {
    float a1, f1, t, et;
    two_sum(qn, qs, a1, f1);
    two_sum(s2, __fmaf_rn(qc, -2.f, a1), t, et);
    s2 = t;
    dl += et + f1;
  }
  FF ty;
  two_prod(cy.x, s2, ty.h, ty.l);
  ty.l = __fmaf_rn(cy.x, dl, __fmaf_rn(cy.y, s2, ty.l));
  // z: a (pd - pc) + c (pu - pc)   (a = 0 at the bottom).
  // Differences first: a constant field maps to exactly zero whatever the
  // rounding of the coefficient splits.  Summing a pd + c pu - (a+c) pc instead
  // leaves a row-sum mismatch of ~2^-48 (a+c) that the near-null vertical mode of
  // the lowest-|k| columns amplifies by their condition number.
  float dd, ed, du, eu, p1, l1, p2, l2;
  two_sum(pd, -pc, dd, ed);
  two_sum(pu, -pc, du, eu);
  {
    // + (q_d - q_c) and (q_u - q_c), exactly: (pd - pc) + (qd - qc) = dd + ed + dq + eq
    float dq, eq, t, et;
    two_sum(qd, -qc, dq, eq);
    two_sum(dd, dq, t, et);
    dd = t;
    ed = ed + (eq + et);
    two_sum(qu, -qc, dq, eq);
    two_sum(du, dq, t, et);
    du = t;
    eu = eu + (eq + et);
  }
  two_prod(A.x, dd, p1, l1);
  two_prod(Cc.x, du, p2, l2);
  l1 = __fmaf_rn(A.x, ed, __fmaf_rn(A.y, dd, l1));
  l2 = __fmaf_rn(Cc.x, eu, __fmaf_rn(Cc.y, du, l2));
  two_sum(p1, p2, s2, e2);
  FF tz{s2, (l1 + l2) + e2};
  FF Lp = ff_add(ff_add(tx, ty), tz);
  float sh, sl, th, tl;
  d2ff_int(S, sh, sl);
  two_sum(sh, -mu.x, th, tl);
  tl += sl - mu.y;
  float rh, rl;
  two_sum(th, -Lp.h, rh, rl);
  return rh + (rl + (tl - Lp.l));
}

template <bool HAS_Q>
__device__ __forceinline__ float residual_point(const ResidualArgs& R, const Geom& g, int i, int j, int k) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long pl = (long long)nx * ny;
  const long long row = ((long long)k * ny + j) * nx;
  const long long idx = row + i;
  const int ie = (i + 1 == nx) ? 0 : i + 1, iw = (i == 0) ? nx - 1 : i - 1;
  const long long rn = ((long long)k * ny + ((j + 1 == ny) ? 0 : j + 1)) * nx;
  const long long rs = ((long long)k * ny + ((j == 0) ? ny - 1 : j - 1)) * nx;
  const float* p0 = R.p0;
  const float pc = p0[idx];
  const float pe = p0[row + ie], pw = p0[row + iw], pn = p0[rn + i], ps = p0[rs + i];
  const bool has_dn = k > 0, has_up = k + 1 < nz;
  const float pd = has_dn ? p0[idx - pl] : pc;
  const float pu = has_up ? p0[idx + pl] : 0.f;
  float qc = 0, qe = 0, qw = 0, qn = 0, qs = 0, qd = 0, qu = 0;
  if (HAS_Q) {
    const float* q = R.q;
    qc = q[idx];
    qe = q[row + ie];
    qw = q[row + iw];
    qn = q[rn + i];
    qs = q[rs + i];
    qd = has_dn ? q[idx - pl] : qc;
    qu = has_up ? q[idx + pl] : 0.f;
  }
  // S is read once per sweep: stream past L2
  return residual_value(pc, pe, pw, pn, ps, pd, pu, qc, qe, qw, qn, qs, qd, qu, __ldcs(&R.S[idx]), R.a_ff[k],
                        R.c_ff[k], R.cx, R.cy, *R.mu_ff);
}

}  // namespace pgb
