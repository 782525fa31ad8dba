// Column solves shared by the column kernels (thomas_kernels.cu) and the fused
// spectral-middle kernel (spectral_fused.cu): after the forward transform each
// (kx, ky) wavenumber gives an independent tridiagonal system along z
// (Section 2.1).  The pivot algebra is stated at the top of thomas_kernels.cu.
#pragma once
#include "kernels.cuh"

namespace pgb {

template <typename T> __device__ __forceinline__ T rcp(T u);
// single MUFU reciprocal (max error ~1 ulp) on the critical path of the float recurrence
template <> __device__ __forceinline__ float rcp<float>(float u) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(u));
  return r;
}
template <> __device__ __forceinline__ double rcp<double>(double u) { return 1.0 / u; }

__device__ __forceinline__ int signed_ky(int ky, int ny) { return ky > ny / 2 ? ky - ny : ky; }

struct LowkArgs {
  const int2* cols;
  int n;
  const double* a_d;
  const double* c_d;
  const double* W_d;
  const double* lamx_d;
  const double* lamy_d;
  const double* target_mean;
  double scale;   // 1/(nx ny) in double for the double-precision columns
  int singular00; // zero flux at the top: the (0,0) column is singular
  const double* inv_tab;   // nullable: [n][nz] pivot reciprocals 1/u_k of the listed columns (double
                           // columns only), from lowk_pivots; the recurrence then reads them
};

// One step of the low-|k| pivot recurrence (rounded step by step, so that the table built ahead by
// k_lowk_pivots and a column solve computing its own pivots agree bit for bit):
// g_k = s + a_k g_{k-1}/u_{k-1} (g_0 = s), u_k = g_k + c_k, returns 1/u_k (0 for the pinned singular top).
template <typename TCm> __device__ __forceinline__ TCm rn_mul(TCm x, TCm y);
template <> __device__ __forceinline__ double rn_mul<double>(double x, double y) { return __dmul_rn(x, y); }
template <> __device__ __forceinline__ float rn_mul<float>(float x, float y) { return __fmul_rn(x, y); }
template <typename TCm> __device__ __forceinline__ TCm rn_add(TCm x, TCm y);
template <> __device__ __forceinline__ double rn_add<double>(double x, double y) { return __dadd_rn(x, y); }
template <> __device__ __forceinline__ float rn_add<float>(float x, float y) { return __fadd_rn(x, y); }
template <typename TCm>
__device__ __forceinline__ TCm lowk_pivot_step(int k, TCm s, TCm ak, TCm ck, TCm& g_prev, TCm inv_prev,
                                               bool last_singular) {
  const TCm gk = (k == 0) ? s : rn_add(s, rn_mul(rn_mul(ak, g_prev), inv_prev));
  const TCm u = rn_add(gk, ck);
  g_prev = gk;
  return last_singular ? (TCm)0 : (TCm)1 / u;   // the singular top pivot is pinned
}

// ---------------------------------------------------------------------------
// Low-|k| and singular columns: one thread per listed column, compute type TCm
// (double in the mixed path), scratch in global memory.  The (0,0) column, when
// zero flux at the top makes it singular:
//   forward: remove the W-weighted mean of the right-hand side (compatibility),
//            pin x_{nz-1} = 0, back-substitute, shift to zero mean;
//   adjoint: remove the plain mean of the right-hand side, pin v_{nz-1} = 0,
//            back-substitute, remove the W direction (x -= W sum(x)/sum(W)).
// ---------------------------------------------------------------------------
// The sequential recurrence of one low-|k| or singular column, run by one thread
// out of shared memory: the right-hand side at zx[k ld], zy[k ld] (real and
// imaginary parts; overwritten by the solution before any mean shift), the
// back-substitution factors in w[k ld], the level tables a, c, W (stride 1).
// red receives (shift_x, shift_y, sum W, sum x, sum y) for the caller's output
// pass; sq_out (nullable, forward only) the sum of |x_k|^2 of the output.
template <typename TCm, bool ADJ>
__device__ __forceinline__ void lowk_recurrence(TCm* zx, TCm* zy, TCm* w, int ld, const TCm* a, const TCm* c,
                                                const TCm* W, int nz, int kx, int ky, bool singular,
                                                const double* __restrict__ lamx, const double* __restrict__ lamy,
                                                double scale, const double* __restrict__ target_mean,
                                                Stats* stats, TCm* red, double* sq_out,
                                                const double* __restrict__ inv_col = nullptr) {
  TCm mean_x = 0, mean_y = 0;
  if (singular) {
    TCm sw = 0;
    for (int k = 0; k < nz; ++k) {
      const TCm wk = ADJ ? (TCm)1 : (TCm)W[k];
      mean_x += wk * zx[k * ld];
      mean_y += wk * zy[k * ld];
      sw += wk;
    }
    mean_x /= sw;
    mean_y /= sw;
    // only the first solve records mu_W (a refinement correction solve has a target mean)
    if (!ADJ && stats && !target_mean) stats->mu_w = (double)mean_x * scale;
  }
  const TCm s = singular ? (TCm)0 : -((TCm)lamx[kx] + (TCm)lamy[ky]);
  const TCm ms = -(TCm)scale;
  TCm g_prev = s, inv_prev = 0, yx = 0, yy = 0;
  for (int k = 0; k < nz; ++k) {
    const TCm bx = ms * (zx[k * ld] - mean_x), by = ms * (zy[k * ld] - mean_y);
    // the pivots depend on the column's wavenumbers and the levels only: read from the plan's table
    // when it has them (no division on the chain), else computed here
    const TCm inv = inv_col ? (TCm)__ldg(inv_col + k)
                            : lowk_pivot_step<TCm>(k, s, (TCm)a[k], (TCm)c[k], g_prev, inv_prev,
                                                   singular && (k == nz - 1));
    if (!ADJ) {
      TCm nx_ = bx, ny_ = by;
      if (k > 0) {
        const TCm f = (TCm)a[k] * inv_prev;
        nx_ += f * yx;
        ny_ += f * yy;
      }
      yx = nx_;
      yy = ny_;
      zx[k * ld] = yx * inv;
      zy[k * ld] = yy * inv;
      w[k * ld] = (TCm)c[k] * inv;
    } else {
      TCm nx_ = bx, ny_ = by;
      if (k > 0) {
        nx_ += (TCm)c[k - 1] * yx;
        ny_ += (TCm)c[k - 1] * yy;
      }
      yx = nx_ * inv;
      yy = ny_ * inv;
      zx[k * ld] = yx;
      zy[k * ld] = yy;
      w[k * ld] = (k + 1 < nz) ? (TCm)a[k + 1] * inv : (TCm)0;
    }
    inv_prev = inv;
  }
  TCm xx = zx[(nz - 1) * ld], xy = zy[(nz - 1) * ld];
  TCm sx = xx, sy = xy;
  for (int k = nz - 2; k >= 0; --k) {
    xx = zx[k * ld] + w[k * ld] * xx;
    xy = zy[k * ld] + w[k * ld] * xy;
    zx[k * ld] = xx;
    zy[k * ld] = xy;
    sx += xx;
    sy += xy;
  }
  TCm shx = 0, shy = 0, swt = 1;
  if (singular) {
    if (!ADJ) {
      shx = sx / (TCm)nz;
      shy = sy / (TCm)nz;
      // refinement sweep: the correction also removes the mean of the current iterate
      if (target_mean) shx += (TCm)__ldcg(target_mean);
    } else {
      swt = 0;
      for (int k = 0; k < nz; ++k) swt += (TCm)W[k];
    }
  }
  red[0] = shx;
  red[1] = shy;
  red[2] = swt;
  red[3] = sx;
  red[4] = sy;
  if (!ADJ && sq_out) {
    TCm sq = 0;
    for (int k = 0; k < nz; ++k) {
      const TCm ox = singular ? zx[k * ld] - shx : zx[k * ld], oy = singular ? zy[k * ld] - shy : zy[k * ld];
      sq += ox * ox + oy * oy;
    }
    *sq_out = (double)sq;
  }
}

// One low-|k| or singular column, solved by the whole block: the strided loads
// and stores of the column and the coefficient tables go through shared memory
// in parallel; thread 0 runs the sequential recurrence out of shared memory.
// sq_out (nullable): thread 0 stores the solution's sum of |x_k|^2 over the levels (forward solve).
template <typename TS, typename TCm, bool ADJ>
__device__ __forceinline__ void lowk_column(unsigned char* smraw, typename CT<TS>::t* __restrict__ spec,
                                            const Geom& g, const double* __restrict__ ag,
                                            const double* __restrict__ cg, const double* __restrict__ Wg,
                                            const double* __restrict__ lamx, const double* __restrict__ lamy,
                                            double scale, int2 colk, Stats* stats,
                                            const double* __restrict__ target_mean, bool singular00,
                                            double* sq_out = nullptr, const double* inv_tab = nullptr,
                                            int col_index = 0) {
  using CS = typename CT<TS>::t;
  const int nz = g.nz;
  TCm* zx = reinterpret_cast<TCm*>(smraw);   // right-hand side, then z, then x (real parts)
  TCm* zy = zx + nz;                          // imaginary parts
  TCm* w = zy + nz;                           // back-substitution factors
  TCm* a = w + nz;                            // coefficient tables
  TCm* c = a + nz;
  TCm* W = c + nz;
  TCm* red = W + nz;                          // shift_x, shift_y, sumw, sum_x, sum_y
  const int kx = colk.x, ky = colk.y;
  const bool singular = singular00 && kx == 0 && ky == 0;   // nonsingular with p = 0 on the top face
  CS* colp = spec + (long long)ky * g.P + kx;
  // the column and the target mean are read at L2 (not through L1), so a persistent kernel that
  // produced them earlier in the same launch on another SM is seen
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    const CS v = __ldcg(&colp[(long long)k * g.plane]);
    zx[k] = (TCm)v.x;
    zy[k] = (TCm)v.y;
    a[k] = (TCm)ag[k];
    c[k] = (TCm)cg[k];
    W[k] = (TCm)Wg[k];
  }
  __syncthreads();
  if (threadIdx.x == 0)
    lowk_recurrence<TCm, ADJ>(zx, zy, w, 1, a, c, W, nz, kx, ky, singular, lamx, lamy, scale, target_mean, stats,
                              red, sq_out,
                              (inv_tab && sizeof(TCm) == 8) ? inv_tab + (size_t)col_index * nz : nullptr);
  __syncthreads();
  const TCm shift_x = red[0], shift_y = red[1], sumw = red[2], sum_x = red[3], sum_y = red[4];
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    TCm ox = zx[k], oy = zy[k];
    if (singular) {
      if (!ADJ) {
        ox -= shift_x;
        oy -= shift_y;
      } else {
        // remove the W direction (the null vector of the transposed column)
        const TCm f = (TCm)W[k] / sumw;
        ox -= f * sum_x;
        oy -= f * sum_y;
      }
    }
    CS o;
    o.x = (TS)ox;
    o.y = (TS)oy;
    colp[(long long)k * g.plane] = o;
  }
}

// ---------------------------------------------------------------------------
// Twisted FP32 solve of the columns of one staged tile [nz][TC] (two threads per
// column): the lower thread eliminates levels 0..m-1 upward with the pivots
// (g_k, u_k = g_k + c_k), the upper one levels nz-1..m+1 downward with the mirror
// recurrence h_{nz-1} = s + c_{nz-1}, h_k = s + c_k h_{k+1}/v_{k+1}, v_k = h_k + a_k;
// they meet at m = nz/2 and substitute back outward (k_thomas_tw states the
// algebra).  Thread t < 2 TC works on column t % TC (upper half when t >= TC);
// every thread of the block calls this (it holds two block barriers); threads
// with part = false only take part in the barriers.  valid: the column is one
// this solve handles; s its row sum -(lambda_x + lambda_y); out: its level-0
// entry in the spectrum (levels plane entries apart).  wp/colp: the column's
// factor and tile slots.  Shared: ac [nz] (a_k, c_k), meet [TC], xm_s [TC].
// Returns the sum of |x_k|^2 over the levels the thread wrote (0 when it wrote none).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tw_solve_tile(float2* colp, float* wp, const float2* __restrict__ ac, float4* meet,
                                               float2* xm_s, int TC, int nz, int col_t, int upper, bool part,
                                               bool valid, float s, float ms, float2* out, long long plane) {
  const int m = nz / 2;
  if (part && upper == 0) {
    // levels 0..m-1, upward elimination
    float g_prev = s, inv_prev = 0.f;
    float2 y = make_float2(0.f, 0.f);
    for (int k = 0; k < m; ++k) {
      const float2 akc = ac[k];
      const float2 d = colp[(size_t)k * TC];
      const float f = (k == 0) ? 0.f : akc.x * inv_prev;
      const float gk = (k == 0) ? s : s + f * g_prev;
      const float inv = rcp(gk + akc.y);
      y = make_float2(fmaf(ms, d.x, f * y.x), fmaf(ms, d.y, f * y.y));
      colp[(size_t)k * TC] = make_float2(y.x * inv, y.y * inv);
      wp[(size_t)k * TC] = akc.y * inv;
      g_prev = gk;
      inv_prev = inv;
    }
    // the level-m terms of the lower part: a_m g_{m-1}/u_{m-1} and a_m z_{m-1}
    const float am = ac[m].x;
    const float2 z = (m > 0) ? colp[(size_t)(m - 1) * TC] : make_float2(0.f, 0.f);
    meet[col_t] = (m > 0) ? make_float4(am * g_prev * inv_prev, am * z.x, am * z.y, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
  } else if (part) {
    // levels nz-1..m+1, downward elimination with the mirror recurrence
    float h_prev = s, inv_prev = 0.f;
    float2 y = make_float2(0.f, 0.f);
    for (int k = nz - 1; k > m; --k) {
      const float2 akc = ac[k];
      const float2 d = colp[(size_t)k * TC];
      const float f = (k == nz - 1) ? 0.f : akc.y * inv_prev;   // c_k / v_{k+1}
      const float hk = (k == nz - 1) ? s + akc.y : s + f * h_prev;
      const float inv = rcp(hk + akc.x);
      y = make_float2(fmaf(ms, d.x, f * y.x), fmaf(ms, d.y, f * y.y));
      colp[(size_t)k * TC] = make_float2(y.x * inv, y.y * inv);
      wp[(size_t)k * TC] = akc.x * inv;
      h_prev = hk;
      inv_prev = inv;
    }
    xm_s[col_t] = make_float2((m + 1 < nz) ? h_prev * inv_prev : 1.f, 0.f);   // h_{m+1}/v_{m+1}
  }
  __syncthreads();
  if (part && upper == 0) {
    const float2 akc = ac[m];
    const float cm = akc.y;
    const float hterm = cm * xm_s[col_t].x;
    const float2 zt = (m + 1 < nz) ? colp[(size_t)(m + 1) * TC] : make_float2(0.f, 0.f);
    const float4 lo = meet[col_t];
    const float2 dm = colp[(size_t)m * TC];
    const float den = s + lo.x + hterm;
    const float2 num = make_float2(fmaf(ms, dm.x, lo.y + cm * zt.x), fmaf(ms, dm.y, lo.z + cm * zt.y));
    const float2 xm = make_float2(__fdiv_rn(num.x, den), __fdiv_rn(num.y, den));
    xm_s[col_t] = xm;   // this thread has read the h-term; no other thread touches the slot before the barrier
  }
  __syncthreads();
  float sq = 0.f;   // sum of |x_k|^2 over the levels this thread writes (x_m by the lower thread)
  if (!part || !valid) return sq;
  const float2 xm = xm_s[col_t];
  if (upper == 0) {
    out[(long long)m * plane] = xm;
    sq = xm.x * xm.x + xm.y * xm.y;
    float2 x = xm;
    for (int k = m - 1; k >= 0; --k) {
      const float2 z = colp[(size_t)k * TC];
      const float w = wp[(size_t)k * TC];
      x = make_float2(z.x + w * x.x, z.y + w * x.y);
      out[(long long)k * plane] = x;
      sq = fmaf(x.x, x.x, fmaf(x.y, x.y, sq));
    }
  } else {
    float2 x = xm;
    for (int k = m + 1; k < nz; ++k) {
      const float2 z = colp[(size_t)k * TC];
      const float w = wp[(size_t)k * TC];
      x = make_float2(z.x + w * x.x, z.y + w * x.y);
      out[(long long)k * plane] = x;
      sq = fmaf(x.x, x.x, fmaf(x.y, x.y, sq));
    }
  }
  return sq;
}

}  // namespace pgb
