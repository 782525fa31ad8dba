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
// tab: w[k ld] holds the column's pivot reciprocals 1/u_k on entry (staged by the caller from the
// plan's table, in parallel): the chain then loads them from shared memory instead of forming
// pivots, and the back substitution forms its factors from them (the same products as when they are
// stored by the forward sweep, so both ways give the same bits).
template <typename TCm, bool ADJ>
__device__ __forceinline__ void lowk_recurrence(TCm* zx, TCm* zy, TCm* w, int ld, const TCm* a, const TCm* c,
                                                const TCm* W, int nz, int kx, int ky, bool singular,
                                                const double* __restrict__ lamx, const double* __restrict__ lamy,
                                                double scale, const double* __restrict__ target_mean,
                                                Stats* stats, TCm* red, double* sq_out, bool tab = false) {
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
    // the pivots depend on the column's wavenumbers and the levels only: staged from the plan's
    // table when it has them (no division on the chain), else computed here
    const TCm inv = tab ? w[k * ld]
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
      if (!tab) w[k * ld] = (TCm)c[k] * inv;
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
      if (!tab) w[k * ld] = (k + 1 < nz) ? (TCm)a[k + 1] * inv : (TCm)0;
    }
    inv_prev = inv;
  }
  TCm xx = zx[(nz - 1) * ld], xy = zy[(nz - 1) * ld];
  TCm sx = xx, sy = xy;
  for (int k = nz - 2; k >= 0; --k) {
    const TCm wk = !tab ? w[k * ld] : (ADJ ? (TCm)a[k + 1] * w[k * ld] : (TCm)c[k] * w[k * ld]);
    xx = zx[k * ld] + wk * xx;
    xy = zy[k * ld] + wk * xy;
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

// Shared memory (in units of the compute type) of one low-|k| column solved by a block.
__host__ __device__ constexpr size_t lowk_smem_elems(int nz) { return 6 * (size_t)nz + 96; }

// Fixed-order sum of three values over the block (every thread gets the result): each thread's
// values, then a shuffle tree in each warp, then the warps in order.  scratch: 3 doubles per warp.
__device__ __forceinline__ double3 lowk_block_sum3(double v0, double v1, double v2, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, o);
    v1 += __shfl_down_sync(0xffffffffu, v1, o);
    v2 += __shfl_down_sync(0xffffffffu, v2, o);
  }
  const int wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();   // scratch may still be read from an earlier sum
  if ((threadIdx.x & 31) == 0) {
    scratch[3 * wid] = v0;
    scratch[3 * wid + 1] = v1;
    scratch[3 * wid + 2] = v2;
  }
  __syncthreads();
  double3 r = make_double3(0.0, 0.0, 0.0);
  for (int w = 0; w < nw; ++w) {
    r.x += scratch[3 * w];
    r.y += scratch[3 * w + 1];
    r.z += scratch[3 * w + 2];
  }
  return r;
}

// One low-|k| or singular column in double precision from the plan's pivot table (inv_col: 1/u_k,
// 0 for the pinned singular top), solved by the whole block (at most 1024 threads).  The FP64 units
// issue a warp's instruction at the same cost however few of its lanes are active, so the serial
// part is kept to the two recurrences alone: the real parts run on lane 0 and the imaginary parts on
// lane 1 of the first warp (one double FMA instruction per level and sweep), and everything that
// does not depend on the previous level (the scaled right-hand side, the elimination and
// back-substitution factors, the means and sums) runs across the block.
//   forward  (M x = b):   y_k = b_k + (a_k/u_{k-1}) y_{k-1},  z_k = y_k/u_k,  x_k = z_k + (c_k/u_k) x_{k+1}
//   adjoint (M^T x = b):  v_k = (b_k + c_{k-1} v_{k-1})/u_k,                  x_k = v_k + (a_{k+1}/u_k) x_{k+1}
template <typename TS, bool ADJ>
__device__ __forceinline__ void lowk_column_tab(unsigned char* smraw, typename CT<TS>::t* __restrict__ spec,
                                                const Geom& g, const double* __restrict__ ag,
                                                const double* __restrict__ cg, const double* __restrict__ Wg,
                                                const double* __restrict__ lamx, const double* __restrict__ lamy,
                                                double scale, int2 colk, Stats* stats,
                                                const double* __restrict__ target_mean, bool singular00,
                                                double* sq_out, const double* __restrict__ inv_col) {
  using CS = typename CT<TS>::t;
  const int nz = g.nz, t = threadIdx.x, nt = blockDim.x;
  double* z = reinterpret_cast<double*>(smraw);   // [2][nz]: real parts, imaginary parts
  double* inv = z + 2 * nz;                        // 1/u_k, then the back-substitution factors
  double* F = inv + nz;                            // forward factors
  double* scratch = F + nz;                        // [3 per warp]
  const int kx = colk.x, ky = colk.y;
  const bool singular = singular00 && kx == 0 && ky == 0;   // nonsingular with p = 0 on the top face
  CS* colp = spec + (long long)ky * g.P + kx;
  // the column is read at L2 (not through L1), so that a persistent kernel that produced it earlier
  // in the same launch on another SM is seen
  double mx = 0.0, my = 0.0, sw = 0.0;
  for (int k = t; k < nz; k += nt) {
    const CS v = __ldcg(&colp[(long long)k * g.plane]);
    z[k] = (double)v.x;
    z[nz + k] = (double)v.y;
    inv[k] = __ldg(inv_col + k);
    if (singular) {   // compatibility: the W-weighted (adjoint: plain) mean of the right-hand side
      const double wk = ADJ ? 1.0 : __ldg(Wg + k);
      mx += wk * (double)v.x;
      my += wk * (double)v.y;
      sw += wk;
    }
  }
  double mean_x = 0.0, mean_y = 0.0;
  if (singular) {
    const double3 m = lowk_block_sum3(mx, my, sw, scratch);
    mean_x = m.x / m.z;
    mean_y = m.y / m.z;
    // only the first solve records mu_W (a refinement correction solve has a target mean)
    if (!ADJ && t == 0 && stats && !target_mean) stats->mu_w = mean_x * scale;
  }
  __syncthreads();
  const double ms = -scale;
  for (int k = t; k < nz; k += nt) {
    z[k] = ms * (z[k] - mean_x);
    z[nz + k] = ms * (z[nz + k] - mean_y);
    F[k] = k == 0 ? 0.0 : (ADJ ? __ldg(cg + k - 1) : __ldg(ag + k) * inv[k - 1]);
  }
  __syncthreads();
  if (t < 2) {   // forward elimination: lane 0 the real parts, lane 1 the imaginary parts
    double* zp = z + t * nz;
    double y = ADJ ? zp[0] * inv[0] : zp[0];
    zp[0] = y;
    for (int k = 1; k < nz; ++k) {
      y = fma(F[k], y, zp[k]);
      if (ADJ) y *= inv[k];
      zp[k] = y;
    }
  }
  __syncthreads();
  for (int k = t; k < nz; k += nt) {
    const double u = inv[k];
    if (!ADJ) {
      z[k] *= u;
      z[nz + k] *= u;
      inv[k] = __ldg(cg + k) * u;
    } else {
      inv[k] = k + 1 < nz ? __ldg(ag + k + 1) * u : 0.0;
    }
  }
  __syncthreads();
  if (t < 2) {   // back substitution
    double* zp = z + t * nz;
    double x = zp[nz - 1];
    for (int k = nz - 2; k >= 0; --k) {
      x = fma(inv[k], x, zp[k]);
      zp[k] = x;
    }
  }
  __syncthreads();
  double shx = 0.0, shy = 0.0, fx = 0.0, fy = 0.0;
  if (singular) {
    double sx = 0.0, sy = 0.0, swt = 0.0;
    for (int k = t; k < nz; k += nt) {
      sx += z[k];
      sy += z[nz + k];
      if (ADJ) swt += __ldg(Wg + k);
    }
    const double3 r = lowk_block_sum3(sx, sy, swt, scratch);
    if (!ADJ) {
      shx = r.x / (double)nz;
      shy = r.y / (double)nz;
      // refinement sweep: the correction also removes the mean of the current iterate
      if (target_mean) shx += __ldcg(target_mean);
    } else {   // remove the W direction (the null vector of the transposed column)
      fx = r.x / r.z;
      fy = r.y / r.z;
    }
  }
  double sq = 0.0;
  for (int k = t; k < nz; k += nt) {
    double ox = z[k], oy = z[nz + k];
    if (singular) {
      if (!ADJ) {
        ox -= shx;
        oy -= shy;
      } else {
        const double wk = __ldg(Wg + k);
        ox -= wk * fx;
        oy -= wk * fy;
      }
    }
    if (!ADJ && sq_out) sq += ox * ox + oy * oy;
    CS o;
    o.x = (TS)ox;
    o.y = (TS)oy;
    colp[(long long)k * g.plane] = o;
  }
  if (!ADJ && sq_out) {
    const double3 r = lowk_block_sum3(sq, 0.0, 0.0, scratch);
    if (t == 0) *sq_out = r.x;
  }
}

// One low-|k| or singular column, solved by the whole block.  With the plan's pivot table (double
// columns) this is lowk_column_tab; otherwise the strided loads and stores of the column and the
// coefficient tables go through shared memory in parallel and thread 0 runs the sequential
// recurrence out of shared memory.  sq_out (nullable): the solution's sum of |x_k|^2 over the
// levels (forward solve), stored by thread 0.  Shared memory: lowk_smem_elems(nz) of TCm.
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
  if (inv_tab && sizeof(TCm) == 8) {   // the plan's pivot table holds double pivots
    lowk_column_tab<TS, ADJ>(smraw, spec, g, ag, cg, Wg, lamx, lamy, scale, colk, stats, target_mean, singular00,
                             sq_out, inv_tab + (size_t)col_index * nz);
    return;
  }
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
                              red, sq_out);
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
