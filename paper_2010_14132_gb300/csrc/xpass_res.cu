// Persistent forward x-pass of a refinement sweep: the transformed rows are the residual.
// (Section 2.1: the x transform of every row of every level; see xpass_common.cuh
// for the persistent staging scheme the kernels share.)
#include "xpass_common.cuh"

// This file is compiled twice: PGB_XRES_ISO 0 here (the general kernels and the dispatcher), and 1
// from xpass_res_iso.cu (the dx == dy kernels), so that the two sets of instances build in parallel.
#ifndef PGB_XRES_ISO
#define PGB_XRES_ISO 0
#endif

namespace pgb {
namespace {

// ---------------------------------------------------------------------------
// forward x-pass of a refinement sweep: the rows transformed are the residual
// r = S - mu_W - L (p0 + q), formed as the group is read.  The group's rows of S,
// p0 (and q) are staged; the x-neighbours come from the staged rows, the y- and
// z-neighbour rows are read through L1/L2 (the neighbouring groups stage them).
// ---------------------------------------------------------------------------
// CTAs per SM the register budget is set for: the correction q's extra stencil values spill at
// three CTAs of 256 threads (80 registers), so the q variant takes two (PGB_XRES_Q_BLOCKS)
#ifndef PGB_XRES_Q_BLOCKS
#define PGB_XRES_Q_BLOCKS 2
#endif
#ifndef PGB_XRES_E3_BLOCKS
#define PGB_XRES_E3_BLOCKS 2
#endif
// (the r0 - L q form holds no S or p0 stencil values: three CTAs, like the first sweep's)
constexpr int xres_min_blocks(int e, bool has_q, bool from_r0 = false) {
  return e % 3 == 0 ? PGB_XRES_E3_BLOCKS : (e >= 16 ? 4 : (has_q && !from_r0 ? PGB_XRES_Q_BLOCKS : 3));
}
// FROM_R0 (with HAS_Q): the rows staged are sweep 1's FP32 residual r0 and the correction q (one bulk
// copy each per row, side by side in the row's slot, whose full width the line buffers need later) and
// r = r0 - L q.
template <int N, int E, bool HAS_Q, bool STAGE_P, bool ISO, bool FROM_R0 = false>
__global__ void __launch_bounds__(xs_threads(E), xres_min_blocks(E, HAS_Q, FROM_R0)) k_xres_s(ResidualArgs R, float2* __restrict__ spec, Geom g,
                                                      const float2* __restrict__ twx, const float2* __restrict__ twr,
                                                      const int* __restrict__ done, unsigned* __restrict__ err,
                                                      int ns, unsigned stage_bytes) {
  using C = float2;
  constexpr int nl = N / E, RB = xs_threads(E) / nl, LS = swizzled_stride(N), NX = 2 * N;
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smraw[];
  const XsLayout L = xs_layout(N, RB, ns, stage_bytes, true);
  C* tw_s = reinterpret_cast<C*>(smraw);
  C* twr_s = tw_s + N;
  C* lines = twr_s + N + 2;
  unsigned char* stg = smraw + L.off_stage;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + L.off_bar);

  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * nl + lane;
  const long long row_begin = (long long)g.lev0 * g.ny, row_end = (long long)g.lev1 * g.ny;
  const long long ngroups = (row_end - row_begin + RB - 1) / RB;
  constexpr unsigned s_bytes = RB * NX * 8, p_bytes = STAGE_P ? RB * NX * 4 : 0;
  st_build_twiddles<N, E>(tw_s, twx, tid, xs_threads(E));
  for (int t = tid; t <= N / 2; t += xs_threads(E)) twr_s[t] = twr[t];
  Ring rg{};
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  pdl_wait();   // the previous kernels of the stream are complete
  if (done && *done) return;
  static_assert(!FROM_R0 || (HAS_Q && !STAGE_P), "r0 - L q is formed with q, from the staged r0 rows");
  auto issue = [&](long long grp, int s) {
    const long long r0 = row_begin + grp * RB;
    const unsigned nv = (unsigned)(row_end - r0 < RB ? row_end - r0 : RB);
    unsigned char* d = stg + (size_t)s * stage_bytes;
    if constexpr (FROM_R0) {
      mbar_arrive_expect_tx(&bar[s], nv * NX * 8u);
      for (unsigned j = 0; j < nv; ++j) {
        bulk_g2s(d + (size_t)j * NX * 8, R.r0 + (r0 + j) * R.r_ld, NX * 4u, &bar[s]);
        bulk_g2s(d + (size_t)j * NX * 8 + NX * 4, R.q + (r0 + j) * NX, NX * 4u, &bar[s]);
      }
      rg.issued[s]++;
      return;
    }
    mbar_arrive_expect_tx(&bar[s], nv * NX * (8u + (STAGE_P ? 4u + (HAS_Q ? 4u : 0u) : 0u)));
    bulk_g2s(d, R.S + r0 * NX, nv * NX * 8u, &bar[s]);
    if constexpr (STAGE_P) {
      bulk_g2s(d + s_bytes, R.p0 + r0 * NX, nv * NX * 4u, &bar[s]);
      if constexpr (HAS_Q) bulk_g2s(d + s_bytes + p_bytes, R.q + r0 * NX, nv * NX * 4u, &bar[s]);
    }
    rg.issued[s]++;
  };
  if (tid == 0)
    for (int s = 0; s < ns; ++s) {
      const long long grp = blockIdx.x + (long long)s * gridDim.x;
      if (grp < ngroups) issue(grp, s);
    }
  const LineSync sync{1 + ty, nl};
  const Swizzled sw{};
  (void)lines;
  const float2 cx = R.cx, cy = R.cy;   // double-float splits of 1/dx^2, 1/dy^2
  float2 racc = make_float2(0.f, 0.f), sacc = racc;   // per-lane sums of r^2 and S^2 (even / odd points)
  bool ok = true;
  int it = 0;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++it) {
    const int s = it % ns;
    const long long row = row_begin + grp * RB + ty;
    const bool valid = row < row_end;
    const long long rc = valid ? row : row_begin;   // neighbour addressing stays inside the field
    const int k = (int)(rc / g.ny), j = (int)(rc - (long long)k * g.ny);
    const long long rn = rc - j + (j + 1 == g.ny ? 0 : j + 1), rs = rc - j + (j == 0 ? g.ny - 1 : j - 1);
    const bool has_dn = k > 0, has_up = k + 1 < g.nz;
    const float2* p0n = reinterpret_cast<const float2*>(R.p0 + rn * NX);
    const float2* p0s = reinterpret_cast<const float2*>(R.p0 + rs * NX);
    const float2* p0d = reinterpret_cast<const float2*>(R.p0 + (has_dn ? rc - g.ny : rc) * NX);
    const float2* p0u = reinterpret_cast<const float2*>(R.p0 + (has_up ? rc + g.ny : rc) * NX);
    const ResCoef K = res_coef(cx, cy, R.a_ff[k], R.c_ff[k], *R.mu_ff);
    const bool got = mbar_wait_bounded(&bar[s], (unsigned)((it / ns) & 1), kWaitPolls);
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      rg.consumed[s]++;
      if (it > 0) {
        const long long gn = grp - gridDim.x + (long long)ns * gridDim.x;
        if (gn < ngroups) {
          fence_proxy_async_smem();
          issue(gn, (it - 1) % ns);
        }
      }
    }
    unsigned char* d = stg + (size_t)s * stage_bytes;
    const double2* Srow = reinterpret_cast<const double2*>(d) + (size_t)ty * N;
    // the row's two line buffers are its staged S row (used once the residual is formed)
    C* la = reinterpret_cast<C*>(d + (size_t)ty * NX * 8);
    C* lb = la + LS;
    // centre rows of p0 and q: staged, or read through L1 next to the other neighbours
    const float* prow = STAGE_P ? reinterpret_cast<const float*>(d + s_bytes) + (size_t)ty * NX : R.p0 + rc * NX;
    const float* qrow = STAGE_P ? reinterpret_cast<const float*>(d + s_bytes + p_bytes) + (size_t)ty * NX
                                : (HAS_Q ? R.q + rc * NX : nullptr);
    C v[E];
    if constexpr (FROM_R0) {
      const float2* r0row = reinterpret_cast<const float2*>(d + (size_t)ty * NX * 8);
      const float* qs_row = reinterpret_cast<const float*>(d + (size_t)ty * NX * 8 + NX * 4);   // staged q row
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int e = st_in_index<N, E, 0>(lane, i);
        const float2 qc = reinterpret_cast<const float2*>(qs_row)[e];
        const float qw = qs_row[e == 0 ? NX - 1 : 2 * e - 1];
        const float qe = qs_row[e == N - 1 ? 0 : 2 * e + 2];
        const float2 qn = reinterpret_cast<const float2*>(R.q + rn * NX)[e];
        const float2 qs = reinterpret_cast<const float2*>(R.q + rs * NX)[e];
        const float2 qd = has_dn ? reinterpret_cast<const float2*>(R.q + (rc - g.ny) * NX)[e] : qc;
        const float2 qu = has_up ? reinterpret_cast<const float2*>(R.q + (rc + g.ny) * NX)[e] : make_float2(0.f, 0.f);
        // the pair's east neighbours are (qc.y, qe), its west neighbours (qw, qc.x)
        v[i] = residual_from_r0<ISO>(r0row[e], qc, make_float2(qc.y, qe), make_float2(qw, qc.x), qn, qs, qd, qu, K);
        if (valid) {
          racc = fma2(v[i], v[i], racc);
          if (R.p_out) {   // the iterate p0 + q as the double the inverse x-pass would store
            const float2 pc = reinterpret_cast<const float2*>(prow)[e];
            float2 sp, tp;
            two_sum2(pc, qc, sp, tp);
            __stcs(reinterpret_cast<double2*>(R.p_out + row * NX) + e,
                   make_double2(ff2d_fast(sp.x, tp.x), ff2d_fast(sp.y, tp.y)));
          }
        }
      }
    } else {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int e = st_in_index<N, E, 0>(lane, i);
      const float2 pc = reinterpret_cast<const float2*>(prow)[e];
      const float pw = prow[e == 0 ? NX - 1 : 2 * e - 1];
      const float pe = prow[e == N - 1 ? 0 : 2 * e + 2];
      const float2 pn = p0n[e], ps = p0s[e];
      const float2 pd = has_dn ? p0d[e] : pc, pu = has_up ? p0u[e] : make_float2(0.f, 0.f);
      float2 qc = make_float2(0.f, 0.f), qn = qc, qs = qc, qd = qc, qu = qc;
      float qw = 0.f, qe = 0.f;
      if constexpr (HAS_Q) {
        qc = reinterpret_cast<const float2*>(qrow)[e];
        qw = qrow[e == 0 ? NX - 1 : 2 * e - 1];
        qe = qrow[e == N - 1 ? 0 : 2 * e + 2];
        qn = reinterpret_cast<const float2*>(R.q + rn * NX)[e];
        qs = reinterpret_cast<const float2*>(R.q + rs * NX)[e];
        qd = has_dn ? reinterpret_cast<const float2*>(R.q + (rc - g.ny) * NX)[e] : qc;
        qu = has_up ? reinterpret_cast<const float2*>(R.q + (rc + g.ny) * NX)[e] : make_float2(0.f, 0.f);
      }
      const double2 S = Srow[e];
      float2 Sh, Sl;
      d2ff_trunc(S.x, Sh.x, Sl.x);
      d2ff_trunc(S.y, Sh.y, Sl.y);
      // the pair's east neighbours are (pc.y, pe), its west neighbours (pw, pc.x)
      v[i] = residual_value2<HAS_Q, ISO>(pc, make_float2(pc.y, pe), make_float2(pw, pc.x), pn, ps, pd, pu, qc,
                                    make_float2(qc.y, qe), make_float2(qw, qc.x), qn, qs, qd, qu, Sh, Sl, K);
      if (valid) {
        racc = fma2(v[i], v[i], racc);
        sacc = fma2(Sh, Sh, sacc);
        if constexpr (!HAS_Q) {   // sweep 1's residual, kept for the verification's first try
          if (R.r_out) __stcs(reinterpret_cast<float2*>(R.r_out + row * R.r_ld) + e, v[i]);
        }
        if constexpr (HAS_Q) {
          if (R.p_out) {   // the iterate p0 + q as the double the inverse x-pass would store
            float2 sp, tp;
            two_sum2(pc, qc, sp, tp);
            __stcs(reinterpret_cast<double2*>(R.p_out + row * NX) + e,
                   make_double2(ff2d_fast(sp.x, tp.x), ff2d_fast(sp.y, tp.y)));
          }
        }
      }
    }
    }
    sync();   // the line's threads have read the staged row before it is overwritten
    const C* fin = st_fft<N, E, -1, false, float>(v, la, lb, sw, lane, tw_s, sync);
    r2c_unpack_store<N, E>(fin, twr_s, spec + (valid ? row : 0) * g.P, lane, valid, R.kmax > 0 ? R.kmax : N);
    fence_proxy_async_smem();   // generic writes to the staged row come before its refill by TMA
  }
  if (tid == 0) {
    if (!ok) atomicOr(err, (unsigned)ERR_WAIT_TIMEOUT);
    ring_drain(rg, bar, ns);
  }
  // per-CTA sums of r^2 and S^2 (fixed-order tree) in the drained staging ring
  constexpr int TH = xs_threads(E);
  static_assert((size_t)TH * 8 <= (size_t)RB * NX * 8, "reduction does not fit the staging ring");
  __syncthreads();
  float (*red)[TH] = reinterpret_cast<float (*)[TH]>(stg);
  red[0][tid] = racc.x + racc.y;
  red[1][tid] = sacc.x + sacc.y;
  __syncthreads();
  for (int h = TH / 2; h > 0; h >>= 1) {
    if (tid < h) {
      red[0][tid] += red[0][tid + h];
      red[1][tid] += red[1][tid + h];
    }
    __syncthreads();
  }
  if (tid == 0 && R.partials) {
    const long long slot = R.part0 + blockIdx.x;
    R.partials[2 * slot] = (double)red[0][0];
    R.partials[2 * slot + 1] = (double)red[1][0];
  }
}

template <bool HAS_Q, bool ISO>
cudaError_t xres_s(const ResidualArgs& R, float2* spec, const Geom& g, int N, int E, const Tables& tb,
                   const int* done, unsigned* err, int* nblocks_out, cudaStream_t st, bool* used) {
  const int RB = xs_threads(E) / (N / E);
  // stage S, p0 (and q) rows while three CTAs per SM still fit, else S rows only
  const unsigned row_bytes_all = (unsigned)(g.nx * (8 + 4 + (HAS_Q ? 4 : 0)));
  const unsigned row_bytes_s = (unsigned)(g.nx * 8);
  const XsConfig c_all = xs_config(N, E, RB * row_bytes_all, 0, true);
  const bool stage_p = c_all.ns > 0 && c_all.smem <= 75 * 1024 * (size_t)xs_threads(E) / 256;
  const XsConfig c = stage_p ? c_all : xs_config(N, E, RB * row_bytes_s, 0, true);
  const long long ngroups = ((long long)g.ny * (g.lev1 - g.lev0) + RB - 1) / RB;
  if constexpr (HAS_Q) {
    if (R.r0) {   // the first try's r0 - L q: r0 rows staged in slots of an S row's width
      const XsConfig c0 = xs_config(N, E, RB * row_bytes_s, 0, true);
      if (c0.ns == 0 || !aligned16(R.r0) || (R.r_ld * 4) % 16 || !aligned16(R.p0) || !aligned16(R.q) ||
          (g.nx * 4) % 16)
        return cudaSuccess;
      PGB_XS_E8_E3_SWITCH(E, PGB_XS_N_SWITCH(N, {
        return xs_launch(k_xres_s<NN, EE, true, false, ISO, true>, NN / EE, RB, c0, ngroups, nblocks_out, st, used,
                         R, spec, g, tb.twx_f, tb.twr_f, done, err);
      }));
      return cudaSuccess;
    }
  }
  if (c.ns == 0 || !aligned16(R.S) || !aligned16(R.p0) || (HAS_Q && !aligned16(R.q)) || (g.nx * 4) % 16)
    return cudaSuccess;
  if (stage_p) {
    PGB_XS_E8_E3_SWITCH(E, PGB_XS_N_SWITCH(N, {
      return xs_launch(k_xres_s<NN, EE, HAS_Q, true, ISO>, NN / EE, RB, c, ngroups, nblocks_out, st, used, R, spec, g,
                       tb.twx_f, tb.twr_f, done, err);
    }));
  } else {
    PGB_XS_E8_E3_SWITCH(E, PGB_XS_N_SWITCH(N, {
      return xs_launch(k_xres_s<NN, EE, HAS_Q, false, ISO>, NN / EE, RB, c, ngroups, nblocks_out, st, used, R, spec, g,
                       tb.twx_f, tb.twr_f, done, err);
    }));
  }
  return cudaSuccess;
}

}  // namespace

#if PGB_XRES_ISO
cudaError_t launch_xres_static_iso(const ResidualArgs& R, void* spec, const Geom& g, const FftPlan& fx,
                                   const Tables& tb, const int* done, unsigned* err, int* nblocks_out,
                                   cudaStream_t st, bool* used) {
  const int E = fx.n % 3 == 0 ? kE3 : 8;
  if (R.q) return xres_s<true, true>(R, (float2*)spec, g, fx.n, E, tb, done, err, nblocks_out, st, used);
  return xres_s<false, true>(R, (float2*)spec, g, fx.n, E, tb, done, err, nblocks_out, st, used);
}
#else
cudaError_t launch_xres_static_iso(const ResidualArgs& R, void* spec, const Geom& g, const FftPlan& fx,
                                   const Tables& tb, const int* done, unsigned* err, int* nblocks_out,
                                   cudaStream_t st, bool* used);

cudaError_t launch_xres_static(const ResidualArgs& R, void* spec, const Geom& g, const FftPlan& fx, const Tables& tb,
                               const int* done, unsigned* err, int* nblocks_out, cudaStream_t st, bool* used) {
  *used = false;
  if (!xpass_static_supported(fx.n)) return cudaSuccess;
  const int E = fx.n % 3 == 0 ? kE3 : 8;   // the residual kernel: 8 elements per thread for powers of two
  // dx == dy: the kernels with the merged horizontal term
  if (R.cx.x == R.cy.x && R.cx.y == R.cy.y)
    return launch_xres_static_iso(R, spec, g, fx, tb, done, err, nblocks_out, st, used);
  if (R.q) return xres_s<true, false>(R, (float2*)spec, g, fx.n, E, tb, done, err, nblocks_out, st, used);
  return xres_s<false, false>(R, (float2*)spec, g, fx.n, E, tb, done, err, nblocks_out, st, used);
}
#endif

}  // namespace pgb
