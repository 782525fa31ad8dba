// Persistent inverse x-pass (C2R) with the solver's epilogues.
// (Section 2.1: the x transform of every row of every level; see xpass_common.cuh
// for the persistent staging scheme the kernels share.)
#include "xpass_common.cuh"

namespace pgb {
namespace {

// ---------------------------------------------------------------------------
// inverse x-pass with the solver's epilogues
// ---------------------------------------------------------------------------
// Three CTAs per SM for 8 or 16 elements per thread: the update epilogue otherwise takes 124 registers,
// which caps it at two.  With 24 elements (lengths with a factor 3) that bound would spill, so those
// kernels keep their registers.
#ifndef PGB_XINV_MIN_BLOCKS
#define PGB_XINV_MIN_BLOCKS 3
#endif
#ifndef PGB_XINV_E3_BLOCKS
#define PGB_XINV_E3_BLOCKS 2
#endif
constexpr int xinv_min_blocks(int e) { return e % 3 == 0 ? PGB_XINV_E3_BLOCKS : PGB_XINV_MIN_BLOCKS; }
template <int N, int E, typename TO, int MODE>
__global__ void __launch_bounds__(xs_threads(E), xinv_min_blocks(E)) k_xinv_s(const float2* __restrict__ spec, TO* __restrict__ out, Geom g,
                                                      const float2* __restrict__ twx, const float2* __restrict__ twr,
                                                      XinvExtra ex, int ns, unsigned stage_bytes) {
  using C = float2;
  constexpr int nl = N / E, RB = xs_threads(E) / nl, LS = swizzled_stride(N);
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smraw[];
  const XsLayout L = xs_layout(N, RB, ns, stage_bytes, false);
  C* tw_s = reinterpret_cast<C*>(smraw);
  C* twr_s = tw_s + N;
  C* lines = twr_s + N + 2;
  unsigned char* stg = smraw + L.off_stage;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + L.off_bar);

  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * nl + lane;
  const long long row_begin = (long long)g.lev0 * g.ny, row_end = (long long)g.lev1 * g.ny;
  const long long ngroups = (row_end - row_begin + RB - 1) / RB;
  const unsigned row_bytes = (unsigned)xs_align((size_t)(N + 1) * sizeof(C), 16);
  st_build_twiddles<N, E>(tw_s, twx, tid, xs_threads(E));
  for (int t = tid; t <= N; t += xs_threads(E)) twr_s[t] = twr[t];
  Ring rg{};
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  pdl_wait();   // the previous kernels of the stream are complete
  if (ex.done && *ex.done) return;
  auto issue = [&](long long grp, int s) {
    const long long r0 = row_begin + grp * RB;
    const int nv = (int)(row_end - r0 < RB ? row_end - r0 : RB);
    mbar_arrive_expect_tx(&bar[s], (unsigned)nv * row_bytes);
    for (int r = 0; r < nv; ++r)
      bulk_g2s(stg + (size_t)s * stage_bytes + (size_t)r * row_bytes, spec + (r0 + r) * g.P, row_bytes, &bar[s]);
    rg.issued[s]++;
  };
  if (tid == 0)
    for (int s = 0; s < ns; ++s) {
      const long long grp = blockIdx.x + (long long)s * gridDim.x;
      if (grp < ngroups) issue(grp, s);
    }
  const LineSync sync{1 + ty, nl};
  const Swizzled sw{};
  C* la = lines + (size_t)ty * 2 * LS;
  C* lb = la + LS;
  // per-lane partial sums (even / odd points): delta^2, p^2 and the double-float sum of p
  float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0, sh = acc0, sl = acc0;
  bool ok = true;
  int it = 0;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++it) {
    const int s = it % ns;
    const long long row = row_begin + grp * RB + ty;
    const bool valid = row < row_end;
    const long long base = (valid ? row : 0) * g.nx;
    // epilogue operands, fetched before the transform so that their latency is hidden
    float2 p0v[E], qv[E];
    if constexpr (MODE == XINV_UPDATE) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int m = st_out_index<N, E>(lane, i);
        p0v[i] = valid ? reinterpret_cast<const float2*>(ex.p0 + base)[m] : make_float2(0.f, 0.f);
        qv[i] = (valid && ex.q_valid) ? reinterpret_cast<const float2*>(ex.q + base)[m] : make_float2(0.f, 0.f);
      }
    }
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
    const C* X = reinterpret_cast<const C*>(stg + (size_t)s * stage_bytes + (size_t)ty * row_bytes);
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int m = st_in_index<N, E, 0>(lane, i);
      C xk = X[m];
      C xc = cconj(X[N - m]);
      if (m == 0) {   // self-conjugate bins: real parts only
        xk.y = 0.f;
        xc.y = 0.f;
      }
      const C ev = cadd(xk, xc);
      const C od = cmul(csub(xk, xc), cconj(twr_s[m]));   // * exp(+2 pi i m/n)
      v[i] = make_float2(ev.x - od.y, ev.y + od.x);        // ev + i od
    }
    st_fft<N, E, +1, true, float>(v, la, lb, sw, lane, tw_s, sync);
    if (valid) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int m = st_out_index<N, E>(lane, i);
        const C z = v[i];
        if constexpr (MODE == XINV_PLAIN) {
          typename V2s<TO>::t o;
          o.x = Cvt<float, TO>::f(z.x);
          o.y = Cvt<float, TO>::f(z.y);
          __stcs(reinterpret_cast<typename V2s<TO>::t*>(out + base) + m, o);
        } else if constexpr (MODE == XINV_P0) {
          __stcs(reinterpret_cast<float2*>(ex.p0 + base) + m, z);
          acc1 = fma2(z, z, acc1);
          float2 e;
          two_sum2(sh, z, sh, e);
          sl = add2(sl, e);
          if (ex.p_out)
            __stcs(reinterpret_cast<double2*>(ex.p_out + base) + m, make_double2(f2d_int(z.x), f2d_int(z.y)));
        } else {   // XINV_UPDATE: q + delta stored as the new q and/or p = p0 + (q + delta) as a double
          const float2 qn = add2(z, qv[i]);
          if (ex.q_out) __stcs(reinterpret_cast<float2*>(ex.q_out + base) + m, qn);
          float2 sp, tp;
          two_sum2(p0v[i], qn, sp, tp);
          if (ex.p_out)
            __stcs(reinterpret_cast<double2*>(ex.p_out + base) + m,
                   make_double2(ff2d_fast(sp.x, tp.x), ff2d_fast(sp.y, tp.y)));
          acc0 = fma2(z, z, acc0);
          acc1 = fma2(sp, sp, acc1);
          float2 e;
          two_sum2(sh, sp, sh, e);
          sl = add2(sl, add2(e, tp));
        }
      }
    }
  }
  if (tid == 0) {
    if (!ok) atomicOr(ex.err, (unsigned)ERR_WAIT_TIMEOUT);
    ring_drain(rg, bar, ns);
  }
  if constexpr (MODE != XINV_PLAIN) {
    // deterministic CTA partial sums: fixed-order tree over the CTA's threads, in the
    // line buffers (no longer in use: every thread is past its last transform)
    constexpr int TH = xs_threads(E);
    static_assert((size_t)TH * 40 <= (size_t)RB * 2 * LS * sizeof(C), "reduction does not fit the line buffers");
    __syncthreads();
    double* redd = reinterpret_cast<double*>(lines);
    float (*red)[TH] = reinterpret_cast<float (*)[TH]>(redd + TH);
    red[0][tid] = acc0.x + acc0.y;
    red[1][tid] = acc1.x + acc1.y;
    redd[tid] = (f2d_int(sh.x) + f2d_int(sl.x)) + (f2d_int(sh.y) + f2d_int(sl.y));
    __syncthreads();
    for (int h = xs_threads(E) / 2; h > 0; h >>= 1) {
      if (tid < h) {
        red[0][tid] += red[0][tid + h];
        red[1][tid] += red[1][tid + h];
        redd[tid] += redd[tid + h];
      }
      __syncthreads();
    }
    __shared__ bool last;
    if (tid == 0) {
      const long long slot = ex.part0 + blockIdx.x;
      ex.partials[3 * slot] = (double)red[0][0];
      ex.partials[3 * slot + 1] = (double)red[1][0];
      ex.partials[3 * slot + 2] = redd[0];
      last = false;
      if (ex.ctl_stats) {
        __threadfence();
        last = atomicAdd(&ex.ctl_stats->control_ticket, 1u) == gridDim.x - 1;
      }
    }
    __syncthreads();
    if (last) {
      // the last CTA to finish sums every CTA's partials in a fixed order and runs the control
      __threadfence();
      double* sums = redd;   // [5][TH] in the line buffers
      double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
      for (int i = tid; i < (int)gridDim.x; i += TH) {
        const long long slot = ex.part0 + i;
        a0 += __ldcg(&ex.partials[3 * slot]);
        a1 += __ldcg(&ex.partials[3 * slot + 1]);
        a2 += __ldcg(&ex.partials[3 * slot + 2]);
      }
      for (int i = tid; i < ex.res_nblocks; i += TH) {   // the sweep's residual norms (forward x-pass)
        a3 += __ldcg(&ex.res_partials[2 * i]);
        a4 += __ldcg(&ex.res_partials[2 * i + 1]);
      }
      __syncthreads();
      sums[tid] = a0;
      sums[TH + tid] = a1;
      sums[2 * TH + tid] = a2;
      sums[3 * TH + tid] = a3;
      sums[4 * TH + tid] = a4;
      __syncthreads();
      for (int h = TH / 2; h > 0; h >>= 1) {
        if (tid < h) {
#pragma unroll
          for (int v = 0; v < 5; ++v) sums[v * TH + tid] += sums[v * TH + tid + h];
        }
        __syncthreads();
      }
      if (tid == 0) {
        ex.ctl_stats->control_ticket = 0u;   // ready for the next pass
        control_decide(ex.ctl_stats, sums[0], sums[TH], sums[2 * TH], sums[3 * TH], sums[4 * TH], ex.ctl_pass,
                       ex.ctl_max_sweeps, ex.ctl_tol, ex.ctl_npoints, ex.p_out != nullptr, *ex.ctl_floor);
      }
    }
  }
}

template <typename TO, int MODE>
cudaError_t xinv_s(const float2* spec, TO* out, const Geom& g, int N, int E, const Tables& tb, const XinvExtra& ex,
                   int* nblocks_out, cudaStream_t st, bool* used) {
  const int RB = xs_threads(E) / (N / E);
  const unsigned row_bytes = (unsigned)xs_align((size_t)(N + 1) * sizeof(float2), 16);
  if ((size_t)g.P * sizeof(float2) < row_bytes || (g.P * sizeof(float2)) % 16 || !aligned16(spec)) return cudaSuccess;
  const XsConfig c = xs_config(N, E, RB * row_bytes, 0, false);
  if (c.ns == 0) return cudaSuccess;
  const long long ngroups = ((long long)g.ny * (g.lev1 - g.lev0) + RB - 1) / RB;
  PGB_XS_E_SWITCH(E, PGB_XS_N_SWITCH(N, {
    return xs_launch(k_xinv_s<NN, EE, TO, MODE>, NN / EE, RB, c, ngroups, nblocks_out, st, used, spec, out, g,
                     tb.twx_f, tb.twr_f, ex);
  }));
  return cudaSuccess;
}

}  // namespace

bool xpass_static_supported(int n_half) {
  switch (n_half) {
    case 32: case 64: case 96: case 128: case 192: case 256: case 384: case 512: case 768: case 1024: case 2048:
      return true;
    default: return false;
  }
}

cudaError_t launch_xinv_static(int to_is_double, int mode, const void* spec, void* out, const Geom& g,
                               const FftPlan& fx, const Tables& tb, const XinvExtra& ex, int* nblocks_out,
                               cudaStream_t st, bool* used) {
  *used = false;
  if (!xpass_static_supported(fx.n)) return cudaSuccess;
  const float2* sp = (const float2*)spec;
  const int E = xs_elems(fx.n, fx.E);
  if (mode == XINV_P0) return xinv_s<float, XINV_P0>(sp, (float*)out, g, fx.n, E, tb, ex, nblocks_out, st, used);
  if (mode == XINV_UPDATE)
    return xinv_s<float, XINV_UPDATE>(sp, (float*)out, g, fx.n, E, tb, ex, nblocks_out, st, used);
  if (to_is_double) return xinv_s<double, XINV_PLAIN>(sp, (double*)out, g, fx.n, E, tb, ex, nblocks_out, st, used);
  return xinv_s<float, XINV_PLAIN>(sp, (float*)out, g, fx.n, E, tb, ex, nblocks_out, st, used);
}

}  // namespace pgb
