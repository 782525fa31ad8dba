// Persistent forward x-pass (R2C) of the FP32 transforms.
// (Section 2.1: the x transform of every row of every level; see xpass_common.cuh
// for the persistent staging scheme the kernels share.)
#include "xpass_common.cuh"

namespace pgb {
namespace {

// ---------------------------------------------------------------------------
// forward x-pass
// ---------------------------------------------------------------------------
template <int N, int E, typename TI>
__global__ void __launch_bounds__(xs_threads(E)) k_xfwd_s(const TI* __restrict__ in, float2* __restrict__ spec, Geom g,
                                                      const float2* __restrict__ twx, const float2* __restrict__ twr,
                                                      const int* __restrict__ done, unsigned* __restrict__ err,
                                                      int ns, unsigned stage_bytes) {
  using C = float2;
  using TI2 = typename V2s<TI>::t;
  constexpr int nl = N / E, RB = xs_threads(E) / nl, LS = swizzled_stride(N);
  constexpr bool ALIAS = sizeof(TI) == 8;
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smraw[];
  const XsLayout L = xs_layout(N, RB, ns, stage_bytes, ALIAS);
  C* tw_s = reinterpret_cast<C*>(smraw);
  C* twr_s = tw_s + N;
  C* lines = twr_s + N + 2;
  unsigned char* stg = smraw + L.off_stage;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + L.off_bar);

  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * nl + lane;
  const long long row_begin = (long long)g.lev0 * g.ny, row_end = (long long)g.lev1 * g.ny;
  const long long ngroups = (row_end - row_begin + RB - 1) / RB;
  constexpr unsigned row_bytes = (unsigned)(2 * N * sizeof(TI));
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
  auto issue = [&](long long grp, int s) {
    const long long r0 = row_begin + grp * RB;
    const long long nv = row_end - r0 < RB ? row_end - r0 : RB;
    const unsigned bytes = (unsigned)(nv * row_bytes);
    mbar_arrive_expect_tx(&bar[s], bytes);
    bulk_g2s(stg + (size_t)s * stage_bytes, in + r0 * g.nx, bytes, &bar[s]);
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
  bool ok = true;
  int it = 0;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++it) {
    const int s = it % ns;
    if constexpr (ALIAS) {   // this row's two line buffers are its staged row
      la = reinterpret_cast<C*>(stg + (size_t)s * stage_bytes + (size_t)ty * row_bytes);
      lb = la + LS;
    }
    const bool got = mbar_wait_bounded(&bar[s], (unsigned)((it / ns) & 1), kWaitPolls);
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      rg.consumed[s]++;
      if (it > 0) {   // every thread is past the previous group: refill its stage
        const long long gn = grp - gridDim.x + (long long)ns * gridDim.x;
        if (gn < ngroups) {
          fence_proxy_async_smem();
          issue(gn, (it - 1) % ns);
        }
      }
    }
    const long long row = row_begin + grp * RB + ty;
    const bool valid = row < row_end;
    const TI2* srow = reinterpret_cast<const TI2*>(stg + (size_t)s * stage_bytes + (size_t)ty * row_bytes);
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const TI2 x = srow[st_in_index<N, E, 0>(lane, i)];
      v[i] = make_float2(to_f<TI>(x.x), to_f<TI>(x.y));
    }
    if constexpr (ALIAS) sync();   // the line's threads have read the row before it is overwritten
    const C* fin = st_fft<N, E, -1, false, float>(v, la, lb, sw, lane, tw_s, sync);
    r2c_unpack_store<N, E>(fin, twr_s, spec + (valid ? row : 0) * g.P, lane, valid);
    // the staged row was written through the generic proxy; order that before its refill by TMA
    if constexpr (ALIAS) fence_proxy_async_smem();
  }
  if (tid == 0) {
    if (!ok) atomicOr(err, (unsigned)ERR_WAIT_TIMEOUT);
    ring_drain(rg, bar, ns);
  }
}

template <typename TI>
cudaError_t xfwd_s(const TI* in, float2* spec, const Geom& g, int N, int E, const Tables& tb, const int* done,
                   unsigned* err, cudaStream_t st, bool* used) {
  const int RB = xs_threads(E) / (N / E);
  const unsigned row_bytes = (unsigned)(g.nx * sizeof(TI));
  const XsConfig c = xs_config(N, E, RB * row_bytes, 0, sizeof(TI) == 8);
  if (c.ns == 0 || !aligned16(in) || row_bytes % 16) return cudaSuccess;
  const long long ngroups = ((long long)g.ny * (g.lev1 - g.lev0) + RB - 1) / RB;
  PGB_XS_E_SWITCH(E, PGB_XS_N_SWITCH(N, {
    return xs_launch(k_xfwd_s<NN, EE, TI>, NN / EE, RB, c, ngroups, nullptr, st, used, in, spec, g, tb.twx_f,
                     tb.twr_f, done, err);
  }));
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_xfwd_static(int ti_is_double, const void* in, void* spec, const Geom& g, const FftPlan& fx,
                               const Tables& tb, const int* done, unsigned* err, cudaStream_t st, bool* used) {
  *used = false;
  if (!xpass_static_supported(fx.n)) return cudaSuccess;
  const int E = xs_elems(fx.n, fx.E);
  if (ti_is_double) return xfwd_s<double>((const double*)in, (float2*)spec, g, fx.n, E, tb, done, err, st, used);
  return xfwd_s<float>((const float*)in, (float2*)spec, g, fx.n, E, tb, done, err, st, used);
}

}  // namespace pgb
