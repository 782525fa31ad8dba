// Persistent x-pass kernels for FP32 transforms of power-of-two half lengths
// (Section 2.1: the x transform of every row of every level).
//
// One CTA per SM slot walks groups of RB consecutive rows.  Each group's input
// rows (the field rows for the forward pass, the spectrum rows for the inverse)
// are brought into a ring of shared staging buffers by 1-D bulk copies (TMA)
// completing on an mbarrier, so the loads of the next groups are in flight
// while the current group is transformed.  The FFT runs with the line length
// fixed at compile time (fft_static.cuh) on twiddle tables held in shared memory.
//
//  * forward (R2C): rows packed as n/2 complex points z_m = x_2m + i x_2m+1; after
//    the transform each thread unpacks the pair of bins (k, n/2 - k):
//      X_k = E_k + w^k O_k,   X_{n/2-k} = conj(E_k - w^k O_k),
//    with E_k = (Z_k + conj Z_{n/2-k})/2, O_k = -i (Z_k - conj Z_{n/2-k})/2 and
//    w = exp(-2 pi i/n) (the second form follows from w^{n/2-k} = -conj(w^k)).
//  * inverse (C2R): each first-stage input z_m is formed directly from the staged
//    bins X_m and X_{n/2-m} (self-conjugate bins keep their real parts), the
//    transform's last stage stays in registers, and the epilogue writes the output
//    (and, in the mixed-precision path, the refinement update and norm partial
//    sums) straight from registers.
#include <mutex>
#include <unordered_map>

#include "async_copy.cuh"
#include "fft_static.cuh"
#include "kernels.cuh"
#include "residual.cuh"
#include "residual2.cuh"

namespace pgb {

namespace {

// CTA size: 256 threads with 8 elements per thread, 128 with 16 (one warp per
// 512-point line); with 16 elements the FFT runs radix-16 stages.
__host__ __device__ constexpr int xs_threads(int E) { return E >= 16 ? 128 : 256; }
constexpr int kXsMaxStages = 4;

template <typename T> struct V2s;
template <> struct V2s<float> { using t = float2; };
template <> struct V2s<double> { using t = double2; };

template <typename TI> __device__ __forceinline__ float to_f(TI x);
template <> __device__ __forceinline__ float to_f<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f<double>(double x) { return d2f_int(x); }

// Shared layout: twiddles (n/2), unpack twiddles (n/2 + 2), RB rows x 2 line
// buffers (none when the lines alias the staged rows), then the staging ring
// (128-byte aligned) and its mbarriers.  A staged row of nx doubles holds
// exactly the two n/2-point line buffers of its own row, so kernels that stage
// double rows run the transform inside the consumed row.
struct XsLayout {
  size_t off_stage, off_bar, total;
};
__host__ __device__ constexpr size_t xs_align(size_t x, size_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline XsLayout xs_layout(int N, int RB, int ns, unsigned stage_bytes, bool alias) {
  XsLayout L{};
  size_t off = (size_t)N * 8 + (size_t)(N + 2) * 8 + (alias ? 0 : (size_t)RB * 2 * swizzled_stride(N) * 8);
  L.off_stage = xs_align(off, 128);
  L.off_bar = xs_align(L.off_stage + (size_t)ns * stage_bytes, 8);
  L.total = L.off_bar + (size_t)ns * 8;
  return L;
}

// Bounded-wait bookkeeping of the staging ring, kept by the issuing thread.
struct Ring {
  int issued[kXsMaxStages];
  int consumed[kXsMaxStages];
};

__device__ __forceinline__ void ring_drain(Ring& rg, uint64_t* bar, int ns) {
  // let every copy still in flight land before the CTA's shared memory is released
  for (int s = 0; s < ns; ++s)
    for (int c = rg.consumed[s]; c < rg.issued[s]; ++c) mbar_wait_bounded(&bar[s], (unsigned)(c & 1), kWaitPolls);
}

// R2C unpacking of a transformed line (natural order in fin) and store of the
// bins 0..N to dst: each thread takes the bin pairs (k, N - k), k = lane + nl q.
template <int N, int E>
__device__ __forceinline__ void r2c_unpack_store(const float2* fin, const float2* twr_s, float2* dst, int lane,
                                                 bool valid) {
  using C = float2;
  constexpr int nl = N / E;
  const Swizzled sw{};
#pragma unroll
  for (int q = 0; q < E / 2; ++q) {
    const int k = lane + nl * q;   // k < N/2
    const C A = fin[sw(k)];
    const C B = cconj(fin[sw(k == 0 ? 0 : N - k)]);
    const C ev = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y + B.y));
    const C dd = make_float2(0.5f * (A.x - B.x), 0.5f * (A.y - B.y));
    const C wo = cmul(twr_s[k], make_float2(dd.y, -dd.x));   // w^k * (-i dd)
    if (valid) {
      dst[k] = cadd(ev, wo);
      dst[N - k] = cconj(csub(ev, wo));
    }
  }
  if (lane == 0) {   // the self-paired bin k = N/2
    const C A = fin[sw(N / 2)];
    const C B = cconj(A);
    const C ev = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y + B.y));
    const C dd = make_float2(0.5f * (A.x - B.x), 0.5f * (A.y - B.y));
    const C wo = cmul(twr_s[N / 2], make_float2(dd.y, -dd.x));
    if (valid) dst[N / 2] = cadd(ev, wo);
  }
}

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
  if (done && *done) return;
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

// ---------------------------------------------------------------------------
// forward x-pass of a refinement sweep: the rows transformed are the residual
// r = S - mu_W - L (p0 + q), formed as the group is read.  The group's rows of S,
// p0 (and q) are staged; the x-neighbours come from the staged rows, the y- and
// z-neighbour rows are read through L1/L2 (the neighbouring groups stage them).
// ---------------------------------------------------------------------------
template <int N, int E, bool HAS_Q, bool STAGE_P>
__global__ void __launch_bounds__(xs_threads(E), E >= 16 ? 4 : 3) k_xres_s(ResidualArgs R, float2* __restrict__ spec, Geom g,
                                                      const float2* __restrict__ twx, const float2* __restrict__ twr,
                                                      const int* __restrict__ done, unsigned* __restrict__ err,
                                                      int ns, unsigned stage_bytes) {
  using C = float2;
  constexpr int nl = N / E, RB = xs_threads(E) / nl, LS = swizzled_stride(N), NX = 2 * N;
  if (done && *done) return;
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
  auto issue = [&](long long grp, int s) {
    const long long r0 = row_begin + grp * RB;
    const unsigned nv = (unsigned)(row_end - r0 < RB ? row_end - r0 : RB);
    unsigned char* d = stg + (size_t)s * stage_bytes;
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
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int e = st_in_index<N, E, 0>(lane, i);
      const float2 pc = reinterpret_cast<const float2*>(prow)[e];
      const float pw = prow[e == 0 ? NX - 1 : 2 * e - 1];
      const float pe = prow[e == N - 1 ? 0 : 2 * e + 2];
      const float2 pn = p0n[e], ps = p0s[e];
      const float2 pd = has_dn ? p0d[e] : pc, pu = has_up ? p0u[e] : pc;
      float2 qc = make_float2(0.f, 0.f), qn = qc, qs = qc, qd = qc, qu = qc;
      float qw = 0.f, qe = 0.f;
      if constexpr (HAS_Q) {
        qc = reinterpret_cast<const float2*>(qrow)[e];
        qw = qrow[e == 0 ? NX - 1 : 2 * e - 1];
        qe = qrow[e == N - 1 ? 0 : 2 * e + 2];
        qn = reinterpret_cast<const float2*>(R.q + rn * NX)[e];
        qs = reinterpret_cast<const float2*>(R.q + rs * NX)[e];
        qd = has_dn ? reinterpret_cast<const float2*>(R.q + (rc - g.ny) * NX)[e] : qc;
        qu = has_up ? reinterpret_cast<const float2*>(R.q + (rc + g.ny) * NX)[e] : qc;
      }
      const double2 S = Srow[e];
      float2 Sh, Sl;
      d2ff_trunc(S.x, Sh.x, Sl.x);
      d2ff_trunc(S.y, Sh.y, Sl.y);
      // the pair's east neighbours are (pc.y, pe), its west neighbours (pw, pc.x)
      v[i] = residual_value2<HAS_Q>(pc, make_float2(pc.y, pe), make_float2(pw, pc.x), pn, ps, pd, pu, qc,
                                    make_float2(qc.y, qe), make_float2(qw, qc.x), qn, qs, qd, qu, Sh, Sl, K);
    }
    sync();   // the line's threads have read the S row before it is overwritten
    const C* fin = st_fft<N, E, -1, false, float>(v, la, lb, sw, lane, tw_s, sync);
    r2c_unpack_store<N, E>(fin, twr_s, spec + (valid ? row : 0) * g.P, lane, valid);
    fence_proxy_async_smem();   // generic writes to the staged row come before its refill by TMA
  }
  if (tid == 0) {
    if (!ok) atomicOr(err, (unsigned)ERR_WAIT_TIMEOUT);
    ring_drain(rg, bar, ns);
  }
}

// ---------------------------------------------------------------------------
// inverse x-pass with the solver's epilogues
// ---------------------------------------------------------------------------
template <int N, int E, typename TO, int MODE>
__global__ void __launch_bounds__(xs_threads(E)) k_xinv_s(const float2* __restrict__ spec, TO* __restrict__ out, Geom g,
                                                      const float2* __restrict__ twx, const float2* __restrict__ twr,
                                                      XinvExtra ex, int ns, unsigned stage_bytes) {
  using C = float2;
  constexpr int nl = N / E, RB = xs_threads(E) / nl, LS = swizzled_stride(N);
  if (ex.done && *ex.done) return;
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
        } else {   // XINV_UPDATE: q += delta, p = p0 + q as a double
          const float2 qn = add2(z, qv[i]);
          __stcs(reinterpret_cast<float2*>(ex.q + base) + m, qn);
          float2 sp, tp;
          two_sum2(p0v[i], qn, sp, tp);
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
    static_assert((size_t)TH * 24 <= (size_t)RB * 2 * LS * sizeof(C), "reduction does not fit the line buffers");
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
      double* sums = redd;   // [3][TH] in the line buffers
      double a0 = 0, a1 = 0, a2 = 0;
      for (int i = tid; i < (int)gridDim.x; i += TH) {
        const long long slot = ex.part0 + i;
        a0 += __ldcg(&ex.partials[3 * slot]);
        a1 += __ldcg(&ex.partials[3 * slot + 1]);
        a2 += __ldcg(&ex.partials[3 * slot + 2]);
      }
      __syncthreads();
      sums[tid] = a0;
      sums[TH + tid] = a1;
      sums[2 * TH + tid] = a2;
      __syncthreads();
      for (int h = TH / 2; h > 0; h >>= 1) {
        if (tid < h) {
          sums[tid] += sums[tid + h];
          sums[TH + tid] += sums[TH + tid + h];
          sums[2 * TH + tid] += sums[2 * TH + tid + h];
        }
        __syncthreads();
      }
      if (tid == 0) {
        ex.ctl_stats->control_ticket = 0u;   // ready for the next pass
        control_decide(ex.ctl_stats, sums[0], sums[TH], sums[2 * TH], ex.ctl_pass, ex.ctl_max_sweeps, ex.ctl_tol,
                       ex.ctl_npoints);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// launch configuration
// ---------------------------------------------------------------------------

int sm_count() {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 0;
  cache[dev] = n;
  return n;
}

struct XsConfig {
  int ns = 0;
  unsigned stage_bytes = 0;
  size_t smem = 0;
};

// Staging depth and CTAs per SM: the most CTAs per SM (up to three) whose
// shared memory still allows two stages, then the deepest ring (up to four
// stages) at that CTA count.
XsConfig xs_config(int N, int E, unsigned stage_bytes, size_t static_smem, bool alias) {
  const int RB = xs_threads(E) / (N / E);
  constexpr size_t kSmPerSm = 228 * 1024, kReserved = 1024, kMaxPerCta = 227 * 1024;
  XsConfig c{};
  c.stage_bytes = stage_bytes;
  for (int ctas = 3; ctas >= 1 && c.ns == 0; --ctas) {
    size_t budget = kSmPerSm / ctas - kReserved - static_smem;
    if (budget > kMaxPerCta - static_smem) budget = kMaxPerCta - static_smem;
    for (int ns = kXsMaxStages; ns >= 2; --ns)
      if (xs_layout(N, RB, ns, stage_bytes, alias).total <= budget) {
        c.ns = ns;
        break;
      }
  }
  if (c.ns) c.smem = xs_layout(N, RB, c.ns, stage_bytes, alias).total;
  return c;
}

template <typename K> cudaError_t prepare(K kernel, int threads, size_t smem, int& grid_cap) {
  static std::mutex mu;
  static std::unordered_map<const void*, std::pair<size_t, int>> done;   // smem granted, CTAs per SM
  std::lock_guard<std::mutex> lock(mu);
  auto& ent = done[reinterpret_cast<const void*>(kernel)];
  if (ent.first < smem || ent.second == 0) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    ent = {smem, per_sm};
  }
  grid_cap = ent.second * sm_count();
  return cudaSuccess;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

#define PGB_XS_E_SWITCH(E, ...)                                 \
  if ((E) == 16) {                                              \
    constexpr int EE = 16;                                      \
    __VA_ARGS__;                                                \
  } else {                                                      \
    constexpr int EE = 8;                                       \
    __VA_ARGS__;                                                \
  }
#define PGB_XS_N_SWITCH(N, ...)                          \
  switch (N) {                                           \
    case 64: { constexpr int NN = 64; __VA_ARGS__; } break;     \
    case 128: { constexpr int NN = 128; __VA_ARGS__; } break;   \
    case 256: { constexpr int NN = 256; __VA_ARGS__; } break;   \
    case 512: { constexpr int NN = 512; __VA_ARGS__; } break;   \
    case 1024: { constexpr int NN = 1024; __VA_ARGS__; } break; \
    case 2048: { constexpr int NN = 2048; __VA_ARGS__; } break; \
    default: return cudaSuccess;                         \
  }

// Launch one persistent x-pass kernel: grid = min(groups, resident CTAs).
template <typename K, typename... Args>
cudaError_t xs_launch(K kern, int threads_x, int RB, const XsConfig& c, long long ngroups, int* nblocks_out,
                      cudaStream_t st, bool* used, Args... args) {
  int cap = 0;
  cudaError_t e = prepare(kern, threads_x * RB, c.smem, cap);
  if (e != cudaSuccess) return e;
  if (cap <= 0) return cudaSuccess;
  const long long grid = ngroups < cap ? ngroups : cap;
  if (grid <= 0) return cudaSuccess;
  if (nblocks_out) *nblocks_out = (int)grid;
  kern<<<(unsigned)grid, dim3(threads_x, RB), c.smem, st>>>(args..., c.ns, c.stage_bytes);
  *used = true;
  return cudaGetLastError();
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

template <bool HAS_Q>
cudaError_t xres_s(const ResidualArgs& R, float2* spec, const Geom& g, int N, int E, const Tables& tb,
                   const int* done, unsigned* err, cudaStream_t st, bool* used) {
  const int RB = xs_threads(E) / (N / E);
  // stage S, p0 (and q) rows while three CTAs per SM still fit, else S rows only
  const unsigned row_bytes_all = (unsigned)(g.nx * (8 + 4 + (HAS_Q ? 4 : 0)));
  const unsigned row_bytes_s = (unsigned)(g.nx * 8);
  const XsConfig c_all = xs_config(N, E, RB * row_bytes_all, 0, true);
  const bool stage_p = c_all.ns > 0 && c_all.smem <= 75 * 1024 * (size_t)xs_threads(E) / 256;
  const XsConfig c = stage_p ? c_all : xs_config(N, E, RB * row_bytes_s, 0, true);
  if (c.ns == 0 || !aligned16(R.S) || !aligned16(R.p0) || (HAS_Q && !aligned16(R.q)) || (g.nx * 4) % 16)
    return cudaSuccess;
  const long long ngroups = ((long long)g.ny * (g.lev1 - g.lev0) + RB - 1) / RB;
  if (stage_p) {
    PGB_XS_E_SWITCH(E, PGB_XS_N_SWITCH(N, {
      return xs_launch(k_xres_s<NN, EE, HAS_Q, true>, NN / EE, RB, c, ngroups, nullptr, st, used, R, spec, g,
                       tb.twx_f, tb.twr_f, done, err);
    }));
  } else {
    PGB_XS_E_SWITCH(E, PGB_XS_N_SWITCH(N, {
      return xs_launch(k_xres_s<NN, EE, HAS_Q, false>, NN / EE, RB, c, ngroups, nullptr, st, used, R, spec, g,
                       tb.twx_f, tb.twr_f, done, err);
    }));
  }
  return cudaSuccess;
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
    case 64: case 128: case 256: case 512: case 1024: case 2048: return true;
    default: return false;
  }
}

cudaError_t launch_xfwd_static(int ti_is_double, const void* in, void* spec, const Geom& g, const FftPlan& fx,
                               const Tables& tb, const int* done, unsigned* err, cudaStream_t st, bool* used) {
  *used = false;
  if (!xpass_static_supported(fx.n)) return cudaSuccess;
  const int E = fx.E == 16 ? 16 : 8;
  if (ti_is_double) return xfwd_s<double>((const double*)in, (float2*)spec, g, fx.n, E, tb, done, err, st, used);
  return xfwd_s<float>((const float*)in, (float2*)spec, g, fx.n, E, tb, done, err, st, used);
}

cudaError_t launch_xres_static(const ResidualArgs& R, void* spec, const Geom& g, const FftPlan& fx, const Tables& tb,
                               const int* done, unsigned* err, cudaStream_t st, bool* used) {
  *used = false;
  if (!xpass_static_supported(fx.n)) return cudaSuccess;
  const int E = fx.E == 16 ? 16 : 8;
  if (R.q) return xres_s<true>(R, (float2*)spec, g, fx.n, E, tb, done, err, st, used);
  return xres_s<false>(R, (float2*)spec, g, fx.n, E, tb, done, err, st, used);
}

cudaError_t launch_xinv_static(int to_is_double, int mode, const void* spec, void* out, const Geom& g,
                               const FftPlan& fx, const Tables& tb, const XinvExtra& ex, int* nblocks_out,
                               cudaStream_t st, bool* used) {
  *used = false;
  if (!xpass_static_supported(fx.n)) return cudaSuccess;
  const float2* sp = (const float2*)spec;
  const int E = fx.E == 16 ? 16 : 8;
  if (mode == XINV_P0) return xinv_s<float, XINV_P0>(sp, (float*)out, g, fx.n, E, tb, ex, nblocks_out, st, used);
  if (mode == XINV_UPDATE)
    return xinv_s<float, XINV_UPDATE>(sp, (float*)out, g, fx.n, E, tb, ex, nblocks_out, st, used);
  if (to_is_double) return xinv_s<double, XINV_PLAIN>(sp, (double*)out, g, fx.n, E, tb, ex, nblocks_out, st, used);
  return xinv_s<float, XINV_PLAIN>(sp, (float*)out, g, fx.n, E, tb, ex, nblocks_out, st, used);
}

}  // namespace pgb
