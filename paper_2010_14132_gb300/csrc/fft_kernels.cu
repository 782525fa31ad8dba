// Transform passes of the direct solve (Section 2.1: each horizontal dimension
// is transformed separately, for all data in that dimension).
//
//  * x-pass forward (R2C): a real row of nx values is packed as nx/2 complex
//    points z_m = x_{2m} + i x_{2m+1}, transformed, and unpacked to the nx/2+1
//    non-redundant coefficients X_k = E_k + exp(-2 pi i k/nx) O_k with
//    E_k = (Z_k + conj Z_{n-k})/2, O_k = -i (Z_k - conj Z_{n-k})/2.
//  * y-pass (C2C, both directions): one level and a tile of TK consecutive kx
//    columns is staged in shared memory as [ny][TK] (row segments of TK complex
//    values are contiguous in HBM), and the TK strided lines are transformed in
//    place.
//  * x-pass inverse (C2R): the mirror of the forward x-pass; the self-conjugate
//    bins kx = 0 and kx = nx/2 contribute their real parts only.  Its epilogue
//    writes the output field and, in the mixed-precision path, performs the
//    refinement update and the norm partial sums.
#include <mutex>
#include <unordered_map>

#include "kernels.cuh"
#include "residual.cuh"

namespace pgb {

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

// ---------------------------------------------------------------------------
// x-pass forward
// ---------------------------------------------------------------------------
// RES = 0: rows of the input array; RES = 1/2: rows of the refinement residual
// (without / with the accumulated correction q), computed as they are loaded.
template <typename TI, typename T, int E, int RES = 0>
__global__ void __launch_bounds__(256) k_xfwd(const TI* __restrict__ in, typename CT<T>::t* __restrict__ spec,
                                               Geom g, FftPlan fx, const typename CT<T>::t* __restrict__ twx,
                                               const typename CT<T>::t* __restrict__ twr, long long nrows,
                                               const int* __restrict__ done, ResidualArgs R) {
  using C = typename CT<T>::t;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int n = fx.n, nl = n / E;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const long long row = (long long)g.lev0 * g.ny + (long long)blockIdx.x * blockDim.y + ty;
  const bool valid = row < nrows;
  C* line = sm + ty * swizzled_stride(n + 1);
  const Swizzled sw{};
  if constexpr (RES == 0) {
    const typename V2<TI>::t* src = reinterpret_cast<const typename V2<TI>::t*>(in + (valid ? row : 0) * g.nx);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int m = lane + nl * q;
      C z = make_c<T>(0, 0);
      if (valid) {
        const typename V2<TI>::t v = __ldcs(&src[m]);   // read once: stream past L2
        z.x = Cvt<TI, T>::f(v.x);
        z.y = Cvt<TI, T>::f(v.y);
      }
      line[sw(m)] = z;
    }
  } else {
    const int jr = valid ? (int)(row % g.ny) : 0, kr = valid ? (int)(row / g.ny) : 0;
    float racc = 0.f, sacc = 0.f;   // sums of r^2 and S^2 over this thread's points
#pragma unroll 4
    for (int q = 0; q < E; ++q) {
      const int m = lane + nl * q;
      C z = make_c<T>(0, 0);
      if (valid) {
        z.x = residual_point<RES == 2>(R, g, 2 * m, jr, kr);
        z.y = residual_point<RES == 2>(R, g, 2 * m + 1, jr, kr);
        const double2 Sv = reinterpret_cast<const double2*>(R.S + row * g.nx)[m];
        racc += (float)z.x * (float)z.x + (float)z.y * (float)z.y;
        sacc += __double2float_rn(Sv.x) * __double2float_rn(Sv.x) + __double2float_rn(Sv.y) * __double2float_rn(Sv.y);
      }
      line[sw(m)] = z;
    }
    // per-block sums of r^2 and S^2 (fixed-order tree over the block's threads)
    __shared__ float rred[2][256];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthreads = blockDim.x * blockDim.y;
    rred[0][tid] = racc;
    rred[1][tid] = sacc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if (tid < h && tid + h < nthreads) {
        rred[0][tid] += rred[0][tid + h];
        rred[1][tid] += rred[1][tid + h];
      }
      __syncthreads();
    }
    if (tid == 0 && R.partials) {
      const long long slot = R.part0 + blockIdx.x;
      R.partials[2 * slot] = (double)rred[0][0];
      R.partials[2 * slot + 1] = (double)rred[1][0];
    }
  }
  __syncthreads();
  stockham_run<E, -1, T>(line, sw, fx, lane, twx, SyncBlock());
  C* dst = spec + (valid ? row : 0) * g.P;
  for (int k = lane; k <= n; k += nl) {
    const C zk = line[sw(k == n ? 0 : k)];
    const C zc = cconj(line[sw(k == 0 ? 0 : n - k)]);
    const C ev = make_c<T>((T)0.5 * (zk.x + zc.x), (T)0.5 * (zk.y + zc.y));
    const C dd = make_c<T>((T)0.5 * (zk.x - zc.x), (T)0.5 * (zk.y - zc.y));
    const C od = make_c<T>(dd.y, -dd.x);  // -i * dd
    if (valid) dst[k] = cadd(ev, cmul(twr[k], od));
  }
}

// ---------------------------------------------------------------------------
// x-pass inverse with epilogues
// ---------------------------------------------------------------------------
template <typename T, typename TO, int MODE, int E>
__global__ void __launch_bounds__(256) k_xinv(const typename CT<T>::t* __restrict__ spec, TO* __restrict__ out,
                                               Geom g, FftPlan fx, const typename CT<T>::t* __restrict__ twx,
                                               const typename CT<T>::t* __restrict__ twr, long long nrows,
                                               XinvExtra ex) {
  using C = typename CT<T>::t;
  if (ex.done && *ex.done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ float red[2][256];
  __shared__ double redd[256];
  C* sm = reinterpret_cast<C*>(smraw);
  const int n = fx.n, nl = n / E;
  const int lane = threadIdx.x, ty = threadIdx.y;
  const long long row = (long long)g.lev0 * g.ny + (long long)blockIdx.x * blockDim.y + ty;
  const bool valid = row < nrows;
  C* line = sm + ty * swizzled_stride(n + 1);
  const Swizzled sw{};
  const C* src = spec + (valid ? row : 0) * g.P;
  {
    // E independent loads per thread (k < n), then the Nyquist entry k = n
    C buf[E];
#pragma unroll
    for (int q = 0; q < E; ++q) buf[q] = valid ? src[lane + nl * q] : make_c<T>(0, 0);
#pragma unroll
    for (int q = 0; q < E; ++q) line[sw(lane + nl * q)] = buf[q];
    if (lane == 0) line[sw(n)] = valid ? src[n] : make_c<T>(0, 0);
  }
  __syncthreads();
  C zr[E];
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int k = lane + nl * q;
    C xk = line[sw(k)];
    C xc = cconj(line[sw(n - k)]);
    if (k == 0) {  // self-conjugate bins: real parts only
      xk.y = 0;
      xc.y = 0;
    }
    const C ev = cadd(xk, xc);
    const C od = cmul(csub(xk, xc), cconj(twr[k]));  // * exp(+2 pi i k/nx)
    zr[q] = make_c<T>(ev.x - od.y, ev.y + od.x);     // ev + i od
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < E; ++q) line[sw(lane + nl * q)] = zr[q];
  __syncthreads();
  stockham_run<E, +1, T>(line, sw, fx, lane, twx, SyncBlock());

  const long long base = (valid ? row : 0) * g.nx;
  float acc0 = 0.f, acc1 = 0.f;
  float sh = 0.f, sl = 0.f;   // double-float running sum of p
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int m = lane + nl * q;
    const C z = line[sw(m)];
    if (!valid) continue;
    if constexpr (MODE == XINV_PLAIN) {
      typename V2<TO>::t v;
      v.x = Cvt<T, TO>::f(z.x);
      v.y = Cvt<T, TO>::f(z.y);
      __stcs(reinterpret_cast<typename V2<TO>::t*>(out + base) + m, v);
    } else if constexpr (MODE == XINV_P0) {
      __stcs(reinterpret_cast<float2*>(ex.p0 + base) + m, make_float2(z.x, z.y));
      acc1 += z.x * z.x + z.y * z.y;
      float e0, e1;
      two_sum(sh, z.x, sh, e0);
      two_sum(sh, z.y, sh, e1);
      sl += e0 + e1;
      if (ex.p_out) __stcs(reinterpret_cast<double2*>(ex.p_out + base) + m, make_double2(f2d_int(z.x), f2d_int(z.y)));
    } else {  // XINV_UPDATE
      const float2 p0 = reinterpret_cast<const float2*>(ex.p0 + base)[m];
      float2 qn = make_float2(z.x, z.y);
      if (ex.q_valid) {
        const float2 qo = reinterpret_cast<const float2*>(ex.q + base)[m];
        qn.x += qo.x;
        qn.y += qo.y;
      }
      if (ex.q_out) __stcs(reinterpret_cast<float2*>(ex.q_out + base) + m, qn);
      float s0, t0, s1, t1;
      two_sum(p0.x, qn.x, s0, t0);
      two_sum(p0.y, qn.y, s1, t1);
      if (ex.p_out)
        __stcs(reinterpret_cast<double2*>(ex.p_out + base) + m, make_double2(ff2d_int(s0, t0), ff2d_int(s1, t1)));
      acc0 += z.x * z.x + z.y * z.y;
      acc1 += s0 * s0 + s1 * s1;
      float e0, e1;
      two_sum(sh, s0, sh, e0);
      two_sum(sh, s1, sh, e1);
      sl += (e0 + e1) + (t0 + t1);
    }
  }
  if constexpr (MODE != XINV_PLAIN) {
    // deterministic block partial sums: fixed-order tree over the block's threads
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;   // <= 256
    red[0][tid] = acc0;
    red[1][tid] = acc1;
    redd[tid] = f2d_int(sh) + f2d_int(sl);
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if (tid < h && tid + h < nthreads) {
        red[0][tid] += red[0][tid + h];
        red[1][tid] += red[1][tid + h];
        redd[tid] += redd[tid + h];
      }
      __syncthreads();
    }
    if (tid == 0) {
      const long long slot = ex.part0 + blockIdx.x;
      ex.partials[3 * slot] = (double)red[0][0];
      ex.partials[3 * slot + 1] = (double)red[1][0];
      ex.partials[3 * slot + 2] = redd[0];
    }
  }
}

// ---------------------------------------------------------------------------
// y-pass, in place on the spectrum
// ---------------------------------------------------------------------------
constexpr int ypass_max_threads(int E) { return E >= 16 ? 512 : 1024; }

template <typename T, int E, int SIGN>
__global__ void __launch_bounds__(ypass_max_threads(E)) k_yfft(typename CT<T>::t* __restrict__ spec, Geom g, FftPlan fy,
                                               const typename CT<T>::t* __restrict__ twy,
                                               const int* __restrict__ done) {
  using C = typename CT<T>::t;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int TK = blockDim.x, l = threadIdx.x, lane = threadIdx.y;
  const int nl = fy.n / E;
  const int kx0 = blockIdx.x * TK;
  C* base = spec + (long long)(g.lev0 + blockIdx.y) * g.plane + kx0;
  const bool vcol = (kx0 + l) < g.nxh;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = lane + nl * q;
    sm[i * TK + l] = vcol ? base[(long long)i * g.P + l] : make_c<T>(0, 0);
  }
  __syncthreads();
  stockham_run<E, SIGN, T>(sm + l, Strided{TK}, fy, lane, twy, SyncBlock());
  if (vcol) {
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane + nl * q;
      base[(long long)i * g.P + l] = sm[i * TK + l];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
bool fft_e_supported(int E) {
  switch (E) {
    case 2: case 3: case 4: case 6: case 8: case 12: case 16: case 24: return true;
    default: return false;
  }
}

#define PGB_E_SWITCH(E, ...)                                      \
  switch (E) {                                                    \
    case 2: { constexpr int EE = 2; __VA_ARGS__; } break;         \
    case 3: { constexpr int EE = 3; __VA_ARGS__; } break;         \
    case 4: { constexpr int EE = 4; __VA_ARGS__; } break;         \
    case 6: { constexpr int EE = 6; __VA_ARGS__; } break;         \
    case 8: { constexpr int EE = 8; __VA_ARGS__; } break;         \
    case 12: { constexpr int EE = 12; __VA_ARGS__; } break;       \
    case 16: { constexpr int EE = 16; __VA_ARGS__; } break;       \
    case 24: { constexpr int EE = 24; __VA_ARGS__; } break;       \
    default: return cudaErrorInvalidValue;                        \
  }

static constexpr int kMaxDynSmem = 227 * 1024;

// Opt a kernel in to `bytes` of dynamic shared memory.  Always done (not only
// above 48 KB): static shared memory counts against the same default limit.
template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> granted;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = granted[reinterpret_cast<const void*>(kernel)];
  if (have >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

// rows per CTA for the x-pass
static int xpass_rows(int n, int E, size_t csize) {
  const int nl = n / E;
  int rb = 256 / nl;
  if (rb < 1) rb = 1;
  while (rb > 1 && (size_t)rb * swizzled_stride(n + 1) * csize > 64 * 1024) rb >>= 1;
  return rb;
}

int xpass_blocks(const Geom& g, const FftPlan& fx, size_t csize) {
  const long long nrows = (long long)g.ny * g.nz;
  const int rb = xpass_rows(fx.n, fx.E, csize);
  long long nb = (nrows + rb - 1) / rb;
  if (csize == sizeof(float2) && xpass_static_supported(fx.n)) {
    const long long rbs = 256 / (fx.n / 8);   // rows per group of the persistent kernels
    const long long ng = (nrows + rbs - 1) / rbs;
    if (ng > nb) nb = ng;
  }
  return (int)nb;
}

template <typename TI, typename T>
static cudaError_t xfwd_t(const TI* in, typename CT<T>::t* spec, const Geom& g, const FftPlan& fx,
                          const typename CT<T>::t* twx, const typename CT<T>::t* twr, const int* done,
                          cudaStream_t st) {
  const long long nrows = (long long)g.ny * g.lev1;   // end row of the chunk
  const int n = fx.n;
  const int rb = xpass_rows(n, fx.E, sizeof(typename CT<T>::t));
  const dim3 block(n / fx.E, rb);
  const long long nb = ((long long)g.ny * (g.lev1 - g.lev0) + rb - 1) / rb;
  const size_t smem = (size_t)rb * swizzled_stride(n + 1) * sizeof(typename CT<T>::t);
  if (smem > kMaxDynSmem || nb > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  PGB_E_SWITCH(fx.E, {
    auto kern = k_xfwd<TI, T, EE>;
    e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nb, block, smem, st>>>(in, spec, g, fx, twx, twr, nrows, done, ResidualArgs{});
  });
  return cudaGetLastError();
}

cudaError_t launch_xfwd_residual(const ResidualArgs& R, void* spec, const Geom& g, const FftPlan& fx,
                                 const Tables& tb, const int* done, int* nblocks_out, cudaStream_t st) {
  using C = float2;
  const long long nrows = (long long)g.ny * g.lev1;   // end row of the chunk
  const int n = fx.n;
  const int rb = xpass_rows(n, fx.E, sizeof(C));
  const dim3 block(n / fx.E, rb);
  const long long nb = ((long long)g.ny * (g.lev1 - g.lev0) + rb - 1) / rb;
  const size_t smem = (size_t)rb * swizzled_stride(n + 1) * sizeof(C);
  if (smem > kMaxDynSmem || nb > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (nblocks_out) *nblocks_out = (int)nb;
  cudaError_t e = cudaSuccess;
  if (R.q) {
    PGB_E_SWITCH(fx.E, {
      auto kern = k_xfwd<float, float, EE, 2>;
      e = allow_smem(kern, smem);
      if (e != cudaSuccess) return e;
      kern<<<(unsigned)nb, block, smem, st>>>(nullptr, (C*)spec, g, fx, tb.twx_f, tb.twr_f, nrows, done, R);
    });
  } else {
    PGB_E_SWITCH(fx.E, {
      auto kern = k_xfwd<float, float, EE, 1>;
      e = allow_smem(kern, smem);
      if (e != cudaSuccess) return e;
      kern<<<(unsigned)nb, block, smem, st>>>(nullptr, (C*)spec, g, fx, tb.twx_f, tb.twr_f, nrows, done, R);
    });
  }
  return cudaGetLastError();
}

cudaError_t launch_xfwd(int ti_is_double, int t_is_double, const void* in, void* spec, const Geom& g,
                        const FftPlan& fx, const Tables& tb, const int* done, cudaStream_t st) {
  if (t_is_double) {
    if (!ti_is_double) return cudaErrorInvalidValue;
    return xfwd_t<double, double>((const double*)in, (double2*)spec, g, fx, tb.twx_d, tb.twr_d, done, st);
  }
  if (ti_is_double)
    return xfwd_t<double, float>((const double*)in, (float2*)spec, g, fx, tb.twx_f, tb.twr_f, done, st);
  return xfwd_t<float, float>((const float*)in, (float2*)spec, g, fx, tb.twx_f, tb.twr_f, done, st);
}

template <typename T, typename TO, int MODE>
static cudaError_t xinv_t(const typename CT<T>::t* spec, TO* out, const Geom& g, const FftPlan& fx,
                          const typename CT<T>::t* twx, const typename CT<T>::t* twr, const XinvExtra& ex,
                          int* nblocks_out, cudaStream_t st) {
  const long long nrows = (long long)g.ny * g.lev1;   // end row of the chunk
  const int n = fx.n;
  const int rb = xpass_rows(n, fx.E, sizeof(typename CT<T>::t));
  const dim3 block(n / fx.E, rb);
  const long long nb = ((long long)g.ny * (g.lev1 - g.lev0) + rb - 1) / rb;
  const size_t smem = (size_t)rb * swizzled_stride(n + 1) * sizeof(typename CT<T>::t);
  if (nblocks_out) *nblocks_out = (int)nb;
  if (smem > kMaxDynSmem || nb > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  PGB_E_SWITCH(fx.E, {
    auto kern = k_xinv<T, TO, MODE, EE>;
    e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nb, block, smem, st>>>(spec, out, g, fx, twx, twr, nrows, ex);
  });
  return cudaGetLastError();
}

cudaError_t launch_xinv(int t_is_double, int to_is_double, int mode, const void* spec, void* out,
                        const Geom& g, const FftPlan& fx, const Tables& tb, const XinvExtra& ex,
                        int* nblocks_out, cudaStream_t st) {
  if (t_is_double) {
    if (!to_is_double || mode != XINV_PLAIN) return cudaErrorInvalidValue;
    return xinv_t<double, double, XINV_PLAIN>((const double2*)spec, (double*)out, g, fx, tb.twx_d, tb.twr_d,
                                              ex, nblocks_out, st);
  }
  if (mode == XINV_P0)
    return xinv_t<float, float, XINV_P0>((const float2*)spec, (float*)out, g, fx, tb.twx_f, tb.twr_f, ex,
                                         nblocks_out, st);
  if (mode == XINV_UPDATE)
    return xinv_t<float, float, XINV_UPDATE>((const float2*)spec, (float*)out, g, fx, tb.twx_f, tb.twr_f, ex,
                                             nblocks_out, st);
  if (to_is_double)
    return xinv_t<float, double, XINV_PLAIN>((const float2*)spec, (double*)out, g, fx, tb.twx_f, tb.twr_f, ex,
                                             nblocks_out, st);
  return xinv_t<float, float, XINV_PLAIN>((const float2*)spec, (float*)out, g, fx, tb.twx_f, tb.twr_f, ex,
                                          nblocks_out, st);
}

// y-pass tile width: requested (or default) clamped by threads and shared memory
static int ypass_tile(int request, int ny, int E, size_t csize) {
  int tk = request > 0 ? request : (csize == 8 ? 8 : 4);
  while (tk > 1 && (long long)tk * (ny / E) > ypass_max_threads(E)) tk >>= 1;
  while (tk > 1 && (size_t)tk * ny * csize > 200 * 1024) tk >>= 1;
  return tk;
}

template <typename T, int SIGN>
static cudaError_t yfft_t(typename CT<T>::t* spec, const Geom& g, const FftPlan& fy,
                          const typename CT<T>::t* twy, int tile, const int* done, cudaStream_t st) {
  const int tk = ypass_tile(tile, fy.n, fy.E, sizeof(typename CT<T>::t));
  const dim3 block(tk, fy.n / fy.E);
  const dim3 grid((g.nxh + tk - 1) / tk, g.lev1 - g.lev0);
  const size_t smem = (size_t)tk * fy.n * sizeof(typename CT<T>::t);
  if (smem > kMaxDynSmem || (int)(block.x * block.y) > ypass_max_threads(fy.E)) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  PGB_E_SWITCH(fy.E, {
    auto kern = k_yfft<T, EE, SIGN>;
    e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, st>>>(spec, g, fy, twy, done);
  });
  return cudaGetLastError();
}

cudaError_t launch_yfft(int t_is_double, int sign, void* spec, const Geom& g, const FftPlan& fy,
                        const Tables& tb, int tile, const int* done, cudaStream_t st) {
  if (t_is_double) {
    if (sign < 0) return yfft_t<double, -1>((double2*)spec, g, fy, tb.twy_d, tile, done, st);
    return yfft_t<double, +1>((double2*)spec, g, fy, tb.twy_d, tile, done, st);
  }
  if (sign < 0) return yfft_t<float, -1>((float2*)spec, g, fy, tb.twy_f, tile, done, st);
  return yfft_t<float, +1>((float2*)spec, g, fy, tb.twy_f, tile, done, st);
}

}  // namespace pgb
