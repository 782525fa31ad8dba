// Self-sorting (Stockham) mixed-radix FFT over lines held in shared memory.
//
// A line of length n = 2^a 3^b is transformed by stages of radix R in {2,3,4,8}.
// Stage s (span Ns = product of the earlier radices) takes butterfly j in
// [0, n/R): inputs x[j + r n/R], twiddles exp(SIGN 2 pi i r (j mod Ns)/(Ns R)),
// an R-point DFT, outputs to y[(j - j mod Ns) R + j mod Ns + r Ns].  After the
// last stage the line is in natural order.  Every thread of a line holds E
// elements (E/R butterflies) in registers between a read phase and a write
// phase, so a single shared buffer serves all stages.
#pragma once
#include "common.cuh"

namespace pgb {

constexpr int kMaxStages = 16;

// Host-built description of one line length.
struct FftPlan {
  int n;                   // line length (complex points)
  int nstages;
  int E;                   // elements per thread (multiple of every radix used)
  int radix[kMaxStages];
};

template <int SIGN, typename C> __device__ __forceinline__ void dft2(C* v) {
  C t = v[0];
  v[0] = cadd(t, v[1]);
  v[1] = csub(t, v[1]);
}

template <int SIGN, typename C, typename T> __device__ __forceinline__ void dft3(C* v) {
  const T h = (T)0.86602540378443864676;   // sqrt(3)/2
  C t = cadd(v[1], v[2]);
  C u = csub(v[1], v[2]);
  C m = {v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y};
  v[0] = cadd(v[0], t);
  C su = cmul_si<SIGN>(cscale(u, h));       // SIGN*i*(sqrt3/2)*u
  v[1] = cadd(m, su);
  v[2] = csub(m, su);
}

template <int SIGN, typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C a = cadd(x0, x2), b = csub(x0, x2);
  C c = cadd(x1, x3), d = cmul_si<SIGN>(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

template <int SIGN, typename C, typename T> __device__ __forceinline__ void dft8(C* v) {
  const T r = (T)0.70710678118654752440;
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<SIGN>(e0, e1, e2, e3);
  dft4<SIGN>(o0, o1, o2, o3);
  // w = exp(SIGN i pi/4) = (1 + SIGN i)/sqrt2; w^2 = SIGN i; w^3 = w * w^2
  C w1o1 = {r * (o1.x - (T)SIGN * o1.y), r * (o1.y + (T)SIGN * o1.x)};
  C w2o2 = cmul_si<SIGN>(o2);
  C t3 = cmul_si<SIGN>(o3);
  C w3o3 = {r * (t3.x - (T)SIGN * t3.y), r * (t3.y + (T)SIGN * t3.x)};
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1o1);
  v[5] = csub(e1, w1o1);
  v[2] = cadd(e2, w2o2);
  v[6] = csub(e2, w2o2);
  v[3] = cadd(e3, w3o3);
  v[7] = csub(e3, w3o3);
}

// multiply by W^m = exp(SIGN 2 pi i m/16) for the inner twiddles of dft16
template <int SIGN, int M, typename C, typename T> __device__ __forceinline__ C w16(C a) {
  constexpr int m = M % 16;
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;   // cos, sin (pi/8)
  const T h = (T)0.70710678118654752440;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 4) {
    return cmul_si<SIGN>(a);
  } else if constexpr (m == 8) {
    return C{-a.x, -a.y};
  } else if constexpr (m == 2 || m == 6) {
    // (cos + SIGN i sin)(pi m/8) with cos = +-h, sin = h
    const T cs = (m == 2) ? h : -h;
    const T sn = (T)SIGN * h;
    return C{cs * a.x - sn * a.y, cs * a.y + sn * a.x};
  } else {
    // m in {1, 3, 9}: cos/sin of pi m/8 from c1, s1
    const T cs = (m == 1) ? c1 : (m == 3 ? s1 : -c1);
    const T sn = (T)SIGN * ((m == 1) ? s1 : (m == 3 ? c1 : -s1));
    return C{cs * a.x - sn * a.y, cs * a.y + sn * a.x};
  }
}

// 16-point DFT as 4 x 4: DFT4 over n1 of x[4 n1 + n2], inner twiddles
// W^(n2 k1), DFT4 over n2; X[k1 + 4 k2] then sits in slot 4 k1 + k2 and is
// moved to natural order.
template <int SIGN, typename C, typename T> __device__ __forceinline__ void dft16(C* v) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<SIGN>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // slot 4 k1 + n2 holds Y[n2][k1]
  v[5] = w16<SIGN, 1, C, T>(v[5]);
  v[6] = w16<SIGN, 2, C, T>(v[6]);
  v[7] = w16<SIGN, 3, C, T>(v[7]);
  v[9] = w16<SIGN, 2, C, T>(v[9]);
  v[10] = w16<SIGN, 4, C, T>(v[10]);
  v[11] = w16<SIGN, 6, C, T>(v[11]);
  v[13] = w16<SIGN, 3, C, T>(v[13]);
  v[14] = w16<SIGN, 6, C, T>(v[14]);
  v[15] = w16<SIGN, 9, C, T>(v[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // slot 4 k1 + k2 holds X[k1 + 4 k2]: transpose the 4 x 4 block
  C t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <int R, int SIGN, typename T> __device__ __forceinline__ void dft_r(typename CT<T>::t* v) {
  if constexpr (R == 2) dft2<SIGN>(v);
  else if constexpr (R == 3) dft3<SIGN, typename CT<T>::t, T>(v);
  else if constexpr (R == 4) dft4<SIGN>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<SIGN, typename CT<T>::t, T>(v);
  else dft16<SIGN, typename CT<T>::t, T>(v);
}

// Shared-memory address of element idx of a line.
//  Strided: line-interleaved tiles (element idx of line l at idx*es + l).
//  Swizzled: contiguous lines; the low 4 bits of the complex index are XORed with
//  the next 4, a bijection within each 16-element block that spreads the
//  power-of-two strides of the early Stockham writes (stride R) over all banks.
struct Strided {
  int es;
  __device__ __forceinline__ int operator()(int idx) const { return idx * es; }
};
struct Swizzled {
  __device__ __forceinline__ int operator()(int idx) const { return idx ^ ((idx >> 4) & 15); }
};
// line length padded so that the swizzle stays inside the line
__host__ __device__ constexpr int swizzled_stride(int len) { return (len + 15) / 16 * 16; }

// Synchronisation of the threads that share one line.
struct SyncBlock { __device__ __forceinline__ void operator()() const { __syncthreads(); } };
struct SyncWarp { __device__ __forceinline__ void operator()() const { __syncwarp(); } };

// One stage on one line: element idx of the line lives at line[addr(idx)].
// lane in [0, nl) indexes the threads of the line; nl * E == n.
template <int R, int E, int SIGN, typename T, typename Sync, typename Addr>
__device__ __forceinline__ void stockham_stage(typename CT<T>::t* line, Addr addr, int n, int Ns, int lane,
                                               int nl, const typename CT<T>::t* __restrict__ tw,
                                               Sync sync) {
  using C = typename CT<T>::t;
  constexpr int B = E / R;
  const int m = n / R;
  C v[E];
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int j = lane + nl * q;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = line[addr(j + r * m)];
  }
  sync();
  const int stride = n / (Ns * R);
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int j = lane + nl * q;
    const int k = j % Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = tw_apply<SIGN>(v[q * R + r], tw[r * k * stride]);
    }
    dft_r<R, SIGN, T>(&v[q * R]);
    const int d = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) line[addr(d + r * Ns)] = v[q * R + r];
  }
  sync();
}

// All stages of a plan.  E is the compile-time elements-per-thread count the
// plan was built for; radices that do not divide E never occur in such a plan.
template <int E, int SIGN, typename T, typename Sync, typename Addr>
__device__ __forceinline__ void stockham_run(typename CT<T>::t* line, Addr addr, const FftPlan& P, int lane,
                                             const typename CT<T>::t* __restrict__ tw, Sync sync) {
  const int nl = P.n / E;
  int Ns = 1;
  for (int s = 0; s < P.nstages; ++s) {
    const int R = P.radix[s];
    if constexpr (E % 8 == 0) {
      if (R == 8) { stockham_stage<8, E, SIGN, T>(line, addr, P.n, Ns, lane, nl, tw, sync); Ns *= 8; continue; }
    }
    if constexpr (E % 4 == 0) {
      if (R == 4) { stockham_stage<4, E, SIGN, T>(line, addr, P.n, Ns, lane, nl, tw, sync); Ns *= 4; continue; }
    }
    if constexpr (E % 3 == 0) {
      if (R == 3) { stockham_stage<3, E, SIGN, T>(line, addr, P.n, Ns, lane, nl, tw, sync); Ns *= 3; continue; }
    }
    if constexpr (E % 2 == 0) {
      if (R == 2) { stockham_stage<2, E, SIGN, T>(line, addr, P.n, Ns, lane, nl, tw, sync); Ns *= 2; continue; }
    }
  }
}

}  // namespace pgb
