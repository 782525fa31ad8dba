// Stockham FFT with the line length known at compile time.
//
// Same transform as fft_engine.cuh (stage s of radix R and span Ns takes inputs
// x[j + r n/R], applies exp(SIGN 2 pi i r (j mod Ns)/(Ns R)), an R-point DFT,
// and writes y[(j - j mod Ns) R + j mod Ns + r Ns]), with every index, span and
// table stride a constant, so the per-element work is the butterfly itself plus
// one shared-memory access.  The values of a thread stay in registers between
// stages; consecutive stages alternate between two shared buffers, so one
// barrier per stage suffices.  The caller supplies the first stage's inputs in
// registers (loaded in whatever way suits it) and receives the result either in
// registers (last stage's layout) or in natural order in a shared buffer.  With 16
// elements per thread the main radix is 16 (one stage fewer than radix 8 for
// most lengths).
#pragma once
#include "fft_engine.cuh"

namespace pgb {

// Radix schedule for n = 2^a 3^b and E elements per thread: radix-3 stages,
// then radix 16 (when E is a multiple of 16), 8 (a multiple of 8) or 4, then a
// final 2, 4 or 8.
constexpr int st_count(int n, int p) {
  int c = 0;
  while (n > 1 && n % p == 0) {
    n /= p;
    ++c;
  }
  return c;
}
constexpr int st_big_log(int e) { return e % 16 == 0 ? 4 : (e % 8 == 0 ? 3 : 2); }   // log2 of the main power-of-two radix
// Elements per thread for lengths with a factor 3: radix 3, then radix 4 (12 values per thread
// keep a line's data in twice as many threads as the radix-8 schedule's 24, for the same shared memory)
constexpr int kE3 = 12;
constexpr int st_nstages(int n, int e) {
  return st_count(n, 3) + st_count(n, 2) / st_big_log(e) + (st_count(n, 2) % st_big_log(e) ? 1 : 0);
}
constexpr int st_radix(int n, int s, int e) {
  const int a = st_count(n, 2), b = st_count(n, 3), L = st_big_log(e);
  if (s < b) return 3;
  if (s - b < a / L) return 1 << L;
  return 1 << (a % L);
}
constexpr int st_span(int n, int s, int e) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= st_radix(n, i, e);
  return ns;
}
// E elements per thread must be a multiple of every radix of the schedule.
constexpr bool st_valid(int n, int e) {
  if (n < 2 || e < 1 || n % e != 0) return false;
  for (int s = 0; s < st_nstages(n, e); ++s)
    if (e % st_radix(n, s, e) != 0) return false;
  return st_span(n, st_nstages(n, e), e) == n;
}

// Element index held in slot i = q R + r of a thread before stage s (inputs x[j + r n/R]).
template <int N, int E, int S> __device__ __forceinline__ int st_in_index(int lane, int i) {
  constexpr int R = st_radix(N, S, E), nl = N / E, m = N / R;
  return lane + nl * (i / R) + (i % R) * m;
}
// Element index held in slot i after the last stage, when it stays in registers.
template <int N, int E> __device__ __forceinline__ int st_out_index(int lane, int i) {
  constexpr int S = st_nstages(N, E) - 1, R = st_radix(N, S, E), nl = N / E, Ns = st_span(N, S, E);
  // last stage: j < Ns, so j mod Ns = j and the outputs are y[j + r Ns]
  return lane + nl * (i / R) + (i % R) * Ns;
}

// Per-line barrier among the nl threads of a line.  Lines of at most 32 threads
// live inside one warp; wider lines use a named barrier per line (ids 1..15).
struct LineSync {
  int id, nthreads;
  __device__ __forceinline__ void operator()() const {
    if (nthreads <= 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
  }
};

// Twiddles in stage order: the stage of span Ns and radix R keeps exp(-2 pi i r k/(Ns R))
// at [(Ns - 1) + (r - 1) Ns + k], r = 1..R-1, k = 0..Ns-1 (N - 1 entries in all, as the
// earlier stages' (R - 1) Ns sum to Ns - 1).  Threads of a line read consecutive k, so the
// reads are free of bank conflicts, unlike the strided r k (N/(Ns R)) reads of one table.
template <int N, int E, typename C>
__device__ __forceinline__ void st_build_twiddles(C* dst, const C* __restrict__ tw_n, int tid, int nthreads) {
  for (int t = tid; t < N - 1; t += nthreads) {
    int Ns = 1, R = st_radix(N, 0, E);
#pragma unroll 1
    for (int s = 0; s < st_nstages(N, E); ++s) {
      R = st_radix(N, s, E);
      if (t < Ns * R - 1) break;
      Ns *= R;
    }
    const int u = t - (Ns - 1), r = u / Ns + 1, k = u - (r - 1) * Ns;
    dst[t] = tw_n[r * k * (N / (Ns * R))];
  }
}

template <int R, int E, int N, int Ns, int SIGN, typename T>
__device__ __forceinline__ void st_butterflies(typename CT<T>::t (&v)[E], int lane,
                                               const typename CT<T>::t* __restrict__ tw) {
  constexpr int B = E / R, nl = N / E;
#pragma unroll
  for (int q = 0; q < B; ++q) {
    if constexpr (Ns > 1) {
      const int k = (lane + nl * q) % Ns;
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = tw_apply<SIGN>(v[q * R + r], tw[(Ns - 1) + (r - 1) * Ns + k]);
    }
    dft_r<R, SIGN, T>(&v[q * R]);
  }
}

template <int R, int E, int N, int Ns, typename C, typename Addr>
__device__ __forceinline__ void st_store(const C (&v)[E], C* buf, Addr addr, int lane) {
  constexpr int B = E / R, nl = N / E;
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int j = lane + nl * q;
    const int k = j % Ns;
    const int d = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[addr(d + r * Ns)] = v[q * R + r];
  }
}

template <int R, int E, int N, typename C, typename Addr>
__device__ __forceinline__ void st_load(C (&v)[E], const C* buf, Addr addr, int lane) {
  constexpr int B = E / R, nl = N / E, m = N / R;
#pragma unroll
  for (int q = 0; q < B; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = buf[addr(lane + nl * q + r * m)];
}

template <int N, int E, int SIGN, bool FINAL_IN_REGS, int S, bool INPLACE, typename T, typename Addr, typename Sync>
__device__ __forceinline__ typename CT<T>::t* st_run_from(typename CT<T>::t (&v)[E], typename CT<T>::t* cur,
                                                          typename CT<T>::t* nxt, Addr addr, int lane,
                                                          const typename CT<T>::t* __restrict__ tw, Sync sync) {
  constexpr int NST = st_nstages(N, E), R = st_radix(N, S, E), Ns = st_span(N, S, E);
  st_butterflies<R, E, N, Ns, SIGN, T>(v, lane, tw);
  if constexpr (S == NST - 1 && FINAL_IN_REGS) {
    return nullptr;
  } else {
    st_store<R, E, N, Ns>(v, cur, addr, lane);
    sync();
    if constexpr (S == NST - 1) {
      return cur;
    } else {
      st_load<st_radix(N, S + 1, E), E, N>(v, cur, addr, lane);
      if constexpr (INPLACE) sync();   // one buffer: every read of this stage precedes the next writes
      return st_run_from<N, E, SIGN, FINAL_IN_REGS, S + 1, INPLACE, T>(v, nxt, cur, addr, lane, tw, sync);
    }
  }
}

// All stages.  v: the first stage's inputs (slot i = element st_in_index<N,E,0>).
// FINAL_IN_REGS: v ends holding element st_out_index<N,E>(lane, i) in slot i and
// nullptr is returned; otherwise the result is stored in natural order in the
// returned buffer (a or b).  tw: the stage-ordered table built by st_build_twiddles.
// The caller makes sure no thread of the line still reads a or b from earlier use.
template <int N, int E, int SIGN, bool FINAL_IN_REGS, typename T, typename Addr, typename Sync,
          bool INPLACE = false>
__device__ __forceinline__ typename CT<T>::t* st_fft(typename CT<T>::t (&v)[E], typename CT<T>::t* a,
                                                     typename CT<T>::t* b, Addr addr, int lane,
                                                     const typename CT<T>::t* __restrict__ tw, Sync sync) {
  static_assert(st_valid(N, E), "unsupported static FFT shape");
  // lane < N/E: lets the compiler split swizzled addresses into a per-thread base plus constants
  __builtin_assume(lane >= 0 && lane < N / E);
  return st_run_from<N, E, SIGN, FINAL_IN_REGS, 0, INPLACE, T>(v, a, b, addr, lane, tw, sync);
}
// In-place variant: one buffer, two barriers per stage.  The caller makes sure every
// thread has read its first-stage inputs from buf before the first store.
template <int N, int E, int SIGN, bool FINAL_IN_REGS, typename T, typename Addr, typename Sync>
__device__ __forceinline__ typename CT<T>::t* st_fft_inplace(typename CT<T>::t (&v)[E], typename CT<T>::t* buf,
                                                             Addr addr, int lane,
                                                             const typename CT<T>::t* __restrict__ tw, Sync sync) {
  return st_fft<N, E, SIGN, FINAL_IN_REGS, T, Addr, Sync, true>(v, buf, buf, addr, lane, tw, sync);
}

}  // namespace pgb
