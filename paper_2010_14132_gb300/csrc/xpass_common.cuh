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
//
// This header holds what the three kernel files (xpass_fwd.cu, xpass_res.cu,
// xpass_inv.cu) share: the shared-memory layout, the staging-ring bookkeeping,
// the R2C unpacking and the launch configuration.
#pragma once
#include <mutex>
#include <unordered_map>

#include "async_copy.cuh"
#include "fft_static.cuh"
#include "kernels.cuh"
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
                                                 bool valid, int kmax = N) {
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
    if (valid) {   // bins above kmax are not stored
      if (k <= kmax) dst[k] = cadd(ev, wo);
      if (N - k <= kmax) dst[N - k] = cconj(csub(ev, wo));
    }
  }
  if (lane == 0) {   // the self-paired bin k = N/2
    const C A = fin[sw(N / 2)];
    const C B = cconj(A);
    const C ev = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y + B.y));
    const C dd = make_float2(0.5f * (A.x - B.x), 0.5f * (A.y - B.y));
    const C wo = cmul(twr_s[N / 2], make_float2(dd.y, -dd.x));
    if (valid && N / 2 <= kmax) dst[N / 2] = cadd(ev, wo);
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

// Elements per thread of the persistent x-pass for a half length N: kE3 when N has
// a factor 3 (radix 3, then 4), else the plan's 8 or 16.
inline int xs_elems(int N, int plan_e) { return N % 3 == 0 ? kE3 : (plan_e == 16 ? 16 : 8); }

// Dispatch to the compile-time (N, E) instance; shapes the engine cannot take are
// never instantiated (and are not reported supported).
#define PGB_XS_E_SWITCH(E, ...)                                 \
  if ((E) == kE3) {                                             \
    constexpr int EE = kE3;                                     \
    __VA_ARGS__;                                                \
  } else if ((E) == 16) {                                       \
    constexpr int EE = 16;                                      \
    __VA_ARGS__;                                                \
  } else {                                                      \
    constexpr int EE = 8;                                       \
    __VA_ARGS__;                                                \
  }
#define PGB_XS_E8_E3_SWITCH(E, ...)                             \
  if ((E) == kE3) {                                             \
    constexpr int EE = kE3;                                     \
    __VA_ARGS__;                                                \
  } else {                                                      \
    constexpr int EE = 8;                                       \
    __VA_ARGS__;                                                \
  }
#define PGB_XS_N_CASE(V, ...) \
  case V: { constexpr int NN = V; if constexpr (st_valid(NN, EE)) { __VA_ARGS__; } } break;
#define PGB_XS_N_SWITCH(N, ...)                          \
  switch (N) {                                           \
    PGB_XS_N_CASE(32, __VA_ARGS__)                       \
    PGB_XS_N_CASE(64, __VA_ARGS__)                       \
    PGB_XS_N_CASE(96, __VA_ARGS__)                       \
    PGB_XS_N_CASE(128, __VA_ARGS__)                      \
    PGB_XS_N_CASE(192, __VA_ARGS__)                      \
    PGB_XS_N_CASE(256, __VA_ARGS__)                      \
    PGB_XS_N_CASE(384, __VA_ARGS__)                      \
    PGB_XS_N_CASE(512, __VA_ARGS__)                      \
    PGB_XS_N_CASE(768, __VA_ARGS__)                      \
    PGB_XS_N_CASE(1024, __VA_ARGS__)                     \
    PGB_XS_N_CASE(2048, __VA_ARGS__)                     \
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
  *used = true;
  return pdl_launch(kern, dim3((unsigned)grid), dim3(threads_x, RB), c.smem, st, args..., c.ns, c.stage_bytes);
}

}  // namespace
}  // namespace pgb
