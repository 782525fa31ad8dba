// Persistent FP32 y-pass for power-of-two ny in [64, 2048] (Section 2.1: the
// transform along y of every kx column of every level).
//
// A tile is one level and TK consecutive kx columns: ny rows of TK complex
// values, brought into shared memory by 2-D TMA boxes (columns past nx/2 read
// as zeros).  A CTA walks tiles with a ring of two tile buffers, so the next
// tile loads while the current one is transformed.  The transform is the
// compile-time Stockham engine (fft_static.cuh) on the TK interleaved columns:
// its first stage reads the TMA tile, the stages alternate between a scratch
// tile and the (by then consumed) input tile in a swizzled layout, and the last
// stage's outputs go from registers straight to global memory (each warp writes
// row segments of TK contiguous values).
#include <mutex>
#include <unordered_map>

#include "async_copy.cuh"
#include "fft_static.cuh"
#include "kernels.cuh"

namespace pgb {

namespace {

// Column-interleaved tile addressing with the complex index swizzled inside
// blocks of 16 (spreads the stride-R first-stage writes over the banks).
struct SwStrided {
  int es;
  __device__ __forceinline__ int operator()(int idx) const { return (idx ^ ((idx >> 4) & 15)) * es; }
};
struct Plain {
  int es;
  __device__ __forceinline__ int operator()(int idx) const { return idx * es; }
};

size_t ys_tile_bytes(int N, int TK) { return ((size_t)N * TK * sizeof(float2) + 127) / 128 * 128; }
size_t ys_smem(int N, int TK, bool inplace) {
  return (inplace ? 2 : 3) * ys_tile_bytes(N, TK) + (size_t)N * sizeof(float2) + 64;
}

constexpr int ys_max_threads(int E) { return E >= 16 || E % 3 == 0 ? 512 : 1024; }
// the single-buffered kernel runs two CTAs per SM: 256 threads for the 12-element lengths keeps
// their registers (128) free of spills
constexpr int ys1_max_threads(int E) { return E % 3 == 0 ? 256 : ys_max_threads(E); }

template <int N, int E, int SIGN, bool INPLACE>
__global__ void __launch_bounds__(ys_max_threads(E)) k_ys(const __grid_constant__ CUtensorMap tm, Geom g,
                                            const float2* __restrict__ twy, float2* __restrict__ spec, int box_rows,
                                            int tiles_per_level, int ntiles, const int* __restrict__ done,
                                            unsigned* __restrict__ err) {
  using C = float2;
  constexpr int nl = N / E;
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smraw[];
  const int TK = blockDim.x, l = threadIdx.x, lane = threadIdx.y;
  const int tid = lane * TK + l, nthreads = TK * nl;
  const size_t tb = ((size_t)N * TK * sizeof(C) + 127) / 128 * 128;
  constexpr int NT = INPLACE ? 2 : 3;   // tile buffers: the TMA ring (+ a scratch tile)
  C* ring[2] = {reinterpret_cast<C*>(smraw), reinterpret_cast<C*>(smraw + tb)};
  C* scratch = reinterpret_cast<C*>(smraw + 2 * tb);
  C* tw_s = reinterpret_cast<C*>(smraw + NT * tb);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + NT * tb + (size_t)N * sizeof(C));
  const unsigned tile_bytes = (unsigned)((size_t)N * TK * sizeof(C));
  st_build_twiddles<N, E>(tw_s, twy, tid, nthreads);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  pdl_wait();   // the previous kernels of the stream are complete
  if (done && *done) return;
  int issued[2] = {0, 0}, consumed[2] = {0, 0};
  auto issue = [&](int t, int b) {
    const int level = t / tiles_per_level, kx0 = (t - level * tiles_per_level) * TK;
    mbar_arrive_expect_tx(&bar[b], tile_bytes);
    for (int r0 = 0; r0 < N; r0 += box_rows) tma_load_2d(ring[b] + (size_t)r0 * TK, &tm, kx0, level * N + r0, &bar[b]);
    issued[b]++;
  };
  const int t0 = g.lev0 * tiles_per_level + blockIdx.x;
  if (tid == 0) {
    if (t0 < ntiles) issue(t0, 0);
    if (t0 + (int)gridDim.x < ntiles) issue(t0 + gridDim.x, 1);
  }
  const SwStrided sw{TK};
  bool ok = true;
  int it = 0;
  for (int t = t0; t < ntiles; t += gridDim.x, ++it) {
    const int b = it & 1;
    const bool got = mbar_wait_bounded(&bar[b], (unsigned)((it >> 1) & 1), kWaitPolls);
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      consumed[b]++;
      // every thread is past the previous tile: its buffer takes the tile after this one
      const int tn = t + gridDim.x;
      if (it > 0 && tn < ntiles) {
        fence_proxy_async_smem();
        issue(tn, b ^ 1);
      }
    }
    C* in = ring[b];
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = in[Plain{TK}(st_in_index<N, E, 0>(lane, i)) + l];
    if constexpr (INPLACE) {
      __syncthreads();   // every thread has its inputs before the tile is overwritten
      st_fft_inplace<N, E, SIGN, true, float>(v, in + l, sw, lane, tw_s, SyncBlock());
    } else {
      st_fft<N, E, SIGN, true, float>(v, scratch + l, in + l, sw, lane, tw_s, SyncBlock());
    }
    (void)scratch;
    const int level = t / tiles_per_level, kx = (t - level * tiles_per_level) * TK + l;
    if (kx < g.nxh) {
      C* col = spec + (long long)level * g.plane + kx;
#pragma unroll
      for (int i = 0; i < E; ++i) col[(long long)st_out_index<N, E>(lane, i) * g.P] = v[i];
    }
    fence_proxy_async_smem();   // generic writes to the ring buffer come before its refill by TMA
  }
  if (tid == 0) {
    if (!ok) atomicOr(err, (unsigned)ERR_WAIT_TIMEOUT);
    for (int b = 0; b < 2; ++b)
      for (int c = consumed[b]; c < issued[b]; ++c) mbar_wait_bounded(&bar[b], (unsigned)(c & 1), kWaitPolls);
  }
}


// Single-buffered variant: one tile per CTA, transformed in place, two CTAs per
// SM (registers capped for it), so one CTA's load overlaps the other's transform.
// The next tile's load is issued as soon as the transform has finished reading the
// tile (its outputs are in registers), so it also overlaps this tile's stores.
template <int N, int E, int SIGN>
__global__ void __launch_bounds__(ys1_max_threads(E), 2) k_ys1(const __grid_constant__ CUtensorMap tm, Geom g,
                                                             const float2* __restrict__ twy,
                                                             float2* __restrict__ spec, int box_rows,
                                                             int tiles_per_level, int ntiles,
                                                             const int* __restrict__ done, unsigned* __restrict__ err) {
  using C = float2;
  constexpr int nl = N / E;
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smraw[];
  const int TK = blockDim.x, l = threadIdx.x, lane = threadIdx.y;
  const int tid = lane * TK + l, nthreads = TK * nl;
  const size_t tb = ((size_t)N * TK * sizeof(C) + 127) / 128 * 128;
  C* tile = reinterpret_cast<C*>(smraw);
  C* tw_s = reinterpret_cast<C*>(smraw + tb);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + tb + (size_t)N * sizeof(C));
  const unsigned tile_bytes = (unsigned)((size_t)N * TK * sizeof(C));
  st_build_twiddles<N, E>(tw_s, twy, tid, nthreads);
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  pdl_wait();   // the previous kernels of the stream are complete
  if (done && *done) return;
  const SwStrided sw{TK};
  int it = 0, pending = 0;
  bool ok = true;
  auto issue = [&](int tt) {
    const int lv = tt / tiles_per_level, k0 = (tt - lv * tiles_per_level) * TK;
    mbar_arrive_expect_tx(bar, tile_bytes);
    for (int r0 = 0; r0 < N; r0 += box_rows) tma_load_2d(tile + (size_t)r0 * TK, &tm, k0, lv * N + r0, bar);
    pending = 1;
  };
  int t = g.lev0 * tiles_per_level + blockIdx.x;
  if (tid == 0 && t < ntiles) issue(t);
  for (; t < ntiles; t += gridDim.x, ++it) {
    const int level = t / tiles_per_level, kx0 = (t - level * tiles_per_level) * TK;
    const bool got = mbar_wait_bounded(bar, (unsigned)(it & 1), kWaitPolls);
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    pending = 0;
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = tile[Plain{TK}(st_in_index<N, E, 0>(lane, i)) + l];
    __syncthreads();   // every thread has its inputs before the tile is overwritten
    st_fft_inplace<N, E, SIGN, true, float>(v, tile + l, sw, lane, tw_s, SyncBlock());
    // The in-place transform ends on a barrier after its last reads of the tile, and its outputs are in
    // registers: refill the tile with the next one while this one is stored.
    fence_proxy_async_smem();   // generic writes to the tile come before its refill by TMA
    __syncthreads();
    if (tid == 0 && t + (int)gridDim.x < ntiles) issue(t + gridDim.x);
    const int kx = kx0 + l;
    if (kx < g.nxh) {
      C* col = spec + (long long)level * g.plane + kx;
#pragma unroll
      for (int i = 0; i < E; ++i) col[(long long)st_out_index<N, E>(lane, i) * g.P] = v[i];
    }
  }
  if (tid == 0) {
    if (!ok) atomicOr(err, (unsigned)ERR_WAIT_TIMEOUT);
    if (pending) mbar_wait_bounded(bar, (unsigned)(it & 1), kWaitPolls);   // let a copy in flight land
  }
}

int largest_divisor_upto(int n, int cap) {
  for (int d = cap; d >= 1; --d)
    if (n % d == 0) return d;
  return 1;
}

#define PGB_YS_N_CASE(V, ...) \
  case V: { constexpr int NN = V; if constexpr (st_valid(NN, E)) { __VA_ARGS__; } } break;
#define PGB_YS_N_SWITCH(N, ...)        \
  switch (N) {                         \
    PGB_YS_N_CASE(64, __VA_ARGS__)     \
    PGB_YS_N_CASE(96, __VA_ARGS__)     \
    PGB_YS_N_CASE(128, __VA_ARGS__)    \
    PGB_YS_N_CASE(192, __VA_ARGS__)    \
    PGB_YS_N_CASE(256, __VA_ARGS__)    \
    PGB_YS_N_CASE(384, __VA_ARGS__)    \
    PGB_YS_N_CASE(512, __VA_ARGS__)    \
    PGB_YS_N_CASE(768, __VA_ARGS__)    \
    PGB_YS_N_CASE(1024, __VA_ARGS__)   \
    PGB_YS_N_CASE(1536, __VA_ARGS__)   \
    PGB_YS_N_CASE(2048, __VA_ARGS__)   \
    default: return cudaSuccess;       \
  }

template <int E, int SIGN, bool INPLACE>
cudaError_t ys_launch(float2* spec, const Geom& g, int N, const float2* twy, int tk, const int* done, unsigned* err,
                      cudaStream_t st, bool* used) {
  const size_t smem = ys_smem(N, tk, INPLACE);
  const int nthreads = tk * (N / E);
  if (smem > 220 * 1024 || nthreads > ys_max_threads(E) || nthreads < 32) return cudaSuccess;
  const int box_rows = largest_divisor_upto(N, 256);
  if (((size_t)box_rows * tk * sizeof(float2)) % 128 != 0 && box_rows != N) return cudaSuccess;
  CUtensorMap tm;
  if (!encode_tensor_2d(&tm, spec, 8, (unsigned long long)g.nxh, (unsigned long long)g.ny * g.nz,
                        (unsigned long long)g.P * sizeof(float2), (unsigned)tk, (unsigned)box_rows))
    return cudaSuccess;
  const int tiles_per_level = (g.nxh + tk - 1) / tk;
  const int ntiles = tiles_per_level * g.lev1;
  const int chunk_tiles = tiles_per_level * (g.lev1 - g.lev0);
  static std::mutex mu;
  static std::unordered_map<const void*, std::pair<size_t, int>> granted;   // per kernel: smem, CTAs per SM
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  PGB_YS_N_SWITCH(N, {
    auto kern = k_ys<NN, E, SIGN, INPLACE>;
    int per_sm = 0;
    {
      std::lock_guard<std::mutex> lock(mu);
      auto& ent = granted[reinterpret_cast<const void*>(kern)];
      if (ent.first != smem || ent.second == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, smem);
        if (e != cudaSuccess) return e;
        ent = {smem, per_sm};
      }
      per_sm = ent.second;
    }
    if (per_sm < 1) return cudaSuccess;
    const int grid = chunk_tiles < sms * per_sm ? chunk_tiles : sms * per_sm;
    if (grid <= 0) return cudaSuccess;
    e = pdl_launch(kern, dim3(grid), dim3(tk, N / E), smem, st, tm, g, twy, spec, box_rows, tiles_per_level, ntiles,
                   done, err);
    if (e != cudaSuccess) return e;
    *used = true;
  });
  return cudaGetLastError();
}


template <int E, int SIGN>
cudaError_t ys1_launch(float2* spec, const Geom& g, int N, const float2* twy, int tk, const int* done, unsigned* err,
                       cudaStream_t st, bool* used) {
  const size_t smem = ys_tile_bytes(N, tk) + (size_t)N * sizeof(float2) + 64;
  const int nthreads = tk * (N / E);
  if (smem > 110 * 1024 || nthreads > ys1_max_threads(E) || nthreads < 32) return cudaSuccess;
  const int box_rows = largest_divisor_upto(N, 256);
  if (((size_t)box_rows * tk * sizeof(float2)) % 128 != 0 && box_rows != N) return cudaSuccess;
  CUtensorMap tm;
  if (!encode_tensor_2d(&tm, spec, 8, (unsigned long long)g.nxh, (unsigned long long)g.ny * g.nz,
                        (unsigned long long)g.P * sizeof(float2), (unsigned)tk, (unsigned)box_rows))
    return cudaSuccess;
  const int tiles_per_level = (g.nxh + tk - 1) / tk;
  const int ntiles = tiles_per_level * g.lev1;
  const int chunk_tiles = tiles_per_level * (g.lev1 - g.lev0);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  PGB_YS_N_SWITCH(N, {
    auto kern = k_ys1<NN, E, SIGN>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaSuccess;
    const int grid = chunk_tiles < sms * per_sm ? chunk_tiles : sms * per_sm;
    if (grid <= 0) return cudaSuccess;
    e = pdl_launch(kern, dim3(grid), dim3(tk, N / E), smem, st, tm, g, twy, spec, box_rows, tiles_per_level, ntiles,
                   done, err);
    if (e != cudaSuccess) return e;
    *used = true;
  });
  return cudaGetLastError();
}

}  // namespace

bool ypass_static_supported(int ny) {
  switch (ny) {
    case 64: case 96: case 128: case 192: case 256: case 384: case 512: case 768: case 1024: case 1536: case 2048:
      return true;
    default: return false;
  }
}

cudaError_t launch_yfft_static(int sign, void* spec, const Geom& g, const FftPlan& fy, const Tables& tb, int tile,
                               int variant, const int* done, unsigned* err, cudaStream_t st, bool* used) {
  *used = false;
  if (!ypass_static_supported(fy.n)) return cudaSuccess;
  int tk = tile > 0 ? tile : 8;   // 64-byte TMA box rows (measured best untuned at 1024^2 and on small domains)
  if (tk % 2) tk += 1;   // 16-byte inner TMA box
  // kE3 elements per thread when ny has a factor 3 (radix 3, then 4)
  const int E = fy.n % 3 == 0 ? kE3 : (fy.E == 16 ? 16 : 8);
  if (variant == 2 && (E == 16 || E == kE3)) {   // single-buffered, in place, two CTAs per SM
    int tk1 = tk;
    while (tk1 > 2 && tk1 * (fy.n / E) > ys1_max_threads(E)) tk1 >>= 1;
    float2* sp = (float2*)spec;
    cudaError_t e;
    if (E == 16)
      e = sign < 0 ? ys1_launch<16, -1>(sp, g, fy.n, tb.twy_f, tk1, done, err, st, used)
                   : ys1_launch<16, +1>(sp, g, fy.n, tb.twy_f, tk1, done, err, st, used);
    else
      e = sign < 0 ? ys1_launch<kE3, -1>(sp, g, fy.n, tb.twy_f, tk1, done, err, st, used)
                   : ys1_launch<kE3, +1>(sp, g, fy.n, tb.twy_f, tk1, done, err, st, used);
    if (e != cudaSuccess || *used) return e;
  }
  const bool inplace = variant == 1;
  while (tk > 2 && (ys_smem(fy.n, tk, inplace) > 220 * 1024 || tk * (fy.n / E) > ys_max_threads(E))) tk >>= 1;
  float2* sp = (float2*)spec;
#define PGB_YS_CALL(EE, SG)                                                                   \
  return inplace ? ys_launch<EE, SG, true>(sp, g, fy.n, tb.twy_f, tk, done, err, st, used)    \
                 : ys_launch<EE, SG, false>(sp, g, fy.n, tb.twy_f, tk, done, err, st, used)
  if (E == kE3) {
    if (sign < 0) PGB_YS_CALL(kE3, -1);
    PGB_YS_CALL(kE3, +1);
  }
  if (E == 16) {
    if (sign < 0) PGB_YS_CALL(16, -1);
    PGB_YS_CALL(16, +1);
  }
  if (sign < 0) PGB_YS_CALL(8, -1);
  PGB_YS_CALL(8, +1);
#undef PGB_YS_CALL
}

}  // namespace pgb
