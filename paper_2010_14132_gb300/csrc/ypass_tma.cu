// Persistent y-pass with TMA tile staging (Section 2.1: the transform along y
// for all data of a level, one dimension at a time).
//
// The spectrum [nz][ny][P] is a 2-D tensor of ny*nz rows by nx/2+1 complex
// columns (row stride P).  A tile is one level and TK consecutive kx columns:
// ny rows of TK complex values, loaded by 2-D TMA boxes straight into the
// [ny][TK] shared layout the Stockham stages use, transformed in place, and
// written back by 2-D TMA stores.  Each CTA walks tiles with two shared buffers:
// the load of its next tile is in flight while it transforms the current one,
// and the store of a tile drains while the next is computed.  Columns beyond
// nx/2 are filled with zeros on load and clipped on store by the TMA unit.
#include <mutex>

#include "async_copy.cuh"
#include "kernels.cuh"

namespace pgb {

constexpr long long kTmaWaitPolls = 1LL << 22;

template <typename T, int E, int SIGN>
__global__ void __launch_bounds__(512) k_yfft_tma(const __grid_constant__ CUtensorMap tm, Geom g, FftPlan fy,
                                                  const typename CT<T>::t* __restrict__ twy, int box_rows,
                                                  int tiles_per_level, int ntiles, const int* __restrict__ done,
                                                  Stats* stats) {
  using C = typename CT<T>::t;
  if (done && *done) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int ny = fy.n, TK = blockDim.x, l = threadIdx.x, lane = threadIdx.y;
  const int tid = lane * TK + l;
  const size_t tile_elems = (size_t)ny * TK;
  const unsigned tile_bytes = (unsigned)(tile_elems * sizeof(C));
  const size_t buf_stride = ((size_t)tile_bytes + 127) & ~(size_t)127;   // TMA shared destinations: 128 B
  C* buf[2] = {reinterpret_cast<C*>(smraw), reinterpret_cast<C*>(smraw + buf_stride)};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + 2 * buf_stride);
  constexpr int XM = sizeof(C) / 8;   // tensor elements per complex value (8-byte elements)
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue_load = [&](int t, C* dst, uint64_t* b) {
    const int level = t / tiles_per_level, kx0 = (t - level * tiles_per_level) * TK;
    mbar_arrive_expect_tx(b, tile_bytes);
    for (int r0 = 0; r0 < ny; r0 += box_rows)
      tma_load_2d(dst + (size_t)r0 * TK, &tm, kx0 * XM, level * ny + r0, b);
  };
  // tiles of the levels [g.lev0, g.lev1) of this launch
  int t = g.lev0 * tiles_per_level + blockIdx.x;
  if (tid == 0 && t < ntiles) issue_load(t, buf[0], &bar[0]);
  bool ok = true;
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int b = it & 1;
    const int tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) {
      bulk_wait_read_all();   // the store that last used the other buffer has read it
      issue_load(tn, buf[b ^ 1], &bar[b ^ 1]);
    }
    // every thread waits (bounded); the decision to give up is block-uniform
    const bool got = mbar_wait_bounded(&bar[b], (unsigned)((it >> 1) & 1), kTmaWaitPolls);
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    stockham_run<E, SIGN, T>(buf[b] + l, Strided{TK}, fy, lane, twy, SyncBlock());
    fence_proxy_async_smem();   // this thread's shared writes become visible to the TMA unit
    __syncthreads();
    if (tid == 0) {
      const int level = t / tiles_per_level, kx0 = (t - level * tiles_per_level) * TK;
      for (int r0 = 0; r0 < ny; r0 += box_rows)
        tma_store_2d(&tm, kx0 * XM, level * ny + r0, buf[b] + (size_t)r0 * TK);
      bulk_commit();
    }
  }
  if (!ok && tid == 0) {
    atomicOr(&stats->err, (unsigned)ERR_WAIT_TIMEOUT);
    // let loads in flight land before the CTA's shared memory is released
    mbar_wait_bounded(&bar[0], 0, kTmaWaitPolls);
    mbar_wait_bounded(&bar[1], 0, kTmaWaitPolls);
  }
  if (tid == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// host side: tensor-map encoding through the runtime's driver entry point
// ---------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

bool encode_tensor_2d(CUtensorMap* tm, void* base, size_t elem_bytes, unsigned long long dim0,
                      unsigned long long dim1, unsigned long long row_stride_bytes, unsigned box0, unsigned box1) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || (elem_bytes != 8)) return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)dim0, (cuuint64_t)dim1};
  const cuuint64_t gstride[1] = {(cuuint64_t)row_stride_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)box0, (cuuint32_t)box1};
  const cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

bool encode_tensor_3d(CUtensorMap* tm, void* base, unsigned long long dim0, unsigned long long dim1,
                      unsigned long long dim2, unsigned long long stride1_bytes, unsigned long long stride2_bytes,
                      unsigned box0, unsigned box1, unsigned box2) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t gdim[3] = {(cuuint64_t)dim0, (cuuint64_t)dim1, (cuuint64_t)dim2};
  const cuuint64_t gstride[2] = {(cuuint64_t)stride1_bytes, (cuuint64_t)stride2_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, (cuuint32_t)box2};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

static int largest_divisor_upto(int n, int cap) {
  for (int d = cap; d >= 1; --d)
    if (n % d == 0) return d;
  return 1;
}

// Tile width and box height of the TMA y-pass; 0 when the shape does not fit.
static int tma_tile(int ny, int E, size_t csize, int request) {
  int tk = request > 0 ? request : (csize == 8 ? 8 : 4);
  if (tk % 2) tk += 1;   // 16-byte inner box
  while (tk > 2 && (long long)tk * (ny / E) > 512) tk >>= 1;
  while (tk > 2 && 2 * (size_t)tk * ny * csize + 64 > 220 * 1024) tk >>= 1;
  if ((long long)tk * (ny / E) > 512 || 2 * (size_t)tk * ny * csize + 64 > 220 * 1024) return 0;
  return tk;
}

template <typename T, int SIGN>
static cudaError_t yfft_tma_t(typename CT<T>::t* spec, const Geom& g, const FftPlan& fy,
                              const typename CT<T>::t* twy, int tile, const int* done, Stats* stats, cudaStream_t st,
                              bool* used) {
  using C = typename CT<T>::t;
  *used = false;
  const int tk = tma_tile(fy.n, fy.E, sizeof(C), tile);
  if (tk == 0 || fy.n < 2) return cudaSuccess;
  const int XM = sizeof(C) / 8;
  const int box_rows = largest_divisor_upto(fy.n, 256);
  if (((size_t)box_rows * tk * sizeof(C)) % 128 != 0 && box_rows != fy.n) return cudaSuccess;  // unaligned boxes
  CUtensorMap tm;
  // 8-byte tensor elements: a float complex is one element, a double complex two
  if (!encode_tensor_2d(&tm, spec, 8, (unsigned long long)g.nxh * XM, (unsigned long long)g.ny * g.nz,
                        (unsigned long long)g.P * sizeof(C), (unsigned)(tk * XM), (unsigned)box_rows))
    return cudaSuccess;   // fall back to the plain y-pass
  const int tiles_per_level = (g.nxh + tk - 1) / tk;
  const int ntiles = tiles_per_level * g.lev1;   // end tile of the chunk
  const int chunk_tiles = tiles_per_level * (g.lev1 - g.lev0);
  const size_t smem = 2 * ((((size_t)tk * fy.n * sizeof(C)) + 127) & ~(size_t)127) + 64;
  const dim3 block(tk, fy.n / fy.E);
  cudaError_t e = cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
#define PGB_YTMA_CASE(EV)                                                                                       \
  case EV: {                                                                                                    \
    auto kern = k_yfft_tma<T, EV, SIGN>;                                                                        \
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                     \
    if (e != cudaSuccess) return e;                                                                             \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block.x * block.y, smem);                      \
    if (per_sm < 1) return cudaSuccess;                                                                         \
    const int grid = chunk_tiles < sms * per_sm ? chunk_tiles : sms * per_sm;                                   \
    kern<<<grid, block, smem, st>>>(tm, g, fy, twy, box_rows, tiles_per_level, ntiles, done, stats);            \
    *used = true;                                                                                               \
  } break;
  switch (fy.E) {
    PGB_YTMA_CASE(2)
    PGB_YTMA_CASE(3)
    PGB_YTMA_CASE(4)
    PGB_YTMA_CASE(6)
    PGB_YTMA_CASE(8)
    PGB_YTMA_CASE(12)
    PGB_YTMA_CASE(16)
    PGB_YTMA_CASE(24)
    default: return cudaSuccess;
  }
#undef PGB_YTMA_CASE
  return cudaGetLastError();
}

cudaError_t launch_yfft_tma(int t_is_double, int sign, void* spec, const Geom& g, const FftPlan& fy,
                            const Tables& tb, int tile, const int* done, Stats* stats, cudaStream_t st, bool* used) {
  if (t_is_double) {
    if (sign < 0) return yfft_tma_t<double, -1>((double2*)spec, g, fy, tb.twy_d, tile, done, stats, st, used);
    return yfft_tma_t<double, +1>((double2*)spec, g, fy, tb.twy_d, tile, done, stats, st, used);
  }
  if (sign < 0) return yfft_tma_t<float, -1>((float2*)spec, g, fy, tb.twy_f, tile, done, stats, st, used);
  return yfft_tma_t<float, +1>((float2*)spec, g, fy, tb.twy_f, tile, done, stats, st, used);
}

}  // namespace pgb
