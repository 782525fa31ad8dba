// Fused spectral middle of one pass of the direct solve: the y transform of every
// kx column, the tridiagonal solve of every (kx, ky) column and the inverse y
// transform (Section 2.1), in one persistent kernel, so that the spectrum is not
// sent back to HBM between the three steps.  This is the single-GPU form of the
// further work of Section 4 (not going back to the transform layout between the
// steps of the solve).
//
// The half spectrum [nz][ny][P] is cut into strips of TK = 8 consecutive kx.
// The kernel works through a list of items, built once per plan:
//   Y(s, k)  forward y transform of strip s at level k   ([ny][TK] tile, 2-D TMA)
//   C(s, t)  FP32 column solves of strip s for ky in [TY t, TY t + TY)
//            ([nz][TY][TK] tile, one 3-D TMA box; two threads per column)
//   L(s, j)  low-|k| or singular column j of the plan's list (strip s), in the
//            precision of the low-|k| columns, by the whole CTA
//   I(s, k)  inverse y transform of strip s at level k
// C and L items of strip s wait until every Y(s, .) is done; I(s, .) items until
// every C(s, .) and L(s, .) is done (per-strip counters in the workspace, acquire
// loads, bounded waits).  The list is a software pipeline over strips: Y of strip
// q, then the low-|k| and column items of strip q - 2, then I of strip q - 4.  CTAs
// take items in list order with an atomic ticket, so a strip's spectrum (ny nz TK
// entries: 8 MB at 1024 x 1024 x 128) is written by its Y items, solved and read
// back by its I items while it is still in L2: HBM sees the spectrum once in and
// once out per pass instead of three times each way.
//
// Progress: every item a CTA waits for precedes its own in the list, and was taken
// by a running CTA whose waits point further back still, so every wait ends
// (without any assumption on how many CTAs are resident).  A wait that runs out
// of polls sets ERR_WAIT_TIMEOUT, skips its item and still counts it done, so the
// items behind it are not held up; the solve then reports POISSON_ERR_TIMEOUT.
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "async_copy.cuh"
#include "columns.cuh"
#include "fft_static.cuh"
#include "kernels.cuh"

namespace pgb {

namespace {

constexpr int kMidTK = 8;                  // kx columns per strip (64-byte tile rows)
constexpr int kMidE = 16;                  // elements per thread of the y transforms
constexpr long long kSpinPolls = 1LL << 22;

enum MidPhase : int { MID_Y = 0, MID_C = 1, MID_L = 2, MID_I = 3 };

// y-tile addressing: TK interleaved columns, the complex index swizzled inside blocks of 16
// (spreads the stride-R first-stage writes over the banks)
struct SwTile {
  __device__ __forceinline__ int operator()(int idx) const { return (idx ^ ((idx >> 4) & 15)) * kMidTK; }
};

struct MidArgs {
  float2* spec;
  Geom g;
  const float2* twy;
  const float* a_f;
  const float* c_f;
  const float* lamx;
  const float* lamy;
  float scale;
  int lowk_r2;
  LowkArgs L;
  const int* items;     // the item list, then the C + L item count of every strip
  int nitems;
  int nstrips;
  unsigned* sched;      // [0] ticket, [1 + s] Y items done in strip s, [1 + nstrips + s] C and L items done
  int box_rows;         // rows per 2-D box of a y tile
  int box_z;            // levels per 3-D box of a column tile
  const int* done;
  Stats* stats;
};

// Shared layout: y twiddles [N] (stage order), (a_k, c_k) [nz], one mbarrier, the
// item slot; then, 128-byte aligned, the item buffer (a y tile, a column tile with
// its factors and meeting terms, or the low-|k| column scratch).
__host__ __device__ constexpr size_t mid_buf_offset(int N, int nz) {
  return ((size_t)N * 8 + (size_t)((nz + 1) & ~1) * 8 + 8 + 16 + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t mid_buf_bytes(int N, int nz, int TC, size_t lowk_elem) {
  const size_t y = (size_t)N * kMidTK * 8;
  const size_t c = (size_t)nz * TC * 12 + (size_t)TC * 24;
  const size_t l = lowk_smem_elems(nz) * lowk_elem;
  return y > c ? (y > l ? y : l) : (c > l ? c : l);
}

template <int N, int TC, typename TCm>
__global__ void __launch_bounds__(kMidTK * (N / kMidE), 2)
    k_mid(const __grid_constant__ CUtensorMap tmy, const __grid_constant__ CUtensorMap tmc, MidArgs A) {
  using C = float2;
  constexpr int E = kMidE, TK = kMidTK, NT = TK * (N / E), TY = TC / TK;
  static_assert(2 * TC <= NT, "a column item needs two threads per column");
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smraw[];
  const int tid = threadIdx.x, nz = A.g.nz;
  C* tw_s = reinterpret_cast<C*>(smraw);
  float2* ac = reinterpret_cast<float2*>(tw_s + N);
  uint64_t* bar = reinterpret_cast<uint64_t*>(ac + ((nz + 1) & ~1));
  int* slot = reinterpret_cast<int*>(bar + 1);   // [0] item, [1] skip
  unsigned char* buf = smraw + mid_buf_offset(N, nz);
  st_build_twiddles<N, E>(tw_s, A.twy, tid, NT);
  for (int k = tid; k < nz; k += NT) ac[k] = make_float2(A.a_f[k], A.c_f[k]);
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  pdl_wait();   // the previous kernels of the stream are complete
  if (A.done && *A.done) return;
  unsigned* ticket = A.sched;
  unsigned* ydone = A.sched + 1;
  unsigned* cdone = A.sched + 1 + A.nstrips;
  const int* ctarget = A.items + A.nitems;
  const Geom& g = A.g;
  unsigned loads = 0;   // TMA loads this CTA has waited for on bar (its phase parity)
  bool ok = true;
  for (;;) {
    if (tid == 0) {
      const unsigned t = atomicAdd(ticket, 1u);
      int item = -1, skip = 0;
      if (t < (unsigned)A.nitems) {
        item = __ldg(&A.items[t]);
        const int ph = item & 3, s = (item >> 2) & 1023;
        const unsigned* cnt = nullptr;
        unsigned target = 0;
        if (ph == MID_C || ph == MID_L) {
          cnt = ydone + s;
          target = (unsigned)nz;
        } else if (ph == MID_I) {
          cnt = cdone + s;
          target = (unsigned)__ldg(&ctarget[s]);
        }
        if (cnt) {
          long long i = 0;
          while (ld_acquire_gpu(cnt) < target && i < kSpinPolls) {
            __nanosleep(64);
            ++i;
          }
          if (i == kSpinPolls) {
            atomicOr(&A.stats->err, (unsigned)ERR_WAIT_TIMEOUT);
            skip = 1;
          }
          fence_proxy_async_global();   // the producers' spectrum writes come before this CTA's tile loads
        }
      }
      slot[0] = item;
      slot[1] = skip;
    }
    __syncthreads();
    const int item = slot[0], skip = slot[1];
    if (item < 0) break;
    const int ph = item & 3, s = (item >> 2) & 1023, sub = item >> 12;
    if (!skip) {
      if (ph == MID_Y || ph == MID_I) {
        C* tile = reinterpret_cast<C*>(buf);
        if (tid == 0) {
          mbar_arrive_expect_tx(bar, (unsigned)(N * TK * sizeof(C)));
          for (int r0 = 0; r0 < N; r0 += A.box_rows) tma_load_2d(tile + (size_t)r0 * TK, &tmy, TK * s, sub * N + r0, bar);
        }
        const bool got = mbar_wait_bounded(bar, loads & 1u, kWaitPolls);
        ++loads;
        if (!__syncthreads_and(got)) {
          ok = false;
          break;
        }
        const int l = tid % TK, lane = tid / TK;
        C v[E];
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = tile[st_in_index<N, E, 0>(lane, i) * TK + l];
        __syncthreads();   // every thread has its inputs before the tile is overwritten
        if (ph == MID_Y) st_fft_inplace<N, E, -1, true, float>(v, tile + l, SwTile{}, lane, tw_s, SyncBlock());
        else st_fft_inplace<N, E, +1, true, float>(v, tile + l, SwTile{}, lane, tw_s, SyncBlock());
        const int kx = TK * s + l;
        if (kx < g.nxh) {
          C* col = A.spec + (long long)sub * g.plane + kx;
#pragma unroll
          for (int i = 0; i < E; ++i) col[(long long)st_out_index<N, E>(lane, i) * g.P] = v[i];
        }
      } else if (ph == MID_C) {
        C* tile = reinterpret_cast<C*>(buf);
        float* wv = reinterpret_cast<float*>(tile + (size_t)nz * TC);
        float4* meet = reinterpret_cast<float4*>(wv + (size_t)nz * TC);
        float2* xm_s = reinterpret_cast<float2*>(meet + TC);
        if (tid == 0) {
          mbar_arrive_expect_tx(bar, (unsigned)(TC * sizeof(C)) * (unsigned)nz);
          for (int z0 = 0; z0 < nz; z0 += A.box_z) tma_load_3d(tile + (size_t)z0 * TC, &tmc, TK * s, TY * sub, z0, bar);
        }
        const bool got = mbar_wait_bounded(bar, loads & 1u, kWaitPolls);
        ++loads;
        if (!__syncthreads_and(got)) {
          ok = false;
          break;
        }
        const bool part = tid < 2 * TC;
        const int col_t = tid % TC, upper = tid / TC;
        const int kx = TK * s + col_t % TK, ky = TY * sub + col_t / TK;
        const int kys = signed_ky(ky, g.ny);
        const bool valid = part && kx < g.nxh && ky < g.ny && (kx * kx + kys * kys > A.lowk_r2);
        const float sv = valid ? -(A.lamx[kx] + A.lamy[ky]) : 1.f;
        tw_solve_tile(tile + col_t, wv + col_t, ac, meet, xm_s, TC, nz, col_t, upper, part, valid, sv, -A.scale,
                      A.spec + (valid ? (long long)ky * g.P + kx : 0), g.plane);
      } else {   // MID_L
        lowk_column<float, TCm, false>(buf, A.spec, g, A.L.a_d, A.L.c_d, A.L.W_d, A.L.lamx_d, A.L.lamy_d, A.L.scale,
                                       A.L.cols[sub], A.stats, A.L.target_mean, A.L.singular00 != 0, nullptr,
                                       A.L.inv_tab, sub);
      }
    }
    // the item's shared-memory accesses precede the next TMA write into the buffer, and its spectrum
    // writes precede the counter release
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      if (ph == MID_Y) atomicAdd(ydone + s, 1u);
      else if (ph == MID_C || ph == MID_L) atomicAdd(cdone + s, 1u);
    }
  }
  if (tid == 0 && !ok) {
    atomicOr(&A.stats->err, (unsigned)ERR_WAIT_TIMEOUT);
    mbar_wait_bounded(bar, (loads - 1u) & 1u, kWaitPolls);   // let the copy in flight land before exiting
  }
}

// Columns per column item: two threads per column within the block, factors and tile within
// the shared budget of two CTAs per SM.
int mid_tc(int ny, int nz) {
  const int nt = kMidTK * (ny / kMidE);
  for (int tc = 64; tc >= 32; tc >>= 1) {
    if (2 * tc > nt) continue;
    const size_t total = mid_buf_offset(ny, nz) + mid_buf_bytes(ny, nz, tc, 8);
    if (total <= 110 * 1024) return tc;
  }
  return 0;
}

bool mid_shape_ok(int ny, int nz) {
  if (ny != 256 && ny != 512 && ny != 1024) return false;
  if (nz < 2 || nz > 256) return false;
  return mid_tc(ny, nz) != 0;
}

}  // namespace

bool spectral_fused_supported(int ny, int nz) { return mid_shape_ok(ny, nz); }

// The item list of a plan (host): see the file comment.  lowk_kx: kx of every listed low-|k|
// column.  Appends, after the items, the C + L item count of each strip.
std::vector<int> spectral_fused_items(int nxh, int ny, int nz, const std::vector<int>& lowk_kx, int* nitems) {
  const int TK = kMidTK, tc = mid_tc(ny, nz);
  std::vector<int> out;
  if (tc == 0) {
    *nitems = 0;
    return out;
  }
  const int ty = tc / TK, nstrips = (nxh + TK - 1) / TK, nct = (ny + ty - 1) / ty;
  std::vector<std::vector<int>> lowk(nstrips);
  for (size_t j = 0; j < lowk_kx.size(); ++j) lowk[lowk_kx[j] / TK].push_back((int)j);
  auto enc = [](int ph, int s, int sub) { return ph | (s << 2) | (sub << 12); };
  constexpr int D = 2;   // lag between the phases of the pipeline, in strips
  for (int q = 0; q < nstrips + 2 * D; ++q) {
    if (q < nstrips)
      for (int k = 0; k < nz; ++k) out.push_back(enc(MID_Y, q, k));
    const int sc = q - D;
    if (sc >= 0 && sc < nstrips) {
      for (int j : lowk[sc]) out.push_back(enc(MID_L, sc, j));   // the long double-precision columns first
      for (int t = 0; t < nct; ++t) out.push_back(enc(MID_C, sc, t));
    }
    const int si = q - 2 * D;
    if (si >= 0 && si < nstrips)
      for (int k = 0; k < nz; ++k) out.push_back(enc(MID_I, si, k));
  }
  *nitems = (int)out.size();
  for (int s = 0; s < nstrips; ++s) out.push_back(nct + (int)lowk[s].size());
  return out;
}

int spectral_fused_sched_words(int nxh) { return 1 + 2 * ((nxh + kMidTK - 1) / kMidTK); }

cudaError_t launch_spectral_fused(const ThomasArgs& T, const Geom& g, const FftPlan& fy, const Tables& tb,
                                  const int* items, int nitems, unsigned* sched, cudaStream_t st, bool* used) {
  *used = false;
  if (T.t_is_double || T.adjoint || !mid_shape_ok(g.ny, g.nz) || fy.n != g.ny || nitems <= 0) return cudaSuccess;
  if (g.lev0 != 0 || g.lev1 != g.nz) return cudaSuccess;
  const int tc = mid_tc(g.ny, g.nz);
  const int TK = kMidTK;
  CUtensorMap tmy, tmc;
  std::memset(&tmy, 0, sizeof(tmy));
  std::memset(&tmc, 0, sizeof(tmc));
  int box_rows = 256;
  while (g.ny % box_rows) box_rows >>= 1;
  const int box_z = g.nz <= 256 ? g.nz : 256;
  if (!encode_tensor_2d(&tmy, T.spec, 8, (unsigned long long)g.nxh, (unsigned long long)g.ny * g.nz,
                        (unsigned long long)g.P * 8, (unsigned)TK, (unsigned)box_rows))
    return cudaSuccess;
  if (!encode_tensor_3d(&tmc, T.spec, (unsigned long long)g.nxh, (unsigned long long)g.ny, (unsigned long long)g.nz,
                        (unsigned long long)g.P * 8, (unsigned long long)g.plane * 8, (unsigned)TK,
                        (unsigned)(tc / TK), (unsigned)box_z))
    return cudaSuccess;
  MidArgs A{};
  A.spec = (float2*)T.spec;
  A.g = g;
  A.twy = tb.twy_f;
  A.a_f = tb.a_f;
  A.c_f = tb.c_f;
  A.lamx = tb.lamx_f;
  A.lamy = tb.lamy_f;
  A.scale = (float)T.scale;
  A.lowk_r2 = T.lowk_r2;
  A.L = LowkArgs{T.lowk_cols, T.n_lowk, tb.a_d, tb.c_d, tb.W_d, tb.lamx_d, tb.lamy_d, T.target_mean, T.scale,
                 T.singular00, T.lowk_inv};
  A.items = items;
  A.nitems = nitems;
  A.nstrips = (g.nxh + TK - 1) / TK;
  A.sched = sched;
  A.box_rows = box_rows;
  A.box_z = box_z;
  A.done = T.done;
  A.stats = T.stats;
  const size_t lowk_elem = T.lowk_double ? 8 : 4;
  const size_t smem = mid_buf_offset(g.ny, g.nz) + mid_buf_bytes(g.ny, g.nz, tc, lowk_elem);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  static std::mutex mu;
  static std::unordered_map<const void*, std::pair<size_t, int>> granted;
  cudaError_t e = cudaSuccess;
  auto run = [&](auto kern, int nthreads) -> cudaError_t {
    int per_sm = 0;
    {
      std::lock_guard<std::mutex> lock(mu);
      auto& ent = granted[reinterpret_cast<const void*>(kern)];
      if (ent.first < smem || ent.second == 0) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, smem);
        if (r != cudaSuccess) return r;
        ent = {smem, per_sm};
      }
      per_sm = ent.second;
    }
    if (per_sm < 1) return cudaSuccess;
    long long grid = (long long)sms * per_sm;
    if (grid > nitems) grid = nitems;
    *used = true;
    return pdl_launch(kern, dim3((unsigned)grid), dim3(nthreads), smem, st, tmy, tmc, A);
  };
#define PGB_MID_CASE(NN)                                                                                  \
  case NN: {                                                                                              \
    constexpr int nt = kMidTK * (NN / kMidE);                                                             \
    if (tc == 64 && 2 * 64 <= nt)                                                                         \
      e = T.lowk_double ? run(k_mid<NN, 64, double>, nt) : run(k_mid<NN, 64, float>, nt);                 \
    else                                                                                                  \
      e = T.lowk_double ? run(k_mid<NN, 32, double>, nt) : run(k_mid<NN, 32, float>, nt);                 \
  } break;
  switch (g.ny) {
    PGB_MID_CASE(256)
    PGB_MID_CASE(512)
    PGB_MID_CASE(1024)
    default: break;
  }
#undef PGB_MID_CASE
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace pgb
