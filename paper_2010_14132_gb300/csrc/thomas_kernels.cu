// Vertical column solves of the direct method (Section 2.1: after the forward
// transform each (kx, ky) wavenumber gives an independent tridiagonal system
// along z, solved up and down the column).
//
// Column matrix T = L_z + (lambda_x + lambda_y) I.  With M = -T (an M-matrix:
// diagonal a_k + c_k + s, off-diagonals -a_k, -c_k, row sums s = -(lambda_x +
// lambda_y) >= 0) the LU pivots are formed without subtraction:
//     g_0 = s,  u_k = g_k + c_k,  g_k = s + a_k g_{k-1} / u_{k-1},
// (g_k is the row sum of the reduced row k), so every pivot is relatively
// accurate however close s is to 0.  For s = 0 (the (0,0) column) g vanishes
// identically; with zero flux through the top face the last pivot is then
// exactly 0, the singular mode.  With p = 0 on the top face (Dirichlet) the top
// coupling c_{nz-1} > 0 enters the last pivot and every column is nonsingular.
//   forward solve   M x = b:  y_k = b_k + (a_k/u_{k-1}) y_{k-1};  x_k = y_k/u_k + (c_k/u_k) x_{k+1}
//   adjoint solve M^T x = b:  v_k = (b_k + c_{k-1} v_{k-1})/u_k;   x_k = v_k + (a_{k+1}/u_k) x_{k+1}
// The spectrum is scaled by 1/(nx ny) here, which makes the inverse transforms
// unnormalised.
#include <cstring>

#include "kernels.cuh"
#include "async_copy.cuh"
#include "columns.cuh"

namespace pgb {

// ---------------------------------------------------------------------------
// Main column kernel: one thread per column, a tile of TC consecutive columns
// (flattened (ky, kx) index with pitch P) staged for all nz levels.
// Shared layout: tile [nz][TC] complex, wv [nz][TC] real, one mbarrier.
// Blocks [0, L.n) solve the listed low-|k| / singular columns (precision TCm);
// the others solve tiles of TC consecutive columns.  The two sets of columns are
// disjoint (the tile blocks skip listed columns), so they run concurrently.
template <typename T, typename TCm, bool ADJ>
__global__ void __launch_bounds__(128) k_thomas(typename CT<T>::t* __restrict__ spec, Geom g,
                                                const T* __restrict__ a, const T* __restrict__ c,
                                                const T* __restrict__ lamx, const T* __restrict__ lamy, T scale,
                                                int lowk_r2, const int* __restrict__ done, Stats* stats,
                                                const __grid_constant__ CUtensorMap tm, int use_tma, int box_rows,
                                                LowkArgs L) {
  using C = typename CT<T>::t;
  if (done && *done) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  if ((int)blockIdx.x < L.n) {
    lowk_column<T, TCm, ADJ>(smraw, spec, g, L.a_d, L.c_d, L.W_d, L.lamx_d, L.lamy_d, L.scale,
                             L.cols[blockIdx.x], stats, L.target_mean, L.singular00 != 0, nullptr, L.inv_tab,
                             blockIdx.x);
    return;
  }
  const int TC = blockDim.x, t = threadIdx.x, nz = g.nz;
  C* tile = reinterpret_cast<C*>(smraw);
  T* wv = reinterpret_cast<T*>(tile + (size_t)nz * TC);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + (((size_t)nz * TC * (sizeof(C) + sizeof(T)) + 15) & ~(size_t)15));

  const long long ncols = g.plane;
  const long long c0 = (long long)(blockIdx.x - L.n) * TC;
  const int tcv = (int)((ncols - c0) < TC ? (ncols - c0) : TC);
  const unsigned row_bytes = (unsigned)(tcv * sizeof(C));
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (t == 0) {
    if (use_tma) {
      // one 2-D box per box_rows levels: TC columns x box_rows levels (out-of-range columns read as 0)
      constexpr int XM = sizeof(C) / 8;
      mbar_arrive_expect_tx(bar, (unsigned)(TC * sizeof(C)) * (unsigned)nz);
      for (int k0 = 0; k0 < nz; k0 += box_rows) tma_load_2d(tile + (size_t)k0 * TC, &tm, (int)c0 * XM, k0, bar);
    } else {
      mbar_arrive_expect_tx(bar, row_bytes * (unsigned)nz);
      for (int k = 0; k < nz; ++k) bulk_g2s(tile + (size_t)k * TC, spec + k * g.plane + c0, row_bytes, bar);
    }
  }
  const bool got = mbar_wait_bounded(bar, 0, kWaitPolls);
  if (!__syncthreads_and(got)) {   // any thread's time-out stops the whole CTA and is reported
    if (t == 0) {
      atomicOr(&stats->err, (unsigned)ERR_WAIT_TIMEOUT);
      mbar_wait_bounded(bar, 0, kWaitPolls);   // let copies in flight land before the CTA exits
    }
    return;
  }

  const long long col = c0 + t;
  const int ky = (int)(col / g.P), kx = (int)(col - (long long)ky * g.P);
  const int kys = signed_ky(ky, g.ny);
  const bool valid = t < tcv && kx < g.nxh && (kx * kx + kys * kys > lowk_r2);
  if (!valid) return;

  const T s = -(lamx[kx] + lamy[ky]);
  const T ms = -scale;
  C* colp = tile + t;
  T* wp = wv + t;
  // forward sweep (pivots in level order)
  T g_prev = s, inv_prev = 0;
  C y_prev = make_c<T>(0, 0);
  for (int k = 0; k < nz; ++k) {
    const C d = colp[(size_t)k * TC];
    const C b = make_c<T>(ms * d.x, ms * d.y);
    T gk;
    C y;
    if (k == 0) {
      gk = s;
    } else {
      if (!ADJ) {
        const T f = a[k] * inv_prev;
        gk = s + f * g_prev;
      } else {
        gk = s + a[k] * g_prev * inv_prev;
      }
    }
    const T u = gk + c[k];
    const T inv = rcp(u);
    if (!ADJ) {
      if (k == 0) {
        y = b;
      } else {
        const T f = a[k] * inv_prev;
        y = make_c<T>(b.x + f * y_prev.x, b.y + f * y_prev.y);
      }
      colp[(size_t)k * TC] = make_c<T>(y.x * inv, y.y * inv);
      wp[(size_t)k * TC] = c[k] * inv;
    } else {
      if (k == 0) {
        y = make_c<T>(b.x * inv, b.y * inv);
      } else {
        const T cm = c[k - 1];
        y = make_c<T>((b.x + cm * y_prev.x) * inv, (b.y + cm * y_prev.y) * inv);
      }
      colp[(size_t)k * TC] = y;
      wp[(size_t)k * TC] = (k + 1 < nz) ? a[k + 1] * inv : (T)0;
    }
    g_prev = gk;
    inv_prev = inv;
    y_prev = y;
  }
  // back substitution, written straight to HBM (coalesced across the tile)
  C x = colp[(size_t)(nz - 1) * TC];
  C* out = spec + col;
  out[(long long)(nz - 1) * g.plane] = x;
  for (int k = nz - 2; k >= 0; --k) {
    const C z = colp[(size_t)k * TC];
    const T w = wp[(size_t)k * TC];
    x = make_c<T>(z.x + w * x.x, z.y + w * x.y);
    out[(long long)k * g.plane] = x;
  }
}

// ---------------------------------------------------------------------------
// Paired FP32 column kernel: ky and ny - ky have the same eigenvalue, so the
// columns (kx, ky) and (kx, ny - ky) share one pivot chain.  A CTA takes TC
// consecutive kx of such a pair of rows (a single row for ky = 0 and ky = ny/2),
// stages both [nz][TC] tiles with one 2-D TMA box each, and every thread runs
// the shared pivots with two right-hand sides.  Shared layout: tile a, tile b
// [nz][TC] complex, factors [nz][TC], (a_k, c_k) pairs [nz], one mbarrier.
// ---------------------------------------------------------------------------
template <bool ADJ>
__device__ __forceinline__ void column_solve_pair(float2* ca, float2* cb, float* wp, int TC, int nz, float s, float ms,
                                                  const float2* __restrict__ ac, float2* __restrict__ oa,
                                                  float2* __restrict__ ob, long long plane, bool two) {
  float g_prev = s, inv_prev = 0.f;
  float2 ya = make_float2(0.f, 0.f), yb = ya;
  for (int k = 0; k < nz; ++k) {
    const float2 akc = ac[k];   // (a_k, c_k)
    const float2 da = ca[(size_t)k * TC];
    const float2 db = two ? cb[(size_t)k * TC] : make_float2(0.f, 0.f);
    float gk;
    if (!ADJ) gk = (k == 0) ? s : s + (akc.x * inv_prev) * g_prev;
    else gk = (k == 0) ? s : s + akc.x * g_prev * inv_prev;
    const float u = gk + akc.y;
    const float inv = rcp(u);
    if (!ADJ) {
      const float f = (k == 0) ? 0.f : akc.x * inv_prev;
      ya = make_float2(fmaf(ms, da.x, f * ya.x), fmaf(ms, da.y, f * ya.y));
      yb = make_float2(fmaf(ms, db.x, f * yb.x), fmaf(ms, db.y, f * yb.y));
      ca[(size_t)k * TC] = make_float2(ya.x * inv, ya.y * inv);
      if (two) cb[(size_t)k * TC] = make_float2(yb.x * inv, yb.y * inv);
      wp[(size_t)k * TC] = akc.y * inv;
    } else {
      const float cm = (k == 0) ? 0.f : ac[k - 1].y;
      ya = make_float2(fmaf(ms, da.x, cm * ya.x) * inv, fmaf(ms, da.y, cm * ya.y) * inv);
      yb = make_float2(fmaf(ms, db.x, cm * yb.x) * inv, fmaf(ms, db.y, cm * yb.y) * inv);
      ca[(size_t)k * TC] = ya;
      if (two) cb[(size_t)k * TC] = yb;
      wp[(size_t)k * TC] = (k + 1 < nz) ? ac[k + 1].x * inv : 0.f;
    }
    g_prev = gk;
    inv_prev = inv;
  }
  float2 xa = ca[(size_t)(nz - 1) * TC], xb = two ? cb[(size_t)(nz - 1) * TC] : make_float2(0.f, 0.f);
  oa[(long long)(nz - 1) * plane] = xa;
  if (two) ob[(long long)(nz - 1) * plane] = xb;
  for (int k = nz - 2; k >= 0; --k) {
    const float w = wp[(size_t)k * TC];
    const float2 za = ca[(size_t)k * TC];
    xa = make_float2(za.x + w * xa.x, za.y + w * xa.y);
    oa[(long long)k * plane] = xa;
    if (two) {
      const float2 zb = cb[(size_t)k * TC];
      xb = make_float2(zb.x + w * xb.x, zb.y + w * xb.y);
      ob[(long long)k * plane] = xb;
    }
  }
}

template <typename TCm, bool ADJ>
__global__ void __launch_bounds__(64) k_thomas_pair(float2* __restrict__ spec, Geom g, const float* __restrict__ a,
                                                    const float* __restrict__ c, const float* __restrict__ lamx,
                                                    const float* __restrict__ lamy, float scale, int lowk_r2,
                                                    const int* __restrict__ done, Stats* stats,
                                                    const __grid_constant__ CUtensorMap tm, int box_rows,
                                                    int kx_chunks, LowkArgs L) {
  if (done && *done) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  if ((int)blockIdx.x < L.n) {
    lowk_column<float, TCm, ADJ>(smraw, spec, g, L.a_d, L.c_d, L.W_d, L.lamx_d, L.lamy_d, L.scale,
                                 L.cols[blockIdx.x], stats, L.target_mean, L.singular00 != 0, nullptr, L.inv_tab,
                                 blockIdx.x);
    return;
  }
  const int TC = blockDim.x, t = threadIdx.x, nz = g.nz;
  const size_t tile_bytes = (size_t)nz * TC * sizeof(float2);
  float2* ta = reinterpret_cast<float2*>(smraw);
  float2* tb = reinterpret_cast<float2*>(smraw + tile_bytes);
  float* wv = reinterpret_cast<float*>(smraw + 2 * tile_bytes);
  float2* ac = reinterpret_cast<float2*>(smraw + 2 * tile_bytes + (((size_t)nz * TC * sizeof(float) + 15) & ~(size_t)15));
  uint64_t* bar = reinterpret_cast<uint64_t*>(ac + nz + (nz & 1));
  const int u = (int)blockIdx.x - L.n;
  const int pair = u / kx_chunks, chunk = u - pair * kx_chunks;
  const int ky_a = pair, ky_b = (g.ny - pair) % g.ny;
  const bool two = ky_b != ky_a;
  const int kx0 = chunk * TC;
  for (int k = t; k < nz; k += TC) ac[k] = make_float2(a[k], c[k]);
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (t == 0) {
    mbar_arrive_expect_tx(bar, (unsigned)tile_bytes * (two ? 2u : 1u));
    for (int k0 = 0; k0 < nz; k0 += box_rows) {
      tma_load_2d(ta + (size_t)k0 * TC, &tm, ky_a * g.P + kx0, k0, bar);
      if (two) tma_load_2d(tb + (size_t)k0 * TC, &tm, ky_b * g.P + kx0, k0, bar);
    }
  }
  const bool got = mbar_wait_bounded(bar, 0, kWaitPolls);
  if (!__syncthreads_and(got)) {   // any thread's time-out stops the whole CTA and is reported
    if (t == 0) {
      atomicOr(&stats->err, (unsigned)ERR_WAIT_TIMEOUT);
      mbar_wait_bounded(bar, 0, kWaitPolls);   // let copies in flight land before the CTA exits
    }
    return;
  }
  const int kx = kx0 + t;
  const int kys = signed_ky(ky_a, g.ny);
  if (kx >= g.nxh || kx * kx + kys * kys <= lowk_r2) return;
  const float s = -(lamx[kx] + lamy[ky_a]);
  column_solve_pair<ADJ>(ta + t, tb + t, wv + t, TC, nz, s, -scale, ac, spec + (long long)ky_a * g.P + kx,
                         spec + (long long)ky_b * g.P + kx, g.plane, two);
}


// ---------------------------------------------------------------------------
// Twisted FP32 column kernel (forward solves): two threads per column.  The
// lower thread eliminates levels 0..m-1 upward with the pivots above
// (g_k, u_k = g_k + c_k), the upper thread eliminates levels nz-1..m+1 downward
// with the mirror recurrence h_{nz-1} = s + c_{nz-1} (the top row's sum: c_{nz-1} = 0
// with zero flux, the Dirichlet coupling otherwise), h_k = s + c_k h_{k+1}/v_{k+1},
// v_k = h_k + a_k (again subtraction-free); they meet at level m = nz/2:
//   x_m = (b_m + a_m z_{m-1} + c_m zt_{m+1}) / (s + a_m g_{m-1}/u_{m-1} + c_m h_{m+1}/v_{m+1}),
// (h_{nz}/v_{nz} = 1 and zt_{nz} = 0 when m is the top level),
// then substitute back outward: x_k = z_k + (c_k/u_k) x_{k+1} below m,
// x_k = zt_k + (a_k/v_k) x_{k-1} above m.  Half the sequential chain of the
// one-thread recurrence and twice the threads for the same shared memory.
// Shared layout: tile [nz][TC] complex, factors [nz][TC], (a_k, c_k) [nz], the
// meeting terms [TC] x 4, one mbarrier.
// ---------------------------------------------------------------------------
// sqn (nullable): CTA b stores sqn[b] = sum over its columns of w_kx sum_k |x_k|^2 (w = 1 for
// kx = 0 and nx/2, 2 otherwise), so that Parseval gives the norm of the correction this solve
// computed before the inverse transforms.  kcut >= 0: only the columns with kx <= kcut and
// |ky'| <= kcut are solved; the grid then holds just their tiles, ceil((kcut + 1)/TC) from the start
// of each of the rows ky = 0..kcut and ny - kcut..ny - 1 (P, a multiple of 16, keeps every tile's
// first entry 16-byte aligned for the TMA box).
template <typename TCm>
__global__ void __launch_bounds__(128) k_thomas_tw(float2* __restrict__ spec, Geom g, const float* __restrict__ a,
                                                  const float* __restrict__ c, const float* __restrict__ lamx,
                                                  const float* __restrict__ lamy, float scale, int lowk_r2,
                                                  const int* __restrict__ done, Stats* stats,
                                                  const __grid_constant__ CUtensorMap tm, int box_rows, LowkArgs L,
                                                  double* __restrict__ sqn, int kcut) {
  pdl_trigger();
  pdl_wait();   // the previous kernels of the stream are complete
  if (done && *done) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  if ((int)blockIdx.x < L.n) {
    double sq = 0.0;
    const int2 ck = L.cols[blockIdx.x];
    lowk_column<float, TCm, false>(smraw, spec, g, L.a_d, L.c_d, L.W_d, L.lamx_d, L.lamy_d, L.scale, ck, stats,
                                   L.target_mean, L.singular00 != 0, sqn ? &sq : nullptr, L.inv_tab, blockIdx.x);
    if (sqn && threadIdx.x == 0) sqn[blockIdx.x] = (ck.x == 0 || ck.x == g.nxh - 1 ? 1.0 : 2.0) * sq;
    return;
  }
  const int TC = blockDim.x / 2, t = threadIdx.x, col_t = t % TC, upper = t / TC, nz = g.nz;
  float2* tile = reinterpret_cast<float2*>(smraw);
  float* wv = reinterpret_cast<float*>(tile + (size_t)nz * TC);
  float2* ac = reinterpret_cast<float2*>(smraw + (((size_t)nz * TC * (sizeof(float2) + sizeof(float)) + 15) & ~(size_t)15));
  float4* meet = reinterpret_cast<float4*>(ac + nz + (nz & 1));   // [TC]: lower part's (g-term, z-term re, im, -)
  float2* xm_s = reinterpret_cast<float2*>(meet + TC);             // [TC]: x_m
  uint64_t* bar = reinterpret_cast<uint64_t*>(xm_s + TC);
  long long c0 = (long long)(blockIdx.x - L.n) * TC;
  auto low_row = [&](long long r) { return r <= kcut || r >= g.ny - kcut; };
  if (kcut >= 0) {   // tile jt of low row r
    const int tpr = (kcut + TC) / TC, tb = (int)blockIdx.x - L.n, r = tb / tpr, jt = tb - r * tpr;
    const int ky = r <= kcut ? r : g.ny - (2 * kcut + 1 - r);
    c0 = (long long)ky * g.P + (long long)jt * TC;
  }
  for (int k = t; k < nz; k += blockDim.x) ac[k] = make_float2(a[k], c[k]);
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (t == 0) {
    mbar_arrive_expect_tx(bar, (unsigned)(TC * sizeof(float2)) * (unsigned)nz);
    for (int k0 = 0; k0 < nz; k0 += box_rows) tma_load_2d(tile + (size_t)k0 * TC, &tm, (int)c0, k0, bar);
  }
  const bool got = mbar_wait_bounded(bar, 0, kWaitPolls);
  if (!__syncthreads_and(got)) {
    if (t == 0) {
      atomicOr(&stats->err, (unsigned)ERR_WAIT_TIMEOUT);
      mbar_wait_bounded(bar, 0, kWaitPolls);   // let copies in flight land before the CTA exits
    }
    return;
  }
  const long long col = c0 + col_t;
  const int ky = (int)(col / g.P), kx = (int)(col - (long long)ky * g.P);
  const int kys = signed_ky(ky, g.ny);
  const bool valid = col < g.plane && kx < g.nxh && (kx * kx + kys * kys > lowk_r2) &&
                     (kcut < 0 || (kx <= kcut && low_row(ky)));
  const float s = valid ? -(lamx[kx] + lamy[ky]) : 1.f;
  const float sq = tw_solve_tile(tile + col_t, wv + col_t, ac, meet, xm_s, TC, nz, col_t, upper, true, valid, s,
                                 -scale, spec + (valid ? col : 0), g.plane);
  if (sqn) {   // fixed-order CTA sum of the weighted squares (in the drained tile's shared memory)
    float v = (kx == 0 || kx == g.nxh - 1) ? sq : 2.f * sq;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    float* wsum = reinterpret_cast<float*>(meet);   // meet is free after the solve's last barrier
    __syncthreads();
    if ((t & 31) == 0) wsum[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += (double)wsum[w];
      sqn[blockIdx.x] = tot;
    }
  }
}

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------
// Columns per CTA: the requested width if its tile fits, else the largest of
// {64, 32, 16} whose tile fits about 56 KB (four CTAs per SM: while some load
// their tile, the others run their recurrences), else the largest that fits.
static int thomas_tile(int nz, size_t entry_bytes, int request) {
  if (request >= 16 && request <= 128 && (size_t)request * nz * entry_bytes + 16 <= 200 * 1024) return request;
  for (int tc = 64; tc >= 16; tc >>= 1)
    if ((size_t)tc * nz * entry_bytes + 16 <= 56 * 1024) return tc;
  for (int tc = 64; tc >= 16; tc >>= 1)
    if ((size_t)tc * nz * entry_bytes + 16 <= 200 * 1024) return tc;
  return 0;
}

// Paired FP32 column kernel (col_tile = 0, the default); *used = false when it does not fit.
template <typename TCm, bool ADJ>
static cudaError_t thomas_pair_launch(const ThomasArgs& A, const Geom& g, const Tables& tb, cudaStream_t st,
                                      bool* used) {
  *used = false;
  int tc = 0;
  for (int t = 32; t >= 16; t >>= 1) {   // 16 or 32 columns per row, tiles of at most ~64 KB
    const size_t sm = 2 * (size_t)g.nz * t * sizeof(float2) + (size_t)g.nz * t * sizeof(float);
    if (sm <= 64 * 1024) {
      tc = t;
      break;
    }
  }
  if (tc == 0) {
    const size_t sm16 = 2 * (size_t)g.nz * 16 * sizeof(float2) + (size_t)g.nz * 16 * sizeof(float);
    if (sm16 > 200 * 1024) return cudaSuccess;
    tc = 16;
  }
  size_t smem = 2 * (size_t)g.nz * tc * sizeof(float2) + (((size_t)g.nz * tc * sizeof(float) + 15) & ~(size_t)15) +
                ((size_t)g.nz + 1) * sizeof(float2) + 16;
  const size_t lowk_smem = lowk_smem_elems(g.nz) * sizeof(TCm);
  if (smem < lowk_smem) smem = lowk_smem;
  int box_rows = 1;
  for (int d = 256; d >= 1; --d)
    if (g.nz % d == 0) {
      box_rows = d;
      break;
    }
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  if (!encode_tensor_2d(&tm, A.spec, 8, (unsigned long long)g.plane, (unsigned long long)g.nz,
                        (unsigned long long)g.plane * sizeof(float2), (unsigned)tc, (unsigned)box_rows))
    return cudaSuccess;
  auto kern = k_thomas_pair<TCm, ADJ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int kx_chunks = (g.nxh + tc - 1) / tc;
  const int npairs = g.ny / 2 + 1;
  const long long nb = (long long)npairs * kx_chunks;
  const LowkArgs L{A.lowk_cols, A.n_lowk, tb.a_d, tb.c_d, tb.W_d, tb.lamx_d, tb.lamy_d, A.target_mean, A.scale,
                   A.singular00, A.lowk_inv};
  kern<<<(unsigned)(nb + A.n_lowk), tc, smem, st>>>((float2*)A.spec, g, tb.a_f, tb.c_f, tb.lamx_f, tb.lamy_f,
                                                    (float)A.scale, A.lowk_r2, A.done, A.stats, tm, box_rows,
                                                    kx_chunks, L);
  *used = true;
  return cudaGetLastError();
}

// Twisted FP32 column kernel for forward solves; *used = false when it does not fit.
template <typename TCm>
static cudaError_t thomas_tw_launch(const ThomasArgs& A, const Geom& g, const Tables& tb, int tc, cudaStream_t st,
                                    bool* used) {
  *used = false;
  size_t smem = (((size_t)g.nz * tc * (sizeof(float2) + sizeof(float)) + 15) & ~(size_t)15) +
                ((size_t)g.nz + 1) * sizeof(float2) + (size_t)tc * (sizeof(float4) + sizeof(float2)) + 16;
  const size_t lowk_smem = lowk_smem_elems(g.nz) * sizeof(TCm);
  if (smem < lowk_smem) smem = lowk_smem;
  if (smem > 200 * 1024) return cudaSuccess;
  int box_rows = 1;
  for (int d = 256; d >= 1; --d)
    if (g.nz % d == 0) {
      box_rows = d;
      break;
    }
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  if (!encode_tensor_2d(&tm, A.spec, 8, (unsigned long long)g.plane, (unsigned long long)g.nz,
                        (unsigned long long)g.plane * sizeof(float2), (unsigned)tc, (unsigned)box_rows))
    return cudaSuccess;
  auto kern = k_thomas_tw<TCm>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // every tile of the plane, or (kcut >= 0) the low rows' first ceil((kcut + 1)/tc) tiles
  const long long nb = A.kcut >= 0 ? (long long)(2 * A.kcut + 1) * ((A.kcut + tc) / tc) : (g.plane + tc - 1) / tc;
  if (A.kcut >= 0 && (2 * A.kcut + 1 > g.ny || A.kcut + tc > g.P || g.P % 16)) return cudaSuccess;
  const LowkArgs L{A.lowk_cols, A.n_lowk, tb.a_d, tb.c_d, tb.W_d, tb.lamx_d, tb.lamy_d, A.target_mean, A.scale,
                   A.singular00, A.lowk_inv};
  *used = true;
  if (A.sqnorm && A.sqnorm_blocks) *A.sqnorm_blocks = (int)(nb + A.n_lowk);
  return pdl_launch(kern, dim3((unsigned)(nb + A.n_lowk)), dim3(2 * tc), smem, st, (float2*)A.spec, g, tb.a_f, tb.c_f,
                    tb.lamx_f, tb.lamy_f, (float)A.scale, A.lowk_r2, A.done, A.stats, tm, box_rows, L, A.sqnorm,
                    A.kcut);
}

template <typename T, typename TCm, bool ADJ>
static cudaError_t thomas_launch(const ThomasArgs& A, const Geom& g, const Tables& tb, const T* a, const T* c,
                                 const T* lx, const T* ly, cudaStream_t st) {
  using C = typename CT<T>::t;
  if constexpr (sizeof(T) == 4) {
    if (!ADJ && (A.col_tile <= 2 || A.col_tile == 4)) {
      // twisted two-thread columns: 32 columns per CTA by default (col_tile 0 or 2), 16 (1) or 64 (4)
      const int tc = A.col_tile == 1 ? 16 : (A.col_tile == 4 ? 64 : 32);
      bool used = false;
      cudaError_t e = thomas_tw_launch<TCm>(A, g, tb, tc, st, &used);
      if (e != cudaSuccess || used) return e;
    }
    if (A.col_tile == 0 || A.col_tile == 3) {
      bool used = false;
      cudaError_t e = thomas_pair_launch<TCm, ADJ>(A, g, tb, st, &used);
      if (e != cudaSuccess || used) return e;
    }
  }
  const int tc = thomas_tile(g.nz, sizeof(C) + sizeof(T), A.col_tile);
  if (tc == 0) return cudaErrorInvalidValue;
  size_t smem = (((size_t)g.nz * tc * (sizeof(C) + sizeof(T)) + 15) & ~(size_t)15) + 16;
  const size_t lowk_smem = lowk_smem_elems(g.nz) * sizeof(TCm);
  if (smem < lowk_smem) smem = lowk_smem;
  const long long nb = (g.plane + tc - 1) / tc;
  auto kern = k_thomas<T, TCm, ADJ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the spectrum as a 2-D tensor: a level's ny*P entries per row, nz rows
  int box_rows = 1;
  for (int d = 256; d >= 1; --d)
    if (g.nz % d == 0) {
      box_rows = d;
      break;
    }
  constexpr int XM = sizeof(C) / 8;
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  const int use_tma = encode_tensor_2d(&tm, A.spec, 8, (unsigned long long)g.plane * XM, (unsigned long long)g.nz,
                                       (unsigned long long)g.plane * sizeof(C), (unsigned)(tc * XM),
                                       (unsigned)box_rows)
                          ? 1
                          : 0;
  const LowkArgs L{A.lowk_cols, A.n_lowk, tb.a_d, tb.c_d, tb.W_d, tb.lamx_d, tb.lamy_d, A.target_mean, A.scale,
                   A.singular00, A.lowk_inv};
  kern<<<(unsigned)(nb + A.n_lowk), tc, smem, st>>>((C*)A.spec, g, a, c, lx, ly, (T)A.scale, A.lowk_r2, A.done,
                                                   A.stats, tm, use_tma, box_rows, L);
  return cudaGetLastError();
}

cudaError_t launch_thomas(const ThomasArgs& A, const Geom& g, const Tables& tb, cudaStream_t st) {
  if (A.t_is_double)
    return A.adjoint ? thomas_launch<double, double, true>(A, g, tb, tb.a_d, tb.c_d, tb.lamx_d, tb.lamy_d, st)
                     : thomas_launch<double, double, false>(A, g, tb, tb.a_d, tb.c_d, tb.lamx_d, tb.lamy_d, st);
  if (A.lowk_double)
    return A.adjoint ? thomas_launch<float, double, true>(A, g, tb, tb.a_f, tb.c_f, tb.lamx_f, tb.lamy_f, st)
                     : thomas_launch<float, double, false>(A, g, tb, tb.a_f, tb.c_f, tb.lamx_f, tb.lamy_f, st);
  return A.adjoint ? thomas_launch<float, float, true>(A, g, tb, tb.a_f, tb.c_f, tb.lamx_f, tb.lamy_f, st)
                   : thomas_launch<float, float, false>(A, g, tb, tb.a_f, tb.c_f, tb.lamx_f, tb.lamy_f, st);
}

}  // namespace pgb
