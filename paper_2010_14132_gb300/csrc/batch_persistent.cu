// Persistent multi-domain solve of the mixed-precision path: many independent
// domains of uneven sizes, every step of every domain's direct solve and
// refinement (Section 2.1 transforms and column solves, Section 2.2's residual
// measure driving the sweeps) in ONE kernel launch.
//
// The launch works through a list of items (domain d, phase f, tile t), built on
// the host once per batch configuration.  The phases of one domain form a chain:
//   XF0  forward x transform of the source rows (first solve)
//   YF   forward y transform of strips of kx columns
//   COL  column solves: the low-|k| and singular columns (double, one per item)
//        and tiles of FP32 columns (twisted pivots, two threads per column)
//   YI   inverse y transform
//   XI0  inverse x transform, p0 stored (first solve), norm partials
//   CTL  refinement control of the pass (one item): stopping rule, done flag
//   then per sweep s: [QR: q rebuilt, s = 3] XR (forward x transform of the
//   double-float residual rows) YF COL [VER: verification, s >= 2] YI XIU
//   (inverse x with the update of q / p) CTL; and FIN (p = p0 + q when the
//   refinement ended on an iterate it had stored only as p0 + q).
// An item of phase f waits until every item of phase f - 1 of its domain is done
// (per-domain counters in the workspace, acquire loads, bounded waits); items of a
// domain that has converged return at once.  The list is phase-major across the
// domains (step f of every domain, largest domain first, then step f + 1), so a
// domain's next phase starts while other domains finish theirs.  CTAs take items in
// list order with an atomic ticket (the next ticket is taken while the current item
// runs).
//
// Progress: every item an item waits for precedes it in the list, so the earliest
// unfinished item belongs to a CTA whose own waits are all satisfied; no item
// waits on a later one, whatever the number of resident CTAs.  A wait that runs out
// of polls sets ERR_WAIT_TIMEOUT in the domain's Stats, skips its item and still
// counts it done, so the items behind it are not held up; the solve then reports
// POISSON_ERR_TIMEOUT.  Data produced inside the launch is read at L2 (ld.cg), not
// through the SMs' non-coherent L1.
//
// The arithmetic of every step is that of the single-domain kernels (same FFT
// stages, residual_value2, tw_solve_tile, lowk_column, control_decide,
// verify_decide); the transforms use plain loads instead of staged TMA rings.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "columns.cuh"
#include "xpass_common.cuh"

namespace pgb {
namespace {

constexpr int kBT = 256;                  // threads per CTA
constexpr long long kBSpin = 1LL << 22;   // polls of a dependency wait (100 ns sleep between polls)
constexpr int kBMaxPh = 40;               // phases of one domain's chain
constexpr size_t kBSmemCap = 110 * 1024;  // dynamic shared memory per CTA (two CTAs per SM)
constexpr int kBXPoints = 32768;          // grid points per x item (about)
constexpr int kBYPoints = 16384;          // complex entries per y item (about)
constexpr int kBEPairs = 32768;           // point pairs per elementwise item
constexpr int kBLowk = 32;                // low-|k| columns per column item (one thread each)

enum BPhase : int { BP_XF0 = 0, BP_XR, BP_YF, BP_YI, BP_COL, BP_XI0, BP_XIU, BP_CTL, BP_VER, BP_QR, BP_FIN };

struct BPh {
  int type, pass, items;
};

// One domain as the kernel sees it (device array, read-only during the launch).
struct BDom {
  Geom g;
  int N;                 // x half length nx/2
  int iso;               // dx == dy: the merged horizontal residual term
  float2 cx, cy;         // double-float 1/dx^2, 1/dy^2
  float scale_f;         // 1/(nx ny)
  double scale_d;
  int lowk_r2, n_lowk, singular00;
  const int2* lowk_cols;
  const double* lowk_inv;   // the plan's pivot table of the listed columns
  const float2* twx;
  const float2* twr;
  const float2* twy;
  const float* a_f;
  const float* c_f;
  const float2* a_ff;
  const float2* c_ff;
  const double* a_d;
  const double* c_d;
  const double* W_d;
  const float* lamx_f;
  const float* lamy_f;
  const double* lamx_d;
  const double* lamy_d;
  const double* floor_d;
  const double* S;
  double* p;
  float2* spec;
  float* p0;
  float* q;
  Stats* stats;
  double* xpart;   // [n_x][3]: delta^2, p^2, sum p of an inverse x item
  double* rpart;   // [n_x][2]: r^2, S^2 of a residual x item
  double* cpart;   // [n_lk + n_ct]: weighted sum |x|^2 of a column item
  unsigned* cnt;   // [nph]: items done per phase
  int max_sweeps, verify;
  double tol;
  int x_rows, n_x;                    // rows per x item, x items
  int y_tk, y_lv, n_ystrips, n_y;     // kx per strip, levels per y item, strips, y items
  int c_tc, n_ct;                     // columns per FP32 column tile, tiles
  int n_lk;                           // low-|k| column items (kBLowk columns each); COL items: n_lk + n_ct
  int e_pairs, n_e;                   // point pairs per elementwise item, items
  int nph;
  BPh ph[kBMaxPh];
};

__host__ __device__ constexpr int bx_elems(int N) { return N % 3 == 0 ? kE3 : 8; }
__host__ __device__ constexpr int by_elems(int ny) { return ny % 3 == 0 ? kE3 : 16; }
__host__ __device__ constexpr size_t b_align(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// fixed-order CTA sums (thread 0 stores)
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_sum_store(double* red, const double (&v)[K], double* out) {
  const int tid = threadIdx.x;
  __syncthreads();   // red may alias buffers the item used
#pragma unroll
  for (int k = 0; k < K; ++k) red[k * kBT + tid] = v[k];
  __syncthreads();
  for (int h = kBT / 2; h > 0; h >>= 1) {
    if (tid < h)
#pragma unroll
      for (int k = 0; k < K; ++k) red[k * kBT + tid] += red[k * kBT + tid + h];
    __syncthreads();
  }
  if (tid == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) __stcg(out + k, red[k * kBT]);
}

// ---------------------------------------------------------------------------
// x items: rows [r0, r1) of the domain, RB rows at a time (one row per nl threads)
// ---------------------------------------------------------------------------
__device__ __noinline__ void fill_xf0(const double* __restrict__ Srow, float2* line, int lane, int nl, int N) {
  const Swizzled sw{};
  const double2* s2 = reinterpret_cast<const double2*>(Srow);
  for (int e0 = lane; e0 < N; e0 += 4 * nl) {   // four loads in flight before the conversions
    double2 s[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = (e0 + j * nl < N) ? __ldg(s2 + e0 + j * nl) : make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (e0 + j * nl < N) line[sw(e0 + j * nl)] = make_float2(d2f_int(s[j].x), d2f_int(s[j].y));
  }
}

// The double-float residual of one row into the line (natural order, swizzled); returns the row's
// sums of r^2 (x, y) and S^2 (z, w) when valid.  store_p: the iterate p0 + q is also stored as the
// double output (the verification sweep's speculative copy).
// The double-float residual of one row into the line, one element at a time with the next one's
// operands in flight.
template <bool HAS_Q, bool ISO>
__device__ __noinline__ float4 fill_xr(const BDom& D, const ResCoef K, long long row, float2* line, int lane,
                                       int nl, bool valid, bool store_p) {
  const int N = D.N, NX = 2 * N;
  const Geom& g = D.g;
  const int k = (int)(row / g.ny), j = (int)(row - (long long)k * g.ny);
  const long long rn = row - j + (j + 1 == g.ny ? 0 : j + 1), rs = row - j + (j == 0 ? g.ny - 1 : j - 1);
  const bool has_dn = k > 0, has_up = k + 1 < g.nz;
  const float* prow = D.p0 + row * NX;
  const float2* p0c = reinterpret_cast<const float2*>(prow);
  const float2* p0n = reinterpret_cast<const float2*>(D.p0 + rn * NX);
  const float2* p0s = reinterpret_cast<const float2*>(D.p0 + rs * NX);
  const float2* p0d = reinterpret_cast<const float2*>(D.p0 + (has_dn ? row - g.ny : row) * NX);
  const float2* p0u = reinterpret_cast<const float2*>(D.p0 + (has_up ? row + g.ny : row) * NX);
  const float* qrow = D.q + row * NX;
  const float2* qc2 = reinterpret_cast<const float2*>(qrow);
  const float2* qn2 = reinterpret_cast<const float2*>(D.q + rn * NX);
  const float2* qs2 = reinterpret_cast<const float2*>(D.q + rs * NX);
  const float2* qd2 = reinterpret_cast<const float2*>(D.q + (has_dn ? row - g.ny : row) * NX);
  const float2* qu2 = reinterpret_cast<const float2*>(D.q + (has_up ? row + g.ny : row) * NX);
  const double2* Srow = reinterpret_cast<const double2*>(D.S + row * NX);
  double2* prow_out = reinterpret_cast<double2*>(D.p + row * NX);
  const Swizzled sw{};
  float2 racc = make_float2(0.f, 0.f), sacc = racc;
  // operands of one element pair; the next pair's are loaded before this pair's arithmetic
  struct Ops {
    float2 pc, pn, ps, pd, pu, qc, qn, qs, qd, qu;
    float pw, pe, qw, qe;
    double2 S;
  };
  auto load = [&](int e) {
    Ops o;
    o.pc = __ldcg(p0c + e);
    o.pw = __ldcg(prow + (e == 0 ? NX - 1 : 2 * e - 1));
    o.pe = __ldcg(prow + (e == N - 1 ? 0 : 2 * e + 2));
    o.pn = __ldcg(p0n + e);
    o.ps = __ldcg(p0s + e);
    o.pd = has_dn ? __ldcg(p0d + e) : o.pc;
    o.pu = has_up ? __ldcg(p0u + e) : make_float2(0.f, 0.f);
    o.qc = o.qn = o.qs = o.qd = o.qu = make_float2(0.f, 0.f);
    o.qw = o.qe = 0.f;
    if constexpr (HAS_Q) {
      o.qc = __ldcg(qc2 + e);
      o.qw = __ldcg(qrow + (e == 0 ? NX - 1 : 2 * e - 1));
      o.qe = __ldcg(qrow + (e == N - 1 ? 0 : 2 * e + 2));
      o.qn = __ldcg(qn2 + e);
      o.qs = __ldcg(qs2 + e);
      o.qd = has_dn ? __ldcg(qd2 + e) : o.qc;
      o.qu = has_up ? __ldcg(qu2 + e) : make_float2(0.f, 0.f);
    }
    o.S = __ldg(Srow + e);
    return o;
  };
  Ops nxt = load(lane);
  for (int e = lane; e < N; e += nl) {
    const Ops o = nxt;
    if (e + nl < N) nxt = load(e + nl);
    float2 Sh, Sl;
    d2ff_trunc(o.S.x, Sh.x, Sl.x);
    d2ff_trunc(o.S.y, Sh.y, Sl.y);
    // the pair's east neighbours are (pc.y, pe), its west neighbours (pw, pc.x)
    const float2 r = residual_value2<HAS_Q, ISO>(o.pc, make_float2(o.pc.y, o.pe), make_float2(o.pw, o.pc.x), o.pn,
                                                 o.ps, o.pd, o.pu, o.qc, make_float2(o.qc.y, o.qe),
                                                 make_float2(o.qw, o.qc.x), o.qn, o.qs, o.qd, o.qu, Sh, Sl, K);
    line[sw(e)] = r;
    if (valid) {
      racc = fma2(r, r, racc);
      sacc = fma2(Sh, Sh, sacc);
      if (HAS_Q && store_p) {
        float2 sp, tp;
        two_sum2(o.pc, o.qc, sp, tp);
        __stcg(prow_out + e, make_double2(ff2d_fast(sp.x, tp.x), ff2d_fast(sp.y, tp.y)));
      }
    }
  }
  return make_float4(racc.x, racc.y, sacc.x, sacc.y);
}

// Per-thread norm sums of an inverse x item: delta^2 (a0), p^2 (a1), double-float sum of p (sh, sl).
struct XAcc {
  float2 a0, a1, sh, sl;
};

// First solve: p0 stored (and p, as a double, when no sweep follows).
__device__ __noinline__ XAcc epi_p0(const BDom& D, long long row, const float2* line, int lane, int nl,
                                    bool store_p, XAcc A) {
  const int N = D.N;
  const Swizzled sw{};
  float2* p0r = reinterpret_cast<float2*>(D.p0 + row * 2 * N);
  double2* pr = reinterpret_cast<double2*>(D.p + row * 2 * N);
  for (int e = lane; e < N; e += nl) {
    const float2 z = line[sw(e)];
    __stcg(p0r + e, z);
    A.a1 = fma2(z, z, A.a1);
    float2 err;
    two_sum2(A.sh, z, A.sh, err);
    A.sl = add2(A.sl, err);
    if (store_p) __stcg(pr + e, make_double2(f2d_int(z.x), f2d_int(z.y)));
  }
  return A;
}

// Sweep: q + delta stored as the new q (q_out) and/or p = p0 + (q + delta) as a double (p_out).
__device__ __noinline__ XAcc epi_upd(const BDom& D, long long row, const float2* line, int lane, int nl,
                                     bool q_valid, bool q_out, bool p_out, XAcc A) {
  const int N = D.N;
  const Swizzled sw{};
  const float2* p0r = reinterpret_cast<const float2*>(D.p0 + row * 2 * N);
  float2* qr = reinterpret_cast<float2*>(D.q + row * 2 * N);
  double2* pr = reinterpret_cast<double2*>(D.p + row * 2 * N);
  float2 p0n = __ldcg(p0r + lane), qvn = q_valid ? __ldcg(qr + lane) : make_float2(0.f, 0.f);
  for (int e = lane; e < N; e += nl) {
    const float2 z = line[sw(e)];
    const float2 p0v = p0n, qv = qvn;
    if (e + nl < N) {   // the next element's operands, in flight during this one's arithmetic
      p0n = __ldcg(p0r + e + nl);
      if (q_valid) qvn = __ldcg(qr + e + nl);
    }
    const float2 qn = add2(z, qv);
    if (q_out) __stcg(qr + e, qn);
    float2 sp, tp;
    two_sum2(p0v, qn, sp, tp);
    if (p_out) __stcg(pr + e, make_double2(ff2d_fast(sp.x, tp.x), ff2d_fast(sp.y, tp.y)));
    A.a0 = fma2(z, z, A.a0);
    A.a1 = fma2(sp, sp, A.a1);
    float2 err;
    two_sum2(A.sh, sp, A.sh, err);
    A.sl = add2(A.sl, add2(err, tp));
  }
  return A;
}

template <int N, int E>
__device__ void item_x(const BDom& D, int type, int pass, int sub, unsigned char* sm) {
  constexpr int nl = N / E, RB = kBT / nl, LS = swizzled_stride(N);
  static_assert(nl <= 32 && kBT % nl == 0, "an x line is transformed inside one warp");
  float2* tw_s = reinterpret_cast<float2*>(sm);
  float2* twr_s = tw_s + N;
  float2* lines = twr_s + N + 2;
  const int tid = threadIdx.x, lane = tid % nl, ty = tid / nl;
  st_build_twiddles<N, E>(tw_s, D.twx, tid, kBT);
  for (int t = tid; t <= N; t += kBT) twr_s[t] = __ldg(&D.twr[t]);
  const Geom& g = D.g;
  const long long rows = (long long)g.ny * g.nz;
  const long long r0 = (long long)sub * D.x_rows, r1 = min(rows, r0 + (long long)D.x_rows);
  float2* line = lines + (size_t)ty * LS;
  const LineSync sync{1 + ty, nl};
  const Swizzled sw{};
  const bool fwd = type == BP_XF0 || type == BP_XR;
  const bool has_q = pass > 1;
  const bool store_p = type == BP_XR ? (D.verify && pass == 2) : (type == BP_XI0 && D.max_sweeps == 0);
  const bool last_allowed = pass == D.max_sweeps;
  const bool q_out = pass == 1 && !last_allowed;
  const float2 mu = type == BP_XR ? __ldcg(&D.stats->mu_ff) : make_float2(0.f, 0.f);
  float4 rs = make_float4(0.f, 0.f, 0.f, 0.f);
  XAcc A{};
  __syncthreads();
  for (long long rb = r0; rb < r1; rb += RB) {
    const long long row = rb + ty;
    const bool valid = row < r1;
    const long long rr = valid ? row : r0;   // addressing stays inside the field
    if (fwd) {
      if (type == BP_XF0) {
        fill_xf0(D.S + rr * 2 * N, line, lane, nl, N);
      } else {
        const int k = (int)(rr / g.ny);
        const ResCoef K = res_coef(D.cx, D.cy, __ldg(&D.a_ff[k]), __ldg(&D.c_ff[k]), mu);
        float4 t;
        if (has_q) t = D.iso ? fill_xr<true, true>(D, K, rr, line, lane, nl, valid, store_p)
                             : fill_xr<true, false>(D, K, rr, line, lane, nl, valid, store_p);
        else t = D.iso ? fill_xr<false, true>(D, K, rr, line, lane, nl, valid, false)
                       : fill_xr<false, false>(D, K, rr, line, lane, nl, valid, false);
        rs.x += t.x;
        rs.y += t.y;
        rs.z += t.z;
        rs.w += t.w;
      }
      sync();
      float2 v[E];
#pragma unroll
      for (int i = 0; i < E; ++i) v[i] = line[sw(st_in_index<N, E, 0>(lane, i))];
      sync();   // every input is read before the transform overwrites the line
      const float2* fin = st_fft_inplace<N, E, -1, false, float>(v, line, sw, lane, tw_s, sync);
      r2c_unpack_store<N, E>(fin, twr_s, D.spec + rr * g.P, lane, valid);
    } else {
      // C2R: each first-stage input from the bins X_m and X_{N-m} (self-conjugate bins real)
      const float2* X = D.spec + rr * g.P;
      float2 v[E];
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int m = st_in_index<N, E, 0>(lane, i);
        float2 xk = __ldcg(X + m);
        float2 xc = cconj(__ldcg(X + N - m));
        if (m == 0) {
          xk.y = 0.f;
          xc.y = 0.f;
        }
        const float2 ev = cadd(xk, xc);
        const float2 od = cmul(csub(xk, xc), cconj(twr_s[m]));   // * exp(+2 pi i m/n)
        v[i] = make_float2(ev.x - od.y, ev.y + od.x);            // ev + i od
      }
      const float2* fin = st_fft_inplace<N, E, +1, false, float>(v, line, sw, lane, tw_s, sync);
      if (valid) {
        if (type == BP_XI0) A = epi_p0(D, row, fin, lane, nl, store_p, A);
        else A = epi_upd(D, row, fin, lane, nl, pass > 1, q_out, !q_out, A);
      }
    }
    sync();   // the line is refilled by the next group
  }
  double* red = reinterpret_cast<double*>(sm);
  if (type == BP_XR) {
    const double v[2] = {(double)rs.x + (double)rs.y, (double)rs.z + (double)rs.w};
    block_sum_store<2>(red, v, D.rpart + 2 * (size_t)sub);
  } else if (type != BP_XF0) {
    const double v[3] = {(double)(A.a0.x + A.a0.y), (double)(A.a1.x + A.a1.y),
                         (f2d_int(A.sh.x) + f2d_int(A.sl.x)) + (f2d_int(A.sh.y) + f2d_int(A.sl.y))};
    block_sum_store<3>(red, v, D.xpart + 3 * (size_t)sub);
  }
}

// ---------------------------------------------------------------------------
// y items: TK consecutive kx of y_lv levels; one column per ny/E threads
// ---------------------------------------------------------------------------
template <int TK> struct SwTileB {
  __device__ __forceinline__ int operator()(int idx) const { return (idx ^ ((idx >> 4) & 15)) * TK; }
};

template <int NY, int E, int SIGN>
__device__ void item_y(const BDom& D, int sub, unsigned char* sm) {
  constexpr int TK = kBT * E / NY;
  static_assert(TK * (NY / E) == kBT, "a y item uses every thread");
  float2* tw_s = reinterpret_cast<float2*>(sm);
  float2* tile = tw_s + ((NY + 1) & ~1);
  const int tid = threadIdx.x;
  st_build_twiddles<NY, E>(tw_s, D.twy, tid, kBT);
  const Geom& g = D.g;
  const int strip = sub % D.n_ystrips, lv0 = (sub / D.n_ystrips) * D.y_lv, lv1 = min(g.nz, lv0 + D.y_lv);
  const int l = tid % TK, lane = tid / TK, kx = strip * TK + l;
  const bool ok = kx < g.nxh;
  for (int k = lv0; k < lv1; ++k) {
    float2* col = D.spec + (long long)k * g.plane + (ok ? kx : 0);
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i)
      v[i] = ok ? __ldcg(col + (long long)st_in_index<NY, E, 0>(lane, i) * g.P) : make_float2(0.f, 0.f);
    __syncthreads();   // the twiddles are built and the previous level's tile reads are done
    st_fft_inplace<NY, E, SIGN, true, float>(v, tile + l, SwTileB<TK>{}, lane, tw_s, SyncBlock());
    if (ok)
#pragma unroll
      for (int i = 0; i < E; ++i) __stcg(col + (long long)st_out_index<NY, E>(lane, i) * g.P, v[i]);
  }
}

// ---------------------------------------------------------------------------
// column items: kBLowk listed low-|k| columns (double, one thread each, the
// recurrence of lowk_column), or a tile of c_tc consecutive plane entries (FP32,
// two threads per column); the weighted sum of |x|^2 of the solved columns goes
// to the item's slot (the verification's Parseval norm)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t col_tile_bytes(int nz, int tc) {
  return b_align((size_t)nz * tc * 12, 16) + (size_t)(nz + (nz & 1)) * 8 + (size_t)tc * 24;
}
__host__ __device__ constexpr size_t lowk_item_bytes(int nz) {
  return ((size_t)3 * nz + (size_t)3 * nz * kBLowk + 6 * kBLowk) * 8;
}

__device__ void item_lowk(const BDom& D, int pass, int sub, unsigned char* sm) {
  const Geom& g = D.g;
  const int nz = g.nz, tid = threadIdx.x, j0 = sub * kBLowk, ncol = min(kBLowk, D.n_lowk - j0);
  double* a = reinterpret_cast<double*>(sm);
  double* c = a + nz;
  double* W = c + nz;
  double* zx = W + nz;                  // [nz][kBLowk]
  double* zy = zx + nz * kBLowk;
  double* w = zy + nz * kBLowk;
  double* red = w + nz * kBLowk;        // [kBLowk][5]
  double* sq = red + 5 * kBLowk;        // [kBLowk]
  const double* target_mean = pass > 0 ? &D.stats->pmean : nullptr;
  for (int k = tid; k < nz; k += kBT) {
    a[k] = __ldg(&D.a_d[k]);
    c[k] = __ldg(&D.c_d[k]);
    W[k] = __ldg(&D.W_d[k]);
  }
  for (int i = tid; i < nz * kBLowk; i += kBT) {
    const int k = i / kBLowk, j = i - k * kBLowk;
    if (j < ncol) {
      const int2 ck = __ldg(&D.lowk_cols[j0 + j]);
      const float2 v = __ldcg(D.spec + (long long)k * g.plane + (long long)ck.y * g.P + ck.x);
      zx[i] = (double)v.x;
      zy[i] = (double)v.y;
      if (D.lowk_inv) w[i] = __ldg(D.lowk_inv + (size_t)(j0 + j) * nz + k);   // the column's pivot table
    }
  }
  __syncthreads();
  if (tid < ncol) {
    const int2 ck = __ldg(&D.lowk_cols[j0 + tid]);
    const bool singular = D.singular00 && ck.x == 0 && ck.y == 0;
    lowk_recurrence<double, false>(zx + tid, zy + tid, w + tid, kBLowk, a, c, W, nz, ck.x, ck.y, singular, D.lamx_d,
                                   D.lamy_d, D.scale_d, target_mean, D.stats, red + 5 * tid, sq + tid,
                                   D.lowk_inv != nullptr);
  }
  __syncthreads();
  for (int i = tid; i < nz * kBLowk; i += kBT) {
    const int k = i / kBLowk, j = i - k * kBLowk;
    if (j < ncol) {
      const int2 ck = __ldg(&D.lowk_cols[j0 + j]);
      double ox = zx[i], oy = zy[i];
      if (D.singular00 && ck.x == 0 && ck.y == 0) {
        ox -= red[5 * j];
        oy -= red[5 * j + 1];
      }
      D.spec[(long long)k * g.plane + (long long)ck.y * g.P + ck.x] = make_float2((float)ox, (float)oy);
    }
  }
  if (tid == 0) {
    double tot = 0.0;
    for (int j = 0; j < ncol; ++j) {
      const int kx = __ldg(&D.lowk_cols[j0 + j]).x;
      tot += (kx == 0 || kx == g.nxh - 1 ? 1.0 : 2.0) * sq[j];
    }
    __stcg(&D.cpart[sub], tot);
  }
}

__device__ void item_col(const BDom& D, int pass, int sub, unsigned char* sm) {
  const Geom& g = D.g;
  const int tid = threadIdx.x;
  if (sub < D.n_lk) {
    item_lowk(D, pass, sub, sm);
    return;
  }
  const int TC = D.c_tc, nz = g.nz;
  float2* tile = reinterpret_cast<float2*>(sm);
  float* wv = reinterpret_cast<float*>(tile + (size_t)nz * TC);
  float2* ac = reinterpret_cast<float2*>(sm + b_align((size_t)nz * TC * 12, 16));
  float4* meet = reinterpret_cast<float4*>(ac + nz + (nz & 1));
  float2* xm_s = reinterpret_cast<float2*>(meet + TC);
  const long long c0 = (long long)(sub - D.n_lk) * TC;
  for (int k = tid; k < nz; k += kBT) ac[k] = make_float2(__ldg(&D.a_f[k]), __ldg(&D.c_f[k]));
  for (int i0 = tid; i0 < nz * TC; i0 += 8 * kBT) {   // eight loads in flight per thread
    float2 r[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = i0 + j * kBT, k = i / TC, c = i - k * TC;
      r[j] = (i < nz * TC && c0 + c < g.plane) ? __ldcg(D.spec + (long long)k * g.plane + c0 + c)
                                               : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (i0 + j * kBT < nz * TC) tile[i0 + j * kBT] = r[j];
  }
  __syncthreads();
  const bool part = tid < 2 * TC;
  const int col_t = tid % TC, upper = tid / TC;
  const long long col = c0 + col_t;
  const int ky = (int)(col / g.P), kx = (int)(col - (long long)ky * g.P);
  const int kys = signed_ky(ky, g.ny);
  const bool valid = part && col < g.plane && kx < g.nxh && (kx * kx + kys * kys > D.lowk_r2);
  const float s = valid ? -(__ldg(&D.lamx_f[kx]) + __ldg(&D.lamy_f[ky])) : 1.f;
  const float sqf = tw_solve_tile(tile + col_t, wv + col_t, ac, meet, xm_s, TC, nz, col_t, upper, part, valid, s,
                                  -D.scale_f, D.spec + (valid ? col : 0), g.plane);
  float v = (kx == 0 || kx == g.nxh - 1) ? sqf : 2.f * sqf;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  float* wsum = reinterpret_cast<float*>(meet);   // free after the solve's last barrier
  __syncthreads();
  if ((tid & 31) == 0) wsum[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < kBT / 32; ++w) tot += (double)wsum[w];
    __stcg(&D.cpart[sub], tot);
  }
}

// ---------------------------------------------------------------------------
// control and verification items (one per pass): the domain's Stats are brought
// into shared memory at L2, updated by one thread with the single-domain rules,
// and written back (every field before err, which other items may set at any time)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void stats_load(Stats* ls, const Stats* gs) {
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(gs);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(ls);
  for (int i = threadIdx.x; i < (int)(sizeof(Stats) / 8); i += kBT) dst[i] = __ldcg(src + i);
}
__device__ __forceinline__ void stats_store(Stats* gs, const Stats* ls) {
  constexpr int nw = (int)(offsetof(Stats, err) / 4);
  const unsigned* src = reinterpret_cast<const unsigned*>(ls);
  unsigned* dst = reinterpret_cast<unsigned*>(gs);
  for (int i = threadIdx.x; i < nw; i += kBT) __stcg(dst + i, src[i]);
}

__device__ void item_ctl(const BDom& D, int type, int pass, unsigned char* sm) {
  Stats* ls = reinterpret_cast<Stats*>(sm);
  double* red = reinterpret_cast<double*>(sm + b_align(sizeof(Stats), 128));
  const int tid = threadIdx.x;
  stats_load(ls, D.stats);
  double v[5] = {0, 0, 0, 0, 0};
  if (type == BP_CTL) {
    for (int i = tid; i < D.n_x; i += kBT) {
      v[0] += __ldcg(&D.xpart[3 * (size_t)i]);
      v[1] += __ldcg(&D.xpart[3 * (size_t)i + 1]);
      v[2] += __ldcg(&D.xpart[3 * (size_t)i + 2]);
    }
  } else {
    for (int i = tid; i < D.n_lk + D.n_ct; i += kBT) v[0] += __ldcg(&D.cpart[i]);
  }
  if (pass > 0)
    for (int i = tid; i < D.n_x; i += kBT) {
      v[3] += __ldcg(&D.rpart[2 * (size_t)i]);
      v[4] += __ldcg(&D.rpart[2 * (size_t)i + 1]);
    }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 5; ++k) red[k * kBT + tid] = v[k];
  __syncthreads();
  for (int h = kBT / 2; h > 0; h >>= 1) {
    if (tid < h)
#pragma unroll
      for (int k = 0; k < 5; ++k) red[k * kBT + tid] += red[k * kBT + tid + h];
    __syncthreads();
  }
  if (tid == 0) {
    const double floor = __ldg(D.floor_d);
    if (type == BP_CTL) {
      const int wrote_p = pass == 0 ? (D.max_sweeps == 0) : !(pass == 1 && pass < D.max_sweeps);
      control_decide(ls, red[0], red[kBT], red[2 * kBT], red[3 * kBT], red[4 * kBT], pass, D.max_sweeps, D.tol,
                     D.g.N, wrote_p, floor);
    } else {
      verify_decide(ls, (double)D.g.nx * D.g.ny * red[0], red[3 * kBT], red[4 * kBT], pass, D.tol, floor,
                    pass == 2 ? 1 : 0);
    }
  }
  __syncthreads();
  stats_store(D.stats, ls);
}

// ---------------------------------------------------------------------------
// elementwise items: q rebuilt from the double iterate (before sweep 3) and the
// final p = p0 + q (when the refinement ended on an iterate stored as p0 + q)
// ---------------------------------------------------------------------------
__device__ void item_elem(const BDom& D, int type, int sub) {
  const long long npairs = D.g.N / 2;
  const long long i0 = (long long)sub * D.e_pairs, i1 = min(npairs, i0 + (long long)D.e_pairs);
  const float2* p0 = reinterpret_cast<const float2*>(D.p0);
  float2* q = reinterpret_cast<float2*>(D.q);
  double2* p = reinterpret_cast<double2*>(D.p);
  if (type == BP_FIN) {
    if (!__ldcg(&D.stats->need_final)) return;
    for (long long i = i0 + threadIdx.x; i < i1; i += kBT) __stcg(p + i, finalize_pair(__ldcg(p0 + i), __ldcg(q + i)));
  } else {
    for (long long i = i0 + threadIdx.x; i < i1; i += kBT) __stcg(q + i, q_rebuild_pair(__ldcg(p + i), __ldcg(p0 + i)));
  }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT, 2) k_batch(const BDom* __restrict__ doms, const uint2* __restrict__ items,
                                                  int nitems, unsigned* __restrict__ ticket, int stall_dom) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint2 s_item;
  __shared__ int s_skip;
  const int tid = threadIdx.x;
  unsigned next = 0;
  if (tid == 0) next = atomicAdd(ticket, 1u);
  for (;;) {
    if (tid == 0) {
      const unsigned t = next;
      uint2 it = make_uint2(0xffffffffu, 0u);
      int skip = 0;
      if (t < (unsigned)nitems) {
        it = __ldg(&items[t]);
        next = atomicAdd(ticket, 1u);   // the next item's ticket, taken while this one runs
        const int d = (int)(it.x & 0xffffu), f = (int)(it.x >> 16);
        const BDom& D = doms[d];
        if (f > 0) {
          unsigned target = (unsigned)D.ph[f - 1].items;
          // test hook: the first control item of domain stall_dom waits for one item more than exists
          if (d == stall_dom && D.ph[f].type == BP_CTL && D.ph[f].pass == 0) target += 1u;
          long long i = 0;
          while (ld_acquire_gpu(&D.cnt[f - 1]) < target && i < kBSpin) {
            __nanosleep(100);
            ++i;
          }
          if (i == kBSpin) {
            atomicOr(&D.stats->err, (unsigned)ERR_WAIT_TIMEOUT);
            skip = 1;
          }
        }
        // a converged domain's remaining items return at once (the final copy excepted)
        if (!skip && D.ph[f].type != BP_FIN && __ldcg(&D.stats->done)) skip = 1;
      }
      s_item = it;
      s_skip = skip;
    }
    __syncthreads();
    const uint2 it = s_item;
    const int skip = s_skip;
    if (it.x == 0xffffffffu) break;
    const int d = (int)(it.x & 0xffffu), f = (int)(it.x >> 16), sub = (int)it.y;
    const BDom& D = doms[d];
    if (!skip) {
      const int type = D.ph[f].type, pass = D.ph[f].pass;
      switch (type) {
        case BP_XF0:
        case BP_XR:
        case BP_XI0:
        case BP_XIU:
          switch (D.N) {
            case 32: item_x<32, bx_elems(32)>(D, type, pass, sub, sm); break;
            case 64: item_x<64, bx_elems(64)>(D, type, pass, sub, sm); break;
            case 128: item_x<128, bx_elems(128)>(D, type, pass, sub, sm); break;
            case 192: item_x<192, bx_elems(192)>(D, type, pass, sub, sm); break;
            case 256: item_x<256, bx_elems(256)>(D, type, pass, sub, sm); break;
            default: break;
          }
          break;
        case BP_YF:
        case BP_YI: {
          const bool fw = type == BP_YF;
          switch (D.g.ny) {
            case 64: fw ? item_y<64, by_elems(64), -1>(D, sub, sm) : item_y<64, by_elems(64), 1>(D, sub, sm); break;
            case 128: fw ? item_y<128, by_elems(128), -1>(D, sub, sm) : item_y<128, by_elems(128), 1>(D, sub, sm); break;
            case 256: fw ? item_y<256, by_elems(256), -1>(D, sub, sm) : item_y<256, by_elems(256), 1>(D, sub, sm); break;
            case 384: fw ? item_y<384, by_elems(384), -1>(D, sub, sm) : item_y<384, by_elems(384), 1>(D, sub, sm); break;
            case 512: fw ? item_y<512, by_elems(512), -1>(D, sub, sm) : item_y<512, by_elems(512), 1>(D, sub, sm); break;
            default: break;
          }
        } break;
        case BP_COL: item_col(D, pass, sub, sm); break;
        case BP_CTL:
        case BP_VER: item_ctl(D, type, pass, sm); break;
        case BP_QR:
        case BP_FIN: item_elem(D, type, sub); break;
        default: break;
      }
    }
    __syncthreads();   // every write of the item precedes the counter release
    if (tid == 0) {
      __threadfence();
      atomicAdd(&D.cnt[f], 1u);
    }
  }
}

// Zero every domain's Stats and phase counters and the ticket (block d: domain d).
__global__ void __launch_bounds__(kBT) k_batch_init(const BDom* __restrict__ doms, unsigned* __restrict__ ticket) {
  const BDom& D = doms[blockIdx.x];
  unsigned* st = reinterpret_cast<unsigned*>(D.stats);
  for (int i = threadIdx.x; i < (int)(sizeof(Stats) / 4); i += kBT) st[i] = 0u;
  for (int i = threadIdx.x; i < D.nph; i += kBT) D.cnt[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0u;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct BGeo {
  int N, Ex, nl, RB, x_rows, n_x, Ey, y_tk, n_ystrips, y_lv, n_y, c_tc, n_ct, n_lk, e_pairs, n_e;
  size_t smem;
};

BGeo b_geometry(const BatchDomIn& in) {
  BGeo b{};
  const Geom& g = in.g;
  b.N = g.nx / 2;
  b.Ex = bx_elems(b.N);
  b.nl = b.N / b.Ex;
  b.RB = kBT / b.nl;
  const int reps = std::max(1, kBXPoints / (b.RB * g.nx));
  b.x_rows = b.RB * reps;
  const long long rows = (long long)g.ny * g.nz;
  b.n_x = (int)((rows + b.x_rows - 1) / b.x_rows);
  b.Ey = by_elems(g.ny);
  b.y_tk = kBT * b.Ey / g.ny;
  b.n_ystrips = (g.nxh + b.y_tk - 1) / b.y_tk;
  b.y_lv = std::max(1, kBYPoints / (g.ny * b.y_tk));
  b.n_y = b.n_ystrips * ((g.nz + b.y_lv - 1) / b.y_lv);
  b.c_tc = 32;
  for (int tc = 128; tc >= 32; tc >>= 1)
    if (col_tile_bytes(g.nz, tc) <= kBSmemCap) {
      b.c_tc = tc;
      break;
    }
  b.n_ct = (int)((g.plane + b.c_tc - 1) / b.c_tc);
  b.n_lk = (in.n_lowk + kBLowk - 1) / kBLowk;
  b.e_pairs = kBEPairs;
  b.n_e = (int)((g.N / 2 + b.e_pairs - 1) / b.e_pairs);
  const size_t sx = (size_t)(2 * b.N + 2) * 8 + (size_t)b.RB * swizzled_stride(b.N) * 8;
  const size_t sy = (size_t)((g.ny + 1) & ~1) * 8 + (size_t)g.ny * b.y_tk * 8;
  const size_t sc = col_tile_bytes(g.nz, b.c_tc);
  const size_t sl = lowk_item_bytes(g.nz);
  const size_t sctl = b_align(sizeof(Stats), 128) + 5 * (size_t)kBT * 8;
  b.smem = std::max({sx, sy, sc, sl, sctl, (size_t)3 * kBT * 8});
  return b;
}

std::vector<BPh> b_chain(const BatchDomIn& in, const BGeo& b) {
  std::vector<BPh> ph;
  const int ncol = b.n_lk + b.n_ct;
  ph.push_back({BP_XF0, 0, b.n_x});
  ph.push_back({BP_YF, 0, b.n_y});
  ph.push_back({BP_COL, 0, ncol});
  ph.push_back({BP_YI, 0, b.n_y});
  ph.push_back({BP_XI0, 0, b.n_x});
  ph.push_back({BP_CTL, 0, 1});
  for (int s = 1; s <= in.max_sweeps; ++s) {
    if (s >= 3) ph.push_back({BP_QR, s, b.n_e});
    ph.push_back({BP_XR, s, b.n_x});
    ph.push_back({BP_YF, s, b.n_y});
    ph.push_back({BP_COL, s, ncol});
    if (in.verify && s >= 2) ph.push_back({BP_VER, s, 1});
    ph.push_back({BP_YI, s, b.n_y});
    ph.push_back({BP_XIU, s, b.n_x});
    ph.push_back({BP_CTL, s, 1});
  }
  if (in.max_sweeps >= 2) ph.push_back({BP_FIN, 0, b.n_e});
  return ph;
}

// Scratch of one domain: counters, then the x, residual and column partial sums.
size_t b_dom_scratch(const BatchDomIn& in, const BGeo& b) {
  return b_align(kBMaxPh * 4, 256) + b_align((size_t)3 * b.n_x * 8, 256) + b_align((size_t)2 * b.n_x * 8, 256) +
         b_align((size_t)(b.n_lk + b.n_ct) * 8, 256);
}

}  // namespace

bool batch_persistent_supported(int nx, int ny, int nz) {
  const int N = nx / 2;
  const bool okx = nx % 2 == 0 && (N == 32 || N == 64 || N == 128 || N == 192 || N == 256);
  const bool oky = ny == 64 || ny == 128 || ny == 256 || ny == 384 || ny == 512;
  return okx && oky && nz >= 2 && nz <= 128;
}

size_t batch_persistent_scratch_bytes(const std::vector<BatchDomIn>& d) {
  size_t off = 256;   // the ticket
  for (const auto& in : d) off += b_dom_scratch(in, b_geometry(in));
  return off;
}

void batch_persistent_free(BatchPersistent* bp) {
  if (bp->doms) cudaFree(bp->doms);
  if (bp->items) cudaFree(bp->items);
  *bp = BatchPersistent{};
}

int batch_persistent_build(BatchPersistent* bp, const std::vector<BatchDomIn>& d, char* scratch, int stall_dom) {
  batch_persistent_free(bp);
  const int n = (int)d.size();
  if (n <= 0 || n > 0xffff) return -1;
  std::vector<BDom> hd(n);
  std::vector<int> nph(n);
  size_t smem = 0, off = 256;
  for (int i = 0; i < n; ++i) {
    const BatchDomIn& in = d[i];
    if (!batch_persistent_supported(in.g.nx, in.g.ny, in.g.nz)) return -1;
    const BGeo b = b_geometry(in);
    const std::vector<BPh> ch = b_chain(in, b);
    if ((int)ch.size() > kBMaxPh) return -1;
    BDom& D = hd[i];
    std::memset(&D, 0, sizeof(D));
    D.g = in.g;
    D.N = b.N;
    D.iso = (in.cx.x == in.cy.x && in.cx.y == in.cy.y) ? 1 : 0;
    D.cx = in.cx;
    D.cy = in.cy;
    D.scale_d = 1.0 / ((double)in.g.nx * in.g.ny);
    D.scale_f = (float)D.scale_d;
    D.lowk_r2 = in.lowk_r2;
    D.n_lowk = in.n_lowk;
    D.singular00 = in.singular00;
    D.lowk_cols = in.lowk_cols;
    D.lowk_inv = in.lowk_inv;
    const Tables& tb = *in.tb;
    D.twx = tb.twx_f;
    D.twr = tb.twr_f;
    D.twy = tb.twy_f;
    D.a_f = tb.a_f;
    D.c_f = tb.c_f;
    D.a_ff = tb.a_ff;
    D.c_ff = tb.c_ff;
    D.a_d = tb.a_d;
    D.c_d = tb.c_d;
    D.W_d = tb.W_d;
    D.lamx_f = tb.lamx_f;
    D.lamy_f = tb.lamy_f;
    D.lamx_d = tb.lamx_d;
    D.lamy_d = tb.lamy_d;
    D.floor_d = tb.floor_d;
    D.S = in.S;
    D.p = in.p;
    D.spec = in.spec;
    D.p0 = in.p0;
    D.q = in.q;
    D.stats = in.stats;
    char* base = scratch + off;
    size_t o = 0;
    D.cnt = reinterpret_cast<unsigned*>(base + o);
    o += b_align(kBMaxPh * 4, 256);
    D.xpart = reinterpret_cast<double*>(base + o);
    o += b_align((size_t)3 * b.n_x * 8, 256);
    D.rpart = reinterpret_cast<double*>(base + o);
    o += b_align((size_t)2 * b.n_x * 8, 256);
    D.cpart = reinterpret_cast<double*>(base + o);
    off += b_dom_scratch(in, b);
    D.max_sweeps = in.max_sweeps;
    D.verify = in.verify;
    D.tol = in.tol;
    D.x_rows = b.x_rows;
    D.n_x = b.n_x;
    D.y_tk = b.y_tk;
    D.y_lv = b.y_lv;
    D.n_ystrips = b.n_ystrips;
    D.n_y = b.n_y;
    D.c_tc = b.c_tc;
    D.n_ct = b.n_ct;
    D.n_lk = b.n_lk;
    D.e_pairs = b.e_pairs;
    D.n_e = b.n_e;
    D.nph = (int)ch.size();
    for (int f = 0; f < D.nph; ++f) D.ph[f] = ch[f];
    nph[i] = D.nph;
    smem = std::max(smem, b.smem);
  }
  if (smem > kBSmemCap) return -1;
  // phase-major list, largest domains first within a step
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hd[x].g.N > hd[y].g.N; });
  const int steps = *std::max_element(nph.begin(), nph.end());
  std::vector<uint2> items;
  for (int f = 0; f < steps; ++f)
    for (int i : order)
      if (f < nph[i])
        for (int t = 0; t < hd[i].ph[f].items; ++t)
          items.push_back(make_uint2((unsigned)i | ((unsigned)f << 16), (unsigned)t));
  cudaError_t e = cudaMalloc(&bp->doms, sizeof(BDom) * n);
  if (e == cudaSuccess) e = cudaMalloc(&bp->items, sizeof(uint2) * items.size());
  if (e == cudaSuccess) e = cudaMemcpy(bp->doms, hd.data(), sizeof(BDom) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bp->items, items.data(), sizeof(uint2) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    batch_persistent_free(bp);
    return -2;
  }
  bp->n = n;
  bp->nitems = (int)items.size();
  bp->smem = b_align(smem, 128);
  bp->ticket = reinterpret_cast<unsigned*>(scratch);
  bp->stall_dom = stall_dom;
  return 0;
}

cudaError_t batch_persistent_launch(const BatchPersistent& bp, cudaStream_t st) {
  if (!bp.doms || bp.nitems <= 0) return cudaErrorInvalidValue;
  static std::mutex mu;
  static int per_sm = -1;
  static size_t granted = 0;
  int ctas = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (per_sm < 0 || granted < bp.smem) {
      cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bp.smem);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kBT, bp.smem);
      if (e != cudaSuccess) return e;
      granted = bp.smem;
    }
    ctas = per_sm;
  }
  if (ctas < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)ctas * sm_count();
  if (grid > bp.nitems) grid = bp.nitems;
  k_batch_init<<<bp.n, kBT, 0, st>>>(reinterpret_cast<const BDom*>(bp.doms), bp.ticket);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_batch<<<(unsigned)grid, kBT, bp.smem, st>>>(reinterpret_cast<const BDom*>(bp.doms),
                                                reinterpret_cast<const uint2*>(bp.items), bp.nitems, bp.ticket,
                                                bp.stall_dom);
  return cudaGetLastError();
}

}  // namespace pgb
