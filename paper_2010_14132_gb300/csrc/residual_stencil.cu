// Refinement residual of a sweep as its own pass: r = S - mu_W - L (p0 + q), the
// 7-point cell-centred operator of the solve (the relative-residual measure of
// Section 2.2 applied to the direct solve's iterate), stored as float for the
// forward x-pass that follows.
//
// One CTA owns a tile of 64 x points (32 lanes, two points each) by 8 rows (one
// warp per row) and marches up ZC levels.  Each thread keeps its two points'
// values of p0 and q at the levels below, at and above the current one in
// registers (loaded one level ahead), so every value is read from memory once;
// the x neighbours come from the adjacent lanes by warp shuffles (the tile's edge
// points by two extra loads), the y neighbours from the rows the other warps
// publish in shared memory (the two halo rows by two extra row loads), one block
// barrier per level.  The arithmetic is residual_value2 (residual2.cuh), so r is
// the value the fused residual x-pass transforms, bit for bit.  Per-CTA sums of
// r^2 and S^2 go to the residual-norm partials.
#include "kernels.cuh"
#include "residual2.cuh"

namespace pgb {

namespace {

constexpr int kRsTX = 64;   // x points per tile (32 lanes x 2)
constexpr int kRsTY = 8;    // rows per tile (one warp each)
constexpr int kRsZC = 16;   // levels per CTA

struct P2 {
  float2 p, q;   // the pair's p0 and q values
};

template <bool HAS_Q>
__device__ __forceinline__ P2 load_pair(const ResidualArgs& R, long long idx2) {
  P2 v;
  v.p = __ldg(reinterpret_cast<const float2*>(R.p0) + idx2);
  v.q = HAS_Q ? __ldg(reinterpret_cast<const float2*>(R.q) + idx2) : make_float2(0.f, 0.f);
  return v;
}

template <bool HAS_Q>
__device__ __forceinline__ float2 load_one(const ResidualArgs& R, long long idx) {
  return make_float2(__ldg(R.p0 + idx), HAS_Q ? __ldg(R.q + idx) : 0.f);
}

template <bool HAS_Q, bool ISO>
__global__ void __launch_bounds__(kRsTX / 2 * kRsTY, 3) k_res_stencil(ResidualArgs R, float* __restrict__ r_out, Geom g,
                                                                   const int* __restrict__ done) {
  pdl_trigger();
  // shared: two buffers of (TY + 2) rows x 32 pairs of (p0, q)
  __shared__ P2 rows[2][kRsTY + 2][kRsTX / 2];
  __shared__ float red[2][kRsTX / 2 * kRsTY];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i2 = blockIdx.x * (kRsTX / 2) + lane;         // point pair (2 i2, 2 i2 + 1)
  const int j = blockIdx.y * kRsTY + w;
  const int k0 = blockIdx.z * kRsZC, k1 = min(nz, k0 + kRsZC);
  const long long plane2 = (long long)nx * ny / 2;        // pairs per level
  const int nx2 = nx / 2;
  const long long row2 = (long long)j * nx2 + i2;         // pair index within a level
  // halo rows (warp 0: j0 - 1, warp TY-1: j0 + TY, periodic) and edge points (lane 0: x0 - 1,
  // lane 31: x0 + 64, periodic)
  const int jh = (w == 0) ? (blockIdx.y * kRsTY + ny - 1) % ny : (blockIdx.y * kRsTY + kRsTY) % ny;
  const long long rowh2 = (long long)jh * nx2 + i2;
  const int xe = (lane == 0) ? (blockIdx.x * kRsTX + nx - 1) % nx : (blockIdx.x * kRsTX + kRsTX) % nx;
  const bool halo = (w == 0 || w == kRsTY - 1);
  const bool edge = (lane == 0 || lane == 31);
  const float2 cx = R.cx, cy = R.cy;
  pdl_wait();   // the previous kernels of the stream are complete
  if (done && *done) return;
  const float2 mu = *R.mu_ff;
  // window: dn = level k-1, c = k, up = k+1 (own pair); nh/ne: level k+1's halo row and edge point
  P2 dn, c, up;
  P2 hl_c, hl_up;        // this warp's halo row value at level k and k+1 (warps 0 and TY-1)
  float2 ed_c, ed_up;    // this lane's edge point (p0, q) at level k and k+1 (lanes 0 and 31)
  c = load_pair<HAS_Q>(R, (long long)k0 * plane2 + row2);
  hl_up = c;
  ed_up = make_float2(0.f, 0.f);
  dn = (k0 > 0) ? load_pair<HAS_Q>(R, (long long)(k0 - 1) * plane2 + row2) : c;
  up = (k0 + 1 < nz) ? load_pair<HAS_Q>(R, (long long)(k0 + 1) * plane2 + row2) : P2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  hl_c = halo ? load_pair<HAS_Q>(R, (long long)k0 * plane2 + rowh2) : c;
  ed_c = edge ? load_one<HAS_Q>(R, (long long)k0 * nx * ny + (long long)j * nx + xe) : make_float2(0.f, 0.f);
  // the source two levels ahead as well (its latency would otherwise stall every level)
  const double2* S2 = reinterpret_cast<const double2*>(R.S) + row2;
  double2 s_c = __ldcs(S2 + (long long)k0 * plane2);
  double2 s_up = (k0 + 1 < k1) ? __ldcs(S2 + (long long)(k0 + 1) * plane2) : s_c;
  float2 racc = make_float2(0.f, 0.f), sacc = racc;
  int b = 0;
  for (int k = k0; k < k1; ++k, b ^= 1) {
    // loads for the next levels (independent of this level's arithmetic)
    const bool has_up = k + 1 < nz, has_up2 = k + 2 < nz;
    P2 up2 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (k + 1 < k1 && has_up2) up2 = load_pair<HAS_Q>(R, (long long)(k + 2) * plane2 + row2);
    double2 s_up2 = s_up;
    if (k + 2 < k1) s_up2 = __ldcs(S2 + (long long)(k + 2) * plane2);
    if (k + 1 < k1 && halo) hl_up = load_pair<HAS_Q>(R, (long long)(k + 1) * plane2 + rowh2);
    if (k + 1 < k1 && edge) ed_up = load_one<HAS_Q>(R, (long long)(k + 1) * nx * ny + (long long)j * nx + xe);
    const double2 Sv = s_c;
    // publish this level's row (and the halo rows) for the y neighbours
    rows[b][w + 1][lane] = c;
    if (w == 0) rows[b][0][lane] = hl_c;
    if (w == kRsTY - 1) rows[b][kRsTY + 1][lane] = hl_c;
    __syncthreads();
    const P2 north = rows[b][w + 2][lane], south = rows[b][w][lane];
    // x neighbours: east of the pair = (c.x of lane+1), west = (c.y of lane-1); the tile's edges
    // from the loaded edge points
    float pe = __shfl_down_sync(0xffffffffu, c.p.x, 1), pw = __shfl_up_sync(0xffffffffu, c.p.y, 1);
    float qe = __shfl_down_sync(0xffffffffu, c.q.x, 1), qw = __shfl_up_sync(0xffffffffu, c.q.y, 1);
    if (lane == 31) {   // east of the tile
      pe = ed_c.x;
      qe = ed_c.y;
    }
    if (lane == 0) {    // west of the tile
      pw = ed_c.x;
      qw = ed_c.y;
    }
    float2 Sh, Sl;
    d2ff_trunc(Sv.x, Sh.x, Sl.x);
    d2ff_trunc(Sv.y, Sh.y, Sl.y);
    const ResCoef K = res_coef(cx, cy, R.a_ff[k], R.c_ff[k], mu);
    const float2 pu = has_up ? up.p : make_float2(0.f, 0.f), qu = has_up ? up.q : make_float2(0.f, 0.f);
    const float2 rr = residual_value2<HAS_Q, ISO>(c.p, make_float2(c.p.y, pe), make_float2(pw, c.p.x), north.p, south.p,
                                             dn.p, pu, c.q, make_float2(c.q.y, qe), make_float2(qw, c.q.x), north.q,
                                             south.q, dn.q, qu, Sh, Sl, K);
    __stcs(reinterpret_cast<float2*>(r_out) + (long long)k * plane2 + row2, rr);
    racc = fma2(rr, rr, racc);
    sacc = fma2(Sh, Sh, sacc);
    // slide the window
    dn = c;
    c = up;
    up = up2;
    s_c = s_up;
    s_up = s_up2;
    hl_c = hl_up;
    ed_c = ed_up;
  }
  // per-CTA sums of r^2 and S^2 (fixed-order tree)
  constexpr int TH = kRsTX / 2 * kRsTY;
  const int tid = threadIdx.x;
  red[0][tid] = racc.x + racc.y;
  red[1][tid] = sacc.x + sacc.y;
  __syncthreads();
  for (int h = TH / 2; h > 0; h >>= 1) {
    if (tid < h) {
      red[0][tid] += red[0][tid + h];
      red[1][tid] += red[1][tid + h];
    }
    __syncthreads();
  }
  if (tid == 0 && R.partials) {
    const long long slot = R.part0 + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    R.partials[2 * slot] = (double)red[0][0];
    R.partials[2 * slot + 1] = (double)red[1][0];
  }
}

}  // namespace

bool residual_stencil_supported(int nx, int ny) { return nx % kRsTX == 0 && ny % kRsTY == 0; }

long long residual_stencil_blocks(int nx, int ny, int nz) {
  return (long long)(nx / kRsTX) * (ny / kRsTY) * ((nz + kRsZC - 1) / kRsZC);
}

cudaError_t launch_residual_stencil(const ResidualArgs& R, float* r_out, const Geom& g, const int* done,
                                    int* nblocks_out, cudaStream_t st, bool* used) {
  *used = false;
  if (!residual_stencil_supported(g.nx, g.ny) || g.lev0 != 0 || g.lev1 != g.nz) return cudaSuccess;
  const dim3 grid(g.nx / kRsTX, g.ny / kRsTY, (g.nz + kRsZC - 1) / kRsZC);
  if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
  *used = true;
  const dim3 block(kRsTX / 2 * kRsTY);
  if (R.cx.x == R.cy.x && R.cx.y == R.cy.y) {   // dx == dy: merged horizontal term
    if (R.q) return pdl_launch(k_res_stencil<true, true>, grid, block, 0, st, R, r_out, g, done);
    return pdl_launch(k_res_stencil<false, true>, grid, block, 0, st, R, r_out, g, done);
  }
  if (R.q) return pdl_launch(k_res_stencil<true, false>, grid, block, 0, st, R, r_out, g, done);
  return pdl_launch(k_res_stencil<false, false>, grid, block, 0, st, R, r_out, g, done);
}

}  // namespace pgb
