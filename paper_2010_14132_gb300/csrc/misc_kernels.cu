// Refinement control, correction rebuild, coefficient tables, rho0-gradient reductions and
// the field-layout conversion.
#include "columns.cuh"
#include "kernels.cuh"
#include "residual2.cuh"

namespace pgb {

// ---------------------------------------------------------------------------
// Vertical coefficient tables (one thread per level, FP64; nz values only).
//   W_k = rho_k dz_k, a_k = rho_{k-1/2}/(W_k h_{k-1/2}), c_k = rho_{k+1/2}/(W_k h_{k+1/2}),
//   h_{k+1/2} = (dz_k + dz_{k+1})/2, rho_{k+1/2} = (rho_k + rho_{k+1})/2; a_0 = 0 (zero flux
//   through the bottom face).  Top face: zero flux gives c_{nz-1} = 0; p = 0 on it (Dirichlet)
//   gives the flux rho_top (0 - p_{nz-1})/(dz_{nz-1}/2), so c_{nz-1} = rho_top/(W h) with
//   h = dz_{nz-1}/2 and rho_top = rho_{nz-1} (only centre densities are given).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 split_ff(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return make_float2(h, l);
}

__global__ void k_coefficients(const double* __restrict__ dz, const double* __restrict__ rho, int nz,
                               double* a_d, double* c_d, double* W_d, float* a_f, float* c_f, float2* a_ff,
                               float2* c_ff, int top_dirichlet) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nz; k += blockDim.x * gridDim.x) {
    const double W = rho[k] * dz[k];
    const double up = (k + 1 < nz)      ? (0.5 * (rho[k] + rho[k + 1])) / (0.5 * (dz[k] + dz[k + 1]))
                      : top_dirichlet ? rho[k] / (0.5 * dz[k])
                                      : 0.0;
    const double dn = (k > 0) ? (0.5 * (rho[k - 1] + rho[k])) / (0.5 * (dz[k - 1] + dz[k])) : 0.0;
    const double a = dn / W, c = up / W;
    a_d[k] = a;
    c_d[k] = c;
    W_d[k] = W;
    a_f[k] = __double2float_rn(a);
    c_f[k] = __double2float_rn(c);
    a_ff[k] = split_ff(a);
    c_ff[k] = split_ff(c);
  }
}

cudaError_t launch_coefficients(const double* dz, const double* rho0, int nz, double* a_d, double* c_d,
                                double* W_d, float* a_f, float* c_f, float2* a_ff, float2* c_ff, int top_dirichlet,
                                cudaStream_t st) {
  k_coefficients<<<(nz + 127) / 128, 128, 0, st>>>(dz, rho0, nz, a_d, c_d, W_d, a_f, c_f, a_ff, c_ff, top_dirichlet);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Limiting accuracy of the mixed refinement: the part of the error that no sweep
// removes, because the residual r = S - mu_W - L p is formed in double-float
// arithmetic (unit roundoff u = 2^-48).  Each of the operator's products rounds
// at about u K |p| (K = max_k (a_k + c_k) + 2/dx^2 + 2/dy^2, the largest
// coefficient sum), so r carries noise of size about u K ||p|| that is
// uncorrelated from point to point, and the correction solved from it carries
// L^{-1} of that noise.  For noise of equal variance in every mode the expected
// norm is u K ||p|| sqrt(mean over the modes of 1/lambda^2), lambda running over
// the eigenvalues lambda_h(kx, ky) + mu_m of the discrete operator (the singular
// mode of the Neumann problem excluded: the solve projects it out).  The
// vertical operator W^{-1} M (M symmetric) is similar to the symmetric
// tridiagonal B = W^{-1/2} M W^{-1/2}; its mu_m come from Sturm-count bisection.
// The similarity is not orthogonal, so a noise vector's plain norm can grow by up
// to the factor eta = nz sum W^2/(sum W)^2 >= 1 in the dominant (vertically
// constant) modes; the term is multiplied by sqrt(eta).  Result:
//     F = u K sqrt(eta) sqrt(sum_{modes} 1/lambda^2 / N),   N = nx ny nz,
// the relative error below which the refinement's error bound cannot certify a
// result; it is added to every bound.  The sum over (kx, ky) uses the
// geometric-grid value g(t_j) >= g(lambda_h), t_j <= lambda_h, of the decreasing
// g(lambda) = sum_m 1/(lambda + mu_m)^2 (at most (t_{j+1}/t_j)^2 = 1.06 too large).
// One block; fixed-order sums (deterministic).
// ---------------------------------------------------------------------------
constexpr int kFloorThreads = 512;   // >= the largest nz a plan accepts
constexpr int kFloorGrid = 512;

__device__ int sturm_count(const double* d, const double* e2, int nz, double x) {
  // eigenvalues of B below x = negative pivots of the LDL^T factorisation of B - x I
  int cnt = 0;
  double q = d[0] - x;
  for (int k = 0;;) {
    if (q < 0) ++cnt;
    if (++k == nz) break;
    const double qq = (q != 0.0) ? q : -1e-300;
    q = d[k] - x - e2[k - 1] / qq;
  }
  return cnt;
}

__global__ void __launch_bounds__(kFloorThreads) k_accuracy_floor(const double* __restrict__ a,
                                                                   const double* __restrict__ c,
                                                                   const double* __restrict__ W, int nz, int nx,
                                                                   int ny, double dx, double dy, int top_dirichlet,
                                                                   double* __restrict__ out) {
  __shared__ double d[kFloorThreads], e2[kFloorThreads], mu[kFloorThreads];
  __shared__ double g[kFloorGrid];
  __shared__ double red[6][kFloorThreads];
  const int t = threadIdx.x;
  double kmax = 0, sw = 0, sw2 = 0, gmax = 0, wmax = 0, wmin = 1e300;
  for (int k = t; k < nz; k += blockDim.x) {
    d[k] = a[k] + c[k];
    e2[k] = (k + 1 < nz) ? c[k] * a[k + 1] : 0.0;   // squared off-diagonal of B between k and k+1
  }
  __syncthreads();
  for (int k = t; k < nz; k += blockDim.x) {
    kmax = fmax(kmax, d[k]);
    wmax = fmax(wmax, W[k]);
    wmin = fmin(wmin, W[k]);
    sw += W[k];
    sw2 += W[k] * W[k];
    const double off = ((k > 0) ? sqrt(e2[k - 1]) : 0.0) + ((k + 1 < nz) ? sqrt(e2[k]) : 0.0);
    gmax = fmax(gmax, d[k] + off);   // Gershgorin bound on the spectrum of B
  }
  red[0][t] = kmax;
  red[1][t] = sw;
  red[2][t] = sw2;
  red[3][t] = gmax;
  red[4][t] = wmax;
  red[5][t] = wmin;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (t < h) {
      red[0][t] = fmax(red[0][t], red[0][t + h]);
      red[1][t] += red[1][t + h];
      red[2][t] += red[2][t + h];
      red[3][t] = fmax(red[3][t], red[3][t + h]);
      red[4][t] = fmax(red[4][t], red[4][t + h]);
      red[5][t] = fmin(red[5][t], red[5][t + h]);
    }
    __syncthreads();
  }
  const double wratio = (red[5][0] > 0) ? red[4][0] / red[5][0] : 1.0;
  const double K = red[0][0] + 2.0 / (dx * dx) + 2.0 / (dy * dy);
  const double eta = (red[1][0] > 0) ? nz * red[2][0] / (red[1][0] * red[1][0]) : 1.0;
  const double top = red[3][0] * (1.0 + 1e-12) + 1e-300;
  // mu_m, m-th smallest eigenvalue of B (count(x) <= m exactly for x <= mu_m), to a relative
  // 1e-7; with zero flux through top and bottom mu_0 = 0 (the constants are the null space)
  for (int m = t; m < nz; m += blockDim.x) {
    double lo = 0.0, hi = top;
    if (m > 0 || top_dirichlet) {
      for (int it = 0; it < 200 && hi - lo > 1e-7 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(d, e2, nz, mid) <= m) lo = mid;
        else hi = mid;
      }
      mu[m] = 0.5 * (lo + hi);
    } else {
      mu[m] = 0.0;
    }
  }
  __syncthreads();
  // g on the grid t_j = lam_lo exp(j h) spanning the nonzero horizontal eigenvalues
  const double sx = sinpi(1.0 / nx), sy = sinpi(1.0 / ny);
  const double lam_lo = fmin(4.0 / (dx * dx) * sx * sx, 4.0 / (dy * dy) * sy * sy);
  const double lam_hi = 4.0 / (dx * dx) + 4.0 / (dy * dy);
  const double hstep = log(lam_hi / lam_lo) / (kFloorGrid - 1);
  for (int j = t; j < kFloorGrid; j += blockDim.x) {
    const double tj = lam_lo * exp(j * hstep);
    double s = 0;
    for (int m = 0; m < nz; ++m) {
      const double v = 1.0 / (tj + mu[m]);
      s += v * v;
    }
    g[j] = s;
  }
  __syncthreads();
  // sum over the wavenumber pairs, each unique |kx|, |ky| with its multiplicity
  const int ux = nx / 2 + 1, uy = ny / 2 + 1;
  double acc = 0;
  for (long long pidx = t; pidx < (long long)ux * uy; pidx += blockDim.x) {
    const int kx = (int)(pidx % ux), ky = (int)(pidx / ux);
    const double mx = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
    const double my = (ky == 0 || 2 * ky == ny) ? 1.0 : 2.0;
    const double s1 = sinpi((double)kx / nx), s2 = sinpi((double)ky / ny);
    const double lam = 4.0 / (dx * dx) * s1 * s1 + 4.0 / (dy * dy) * s2 * s2;
    double gv;
    if (kx == 0 && ky == 0) {   // the mean column: its own eigenvalues, the singular one excluded
      gv = 0;
      for (int m = top_dirichlet ? 0 : 1; m < nz; ++m) gv += 1.0 / (mu[m] * mu[m]);
    } else {
      int j = (int)floor(log(lam / lam_lo) / hstep);
      j = max(0, min(kFloorGrid - 1, j));
      while (j > 0 && lam_lo * exp(j * hstep) > lam) --j;
      gv = g[j];
    }
    acc += mx * my * gv;
  }
  red[0][t] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (t < h) red[0][t] += red[0][t + h];
    __syncthreads();
  }
  if (t == 0) {
    const double u = 0x1p-48;
    const double npts = (double)nx * ny * nz;
    out[0] = u * K * sqrt(eta) * sqrt(red[0][0] / npts);
    out[1] = wratio;
    out[2] = sqrt(eta) * sqrt(red[0][0] / npts);   // the same amplification for any residual noise
  }
}

cudaError_t launch_accuracy_floor(const double* a_d, const double* c_d, const double* W_d, int nz, int nx, int ny,
                                  double dx, double dy, int top_dirichlet, double* out, cudaStream_t st) {
  if (nz > kFloorThreads) return cudaErrorInvalidValue;
  k_accuracy_floor<<<1, kFloorThreads, 0, st>>>(a_d, c_d, W_d, nz, nx, ny, dx, dy, top_dirichlet, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pivot reciprocals of the listed low-|k| columns, one thread per column, with the step the column
// solves use (lowk_pivot_step), so that reading the table gives the same solution bit for bit.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_lowk_pivots(const int2* __restrict__ cols, int n,
                                                     const double* __restrict__ a, const double* __restrict__ c,
                                                     const double* __restrict__ lamx,
                                                     const double* __restrict__ lamy, int nz, int singular00,
                                                     double* __restrict__ inv_tab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int2 ck = cols[j];
  const bool singular = singular00 && ck.x == 0 && ck.y == 0;
  const double s = singular ? 0.0 : -(lamx[ck.x] + lamy[ck.y]);
  double g_prev = s, inv_prev = 0.0;
  for (int k = 0; k < nz; ++k) {
    const double inv = lowk_pivot_step<double>(k, s, a[k], c[k], g_prev, inv_prev, singular && (k == nz - 1));
    inv_tab[(size_t)j * nz + k] = inv;
    inv_prev = inv;
  }
}

cudaError_t launch_lowk_pivots(const int2* cols, int n, const double* a_d, const double* c_d, const double* lamx_d,
                               const double* lamy_d, int nz, int singular00, double* inv_tab, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_lowk_pivots<<<(n + 127) / 128, 128, 0, st>>>(cols, n, a_d, c_d, lamx_d, lamy_d, nz, singular00, inv_tab);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Refinement control: sums the x-pass partials in a fixed order (the inverse
// x-pass's delta^2, p^2, sum p and the forward x-pass's r^2, S^2), records the
// relative update, relative residual and error bound, and sets the done flag
// (control_decide in kernels.cuh states the stopping rule).
// ---------------------------------------------------------------------------
// Stage 1 (kControlBlocks blocks): each block sums a contiguous range of the
// partials in a fixed order; the last block to finish (ticket counter) sums the
// block results in block order and applies the stopping rule.  Deterministic.
constexpr int kControlBlocks = 64;

__global__ void __launch_bounds__(256) k_control(Stats* st, const double* __restrict__ partials, int nblocks,
                                                  const double* __restrict__ res_partials, int res_nblocks,
                                                  int pass, int max_sweeps, double tol,
                                                  const double* __restrict__ floor, long long npoints,
                                                  int wrote_p, double* __restrict__ stage,
                                                  unsigned* __restrict__ ticket) {
  __shared__ double sh[5][256];
  __shared__ bool last;
  if (st->done) return;   // later sweeps after convergence: nothing to do
  const int t = threadIdx.x;
  const int per = (nblocks + gridDim.x - 1) / gridDim.x;
  const int b0 = blockIdx.x * per, b1 = min(nblocks, b0 + per);
  const int rper = (res_nblocks + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rper, r1 = min(res_nblocks, r0 + rper);
  double v[5] = {0, 0, 0, 0, 0};
  for (int i = b0 + t; i < b1; i += blockDim.x) {
    v[0] += partials[3 * i];
    v[1] += partials[3 * i + 1];
    v[2] += partials[3 * i + 2];
  }
  for (int i = r0 + t; i < r1; i += blockDim.x) {
    v[3] += res_partials[2 * i];
    v[4] += res_partials[2 * i + 1];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) sh[k][t] = v[k];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (t < h) {
#pragma unroll
      for (int k = 0; k < 5; ++k) sh[k][t] += sh[k][t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) stage[5 * blockIdx.x + k] = sh[k][0];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || t != 0) return;
  __threadfence();
  double tot[5] = {0, 0, 0, 0, 0};
  for (int i = 0; i < (int)gridDim.x; ++i)
#pragma unroll
    for (int k = 0; k < 5; ++k) tot[k] += stage[5 * i + k];
  *ticket = 0;   // ready for the next pass
  control_decide(st, tot[0], tot[1], tot[2], tot[3], tot[4], pass, max_sweeps, tol, npoints, wrote_p, *floor);
}

// ---------------------------------------------------------------------------
// Verification of the current iterate by the next correction's norm (see launch_verify in
// kernels.cuh).  One block; fixed-order sums.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_verify(Stats* st, const double* __restrict__ sq, int nsq,
                                                 const double* __restrict__ res_partials, int res_nblocks, int pass,
                                                 double tol, const double* __restrict__ floor, double nxny,
                                                 int p_stored, double inv_lcut2, int from_r0) {
  __shared__ double sh[3][1024];
  if (st->done) return;   // an earlier pass already ended the refinement
  const int t = threadIdx.x;
  double a = 0, b = 0, c = 0;
  for (int i = t; i < nsq; i += blockDim.x) a += sq[i];
  for (int i = t; i < res_nblocks; i += blockDim.x) {
    b += res_partials[2 * i];
    c += res_partials[2 * i + 1];
  }
  sh[0][t] = a;
  sh[1][t] = b;
  sh[2][t] = c;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (t < h) {
      sh[0][t] += sh[0][t + h];
      sh[1][t] += sh[1][t + h];
      sh[2][t] += sh[2][t + h];
    }
    __syncthreads();
  }
  if (t != 0) return;
  double sd = nxny * sh[0][0];
  // low wavenumbers only: every other column of the correction is (lambda_h + T)^{-1} of the residual's
  // column, with T = W^{-1} M similar to a positive semidefinite matrix through W^{1/2}, so its norm is at
  // most sqrt(W_max/W_min)/lambda_h <= sqrt(W_max/W_min)/lambda_cut times the residual column's (Parseval)
  if (inv_lcut2 > 0) sd += floor[1] * inv_lcut2 * sh[1][0];
  double fl = floor[0], ss = sh[2][0];
  if (from_r0 && pass >= 2) {
    // the residual was formed as r0 - L q from the previous sweep's residual r0 stored in FP32: its
    // rounding (at most 2^-24 ||r0|| in the 2-norm) reaches the correction like the residual's own
    // rounding does, so it adds 2^-24 ||r0|| G/||p|| to the limiting accuracy (G = floor[2]); the
    // source norm is the previous sweep's (this pass did not read S)
    const double sp = st->sq_p[pass - 1];
    if (sp > 0) fl += 0x1p-24 * sqrt(st->sq_res[pass - 2]) * floor[2] / sqrt(sp);
    ss = st->sq_src[pass - 2];
  }
  verify_decide(st, sd, sh[1][0], ss, pass, tol, fl, p_stored);
}

cudaError_t launch_verify(Stats* st_dev, const double* sq, int nsq, const double* res_partials, int res_nblocks,
                          int pass, double tol, const double* floor, double nxny, int p_stored, double inv_lcut2,
                          int from_r0, cudaStream_t st) {
  k_verify<<<1, 1024, 0, st>>>(st_dev, sq, nsq, res_partials, res_nblocks, pass, tol, floor, nxny, p_stored,
                               inv_lcut2, from_r0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Final iterate when the refinement stopped after a sweep that stored only the
// float correction q: p = p0 + q as a double (exact sum of the two floats up to
// the double rounding).  A no-op unless Stats::need_final is set.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finalize(const float2* __restrict__ p0, const float2* __restrict__ q,
                                                  double2* __restrict__ p, long long npairs,
                                                  const Stats* __restrict__ stats) {
  pdl_trigger();
  pdl_wait();   // the previous kernels of the stream are complete
  if (!stats->need_final) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npairs;
       i += (long long)gridDim.x * blockDim.x) {
    __stcs(&p[i], finalize_pair(__ldcs(&p0[i]), __ldcs(&q[i])));
  }
}

// ---------------------------------------------------------------------------
// Accumulated correction of the refinement, rebuilt before a second or third
// sweep: q = p - p0 to float accuracy, from the double iterate p = p0 + q the
// previous sweep stored ((h, l) = p split into floats; h - p0 is exact when h
// and p0 are within a factor 2, and rounds at 2^-24 |q| otherwise).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_q_rebuild(const double2* __restrict__ p, const float2* __restrict__ p0,
                                                   float2* __restrict__ q, long long npairs,
                                                   const int* __restrict__ done) {
  pdl_trigger();
  pdl_wait();   // the previous kernels of the stream are complete
  if (done && *done) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npairs;
       i += (long long)gridDim.x * blockDim.x) {
    __stcs(&q[i], q_rebuild_pair(__ldcs(&p[i]), __ldcs(&p0[i])));
  }
}

cudaError_t launch_q_rebuild(const double* p, const float* p0, float* q, long long n, const int* done,
                             cudaStream_t st) {
  const long long npairs = n / 2;   // nx is even
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (npairs + 255) / 256;
  const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return pdl_launch(k_q_rebuild, dim3((unsigned)blocks), dim3(256), 0, st, (const double2*)p, (const float2*)p0,
                    (float2*)q, npairs, done);
}

cudaError_t launch_control(Stats* st_dev, const double* partials, int nblocks, const double* res_partials,
                           int res_nblocks, int pass, int max_sweeps, double tol, const double* floor,
                           long long npoints, int wrote_p, cudaStream_t st) {
  k_control<<<kControlBlocks, 256, 0, st>>>(st_dev, partials, nblocks, res_partials, res_nblocks, pass, max_sweeps,
                                            tol, floor, npoints, wrote_p, st_dev->control_stage,
                                            &st_dev->control_ticket);
  return cudaGetLastError();
}

__global__ void k_set_if_not_done(cudaGraphConditionalHandle h, const int* __restrict__ done) {
  cudaGraphSetConditional(h, *done ? 0u : 1u);
}

cudaError_t launch_set_if_not_done(cudaGraphConditionalHandle h, const int* done, cudaStream_t st) {
  k_set_if_not_done<<<1, 1, 0, st>>>(h, done);
  return cudaGetLastError();
}

// Zeroes n 32-bit words.  A kernel rather than cudaMemsetAsync: the solve's statistics are cleared on the
// compute stream, where a memset can be served by a copy engine and wait behind a host copy in flight.
__global__ void __launch_bounds__(256) k_zero_words(unsigned* __restrict__ p, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = 0u;
}

cudaError_t launch_zero_words(void* p, size_t bytes, cudaStream_t st) {
  if (bytes % 4) return cudaErrorInvalidValue;
  const long long n = (long long)(bytes / 4);
  if (n == 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 64) blocks = 64;
  k_zero_words<<<(unsigned)blocks, 256, 0, st>>>((unsigned*)p, n);
  return cudaGetLastError();
}

// four ints (src need not be 16-byte aligned)
__global__ void k_copy_status(const int* __restrict__ src, int* dst) {
  dst[0] = src[0];
  dst[1] = src[1];
  dst[2] = src[2];
  dst[3] = src[3];
}

cudaError_t launch_copy_status(const int* src, int* dst, cudaStream_t st) {
  k_copy_status<<<1, 1, 0, st>>>(src, dst);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const float* p0, const float* q, double* p, long long n, const Stats* stats,
                            cudaStream_t st) {
  const long long npairs = n / 2;   // nx is even
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (npairs + 255) / 256;
  const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return pdl_launch(k_finalize, dim3((unsigned)blocks), dim3(256), 0, st, (const float2*)p0, (const float2*)q,
                    (double2*)p, npairs, stats);
}

// ---------------------------------------------------------------------------
// rho0 gradient.  With g = G^T (dL/dp) and D_f = p_{k+1} - p_k on face f = k+1/2:
//   Lo_f = sum_ij g_k D_f,  Up_f = sum_ij g_{k+1} D_f,
//   dL/drho_m = -sum_k (da_k/drho_m * Ma_k + dc_k/drho_m * Mc_k),
//   Mc_k = Lo_k,  Ma_k = -Up_{k-1}.
// Partials per (face, block) are reduced in a fixed order (deterministic).
// ---------------------------------------------------------------------------
template <typename TIO>
__global__ void __launch_bounds__(256) k_grho_partial(const TIO* __restrict__ gS, const TIO* __restrict__ p,
                                                      long long plane, double* __restrict__ partials) {
  __shared__ double s0[256], s1[256];
  const int f = blockIdx.y;
  const TIO* g0 = gS + f * plane;
  const TIO* g1 = g0 + plane;
  const TIO* p0 = p + f * plane;
  const TIO* p1 = p0 + plane;
  TIO lo = 0, up = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (long long)gridDim.x * blockDim.x) {
    const TIO d = p1[i] - p0[i];
    lo += g0[i] * d;
    up += g1[i] * d;
  }
  const int t = threadIdx.x;
  s0[t] = (double)lo;
  s1[t] = (double)up;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) {
      s0[t] += s0[t + h];
      s1[t] += s1[t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    partials[2 * ((long long)f * gridDim.x + blockIdx.x)] = s0[0];
    partials[2 * ((long long)f * gridDim.x + blockIdx.x) + 1] = s1[0];
  }
}

// Mixed dtype: double fields converted with integer operations, float products.
__global__ void __launch_bounds__(256) k_grho_partial_mixed(const double* __restrict__ gS,
                                                            const double* __restrict__ p, long long plane,
                                                            double* __restrict__ partials) {
  __shared__ double s0[256], s1[256];
  const int f = blockIdx.y;
  const double* g0 = gS + f * plane;
  const double* g1 = g0 + plane;
  const double* p0 = p + f * plane;
  const double* p1 = p0 + plane;
  float lo = 0, up = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (long long)gridDim.x * blockDim.x) {
    const float d = d2f_int(p1[i]) - d2f_int(p0[i]);
    lo += d2f_int(g0[i]) * d;
    up += d2f_int(g1[i]) * d;
  }
  const int t = threadIdx.x;
  s0[t] = (double)lo;
  s1[t] = (double)up;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) {
      s0[t] += s0[t + h];
      s1[t] += s1[t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    partials[2 * ((long long)f * gridDim.x + blockIdx.x)] = s0[0];
    partials[2 * ((long long)f * gridDim.x + blockIdx.x) + 1] = s1[0];
  }
}

// One thread per level m; each sums the partials of faces m-1 and m in fixed order.
__global__ void k_grho_final(const double* __restrict__ partials, int nb, int nz, const double* __restrict__ dz,
                             const double* __restrict__ rho, const double* __restrict__ a,
                             const double* __restrict__ c, const double* __restrict__ W, double* __restrict__ grho) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nz) return;
  auto face = [&](int f, int which) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += partials[2 * ((long long)f * nb + b) + which];
    return s;
  };
  auto hf = [&](int f) { return 0.5 * (dz[f] + dz[f + 1]); };
  double acc = 0;
  // a-terms: k = m (face m-1) and k = m+1 (face m); Ma_k = -Up_{k-1}
  if (m >= 1) {
    const double Ma = -face(m - 1, 1);
    acc += (0.5 / (W[m] * hf(m - 1)) - a[m] / rho[m]) * Ma;
  }
  if (m + 1 <= nz - 1) {
    const double Ma = -face(m, 1);
    acc += (0.5 / (W[m + 1] * hf(m))) * Ma;
  }
  // c-terms: k = m (face m) and k = m-1 (face m-1); Mc_k = Lo_k
  if (m <= nz - 2) {
    const double Mc = face(m, 0);
    acc += (0.5 / (W[m] * hf(m)) - c[m] / rho[m]) * Mc;
  }
  if (m >= 1) {
    const double Mc = face(m - 1, 0);
    acc += (0.5 / (W[m - 1] * hf(m - 1))) * Mc;
  }
  grho[m] = -acc;
}

cudaError_t launch_grho(int kind, const void* g, const void* p, const Geom& g_, const Tables& tb, const double* dz,
                        const double* rho0, double* partials, int nparts_max, double* grho, cudaStream_t st) {
  const long long plane = (long long)g_.nx * g_.ny;
  int nb = (int)((plane + 255) / 256);
  if (nb > nparts_max) nb = nparts_max;
  if (nb < 1) nb = 1;
  const dim3 grid(nb, g_.nz - 1);
  if (kind == 0)
    k_grho_partial<double><<<grid, 256, 0, st>>>((const double*)g, (const double*)p, plane, partials);
  else if (kind == 1)
    k_grho_partial<float><<<grid, 256, 0, st>>>((const float*)g, (const float*)p, plane, partials);
  else
    k_grho_partial_mixed<<<grid, 256, 0, st>>>((const double*)g, (const double*)p, plane, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_grho_final<<<(g_.nz + 127) / 128, 128, 0, st>>>(partials, nb, g_.nz, dz, rho0, tb.a_d, tb.c_d, tb.W_d, grho);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Field layout conversion.  MONC keeps its fields with the vertical index
// fastest, [nx][ny][nz]; the solver works on [nz][ny][nx].  Both directions are
// the same operation, dst[b][m][a] = src[a][m][b] (a < A, m < M, b < B): a swap
// of the outer and inner axes, done in 32 x 32 tiles of one m through shared
// memory so that the reads (along b) and the writes (along a) are coalesced.
// The padded row (33) keeps the transposed shared reads free of bank conflicts
// for 4-byte elements and for each half-warp of 8-byte ones.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_swap_outer_inner(const T* __restrict__ src, T* __restrict__ dst, int A,
                                                          int M, int B) {
  __shared__ T tile[32][33];
  const int b0 = blockIdx.x * 32, a0 = blockIdx.y * 32, m = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long src_a = (long long)M * B, dst_b = (long long)M * A;
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx;
    if (a < A && b < B) tile[r][tx] = __ldcs(&src[a * src_a + (long long)m * B + b]);   // read once
  }
  __syncthreads();
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r, a = a0 + tx;
    if (a < A && b < B) dst[b * dst_b + (long long)m * A + a] = tile[tx][r];
  }
}

cudaError_t launch_swap_outer_inner(const void* src, void* dst, int A, int M, int B, int elem_bytes,
                                    cudaStream_t st) {
  if (A <= 0 || M <= 0 || B <= 0 || M > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((B + 31) / 32), (unsigned)((A + 31) / 32), (unsigned)M), block(32, 8);
  if (elem_bytes == 8)
    k_swap_outer_inner<double><<<grid, block, 0, st>>>((const double*)src, (double*)dst, A, M, B);
  else
    k_swap_outer_inner<float><<<grid, block, 0, st>>>((const float*)src, (float*)dst, A, M, B);
  return cudaGetLastError();
}

}  // namespace pgb
