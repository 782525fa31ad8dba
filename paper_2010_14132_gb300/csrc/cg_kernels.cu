// Preconditioned conjugate gradients for a density that varies in x, y and z,
// with the direct FFT solve as the preconditioner.  This is the iterative
// alternative of Section 2.2 (a matrix-free CG whose cost per iteration is a
// stencil application and a few vector updates, preconditioned by a cheap
// approximate inverse), for the case the direct method alone cannot handle: a
// horizontally varying density does not separate under the Fourier transform.
//
// Operator (flux form, cell weights W_ijk = rho_ijk dz_k):
//   (W A d)_ijk = dz_k [ (F^x_{i+1/2} - F^x_{i-1/2})/dx + (F^y_{j+1/2} - F^y_{j-1/2})/dy ]
//               + F^z_{k+1/2} - F^z_{k-1/2},
//   F^x_{i+1/2} = rho_{i+1/2} (d_{i+1} - d_i)/dx, rho_{i+1/2} = (rho_i + rho_{i+1})/2 (periodic);
//   F^y likewise; F^z_{k+1/2} = rho_{k+1/2} (d_{k+1} - d_k)/h_{k+1/2}, zero at the bottom face and
//   at the top face, or rho_{nz-1} (0 - d_{nz-1})/(dz_{nz-1}/2) with p = 0 on the top face.
// CG runs on K = -W A (symmetric, positive semidefinite) with b = -W (S - mu_W); the
// preconditioner is z = -G(r / Wbar): G is the plan's solve for the level density
// rho0 (weights Wbar_k = rho0_k dz_k).  Polak-Ribiere beta = -alpha (q . z_new)/(r . z)
// keeps the iteration robust to a preconditioner that is applied in reduced precision.
// All vectors and reductions are FP64; the partial sums go to the host in block order.
// The FP64 pipe (1/65 of the FP32 rate here) would bound these kernels, so no FP64
// division runs per point: the level reciprocals come from small tables, and the
// residual's weight 1/rho (needed only for the stopping test) is a float reciprocal.
// The operator itself runs in double-float arithmetic: its six face coefficients are
// formed once per solve in FP64 and stored as float pairs, and each application
// splits the FP64 direction into float pairs with integer operations and forms
// sum_f c_f (d_f - d_c) with error-free transformations, differences first.
#include "kernels.cuh"
#include "residual2.cuh"

namespace pgb {
namespace {

struct CgDims {
  int nx, ny, nz;
  long long plane, n;
  double hx2, hy2;     // 0.5/dx^2, 0.5/dy^2 (the 0.5 of the face-density mean folded in)
  int top_dirichlet;
};

__device__ __forceinline__ void block_sum2(double a, double b, double* partials) {
  __shared__ double s0[256], s1[256];
  const int t = threadIdx.x;
  s0[t] = a;
  s1[t] = b;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) {
      s0[t] += s0[t + h];
      s1[t] += s1[t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    partials[2 * blockIdx.x] = s0[0];
    partials[2 * blockIdx.x + 1] = s1[0];
  }
}

// Face coefficients of W A, once per solve, as float pairs (hi, lo):
//   ce = 0.5/dx^2 (rho_i + rho_{i+1}) dz_k (east face), cn = 0.5/dy^2 (rho_j + rho_{j+1}) dz_k (north),
//   cu = (rho_k + rho_{k+1}) 0.5/h_{k+1/2} (upper; at the top rho_k 2/dz_k with p = 0 on the face, else 0).
// x as a float pair (h, l) with integer operations (h + l within 2^-47 |x|), keeping the
// conversions off the FP64 pipe; the sums and products above stay in FP64 (6 operations per point)
__device__ __forceinline__ float2 split_int(double x) {
  float h, l;
  d2ff_trunc(x, h, l);
  return make_float2(h, l);
}

__global__ void __launch_bounds__(256) k_cg_faces(const double* __restrict__ rho, float2* __restrict__ ce,
                                                  float2* __restrict__ cn, float2* __restrict__ cu,
                                                  const CgLevel* __restrict__ lv, CgDims D) {
  const long long rows = (long long)D.nz * D.ny;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int k = (int)(row / D.ny), j = (int)(row - (long long)k * D.ny);
    const CgLevel L = lv[k];
    const long long base = row * D.nx;
    const long long dn_ = (j + 1 == D.ny ? (1 - D.ny) * (long long)D.nx : D.nx);
    for (int i = threadIdx.x; i < D.nx; i += blockDim.x) {
      const long long idx = base + i;
      const long long e = idx + (i + 1 == D.nx ? 1 - D.nx : 1);
      const double rc = rho[idx];
      ce[idx] = split_int(D.hx2 * (rc + rho[e]) * L.dz);
      cn[idx] = split_int(D.hy2 * (rc + rho[idx + dn_]) * L.dz);
      double up = 0.0;
      if (k + 1 < D.nz) up = (rc + rho[idx + D.plane]) * L.hup;
      else if (D.top_dirichlet) up = rc * L.hup;
      cu[idx] = split_int(up);
    }
  }
}

// c (d_f - d_c) as an unnormalised float pair (ph, pl): the difference of the split values first
// (exact high part), then the product with the split coefficient (exact high product).
__device__ __forceinline__ void face_term(float fh, float fl, float ch, float cl, float2 c, float& ph, float& pl) {
  float s, e;
  two_sum(fh, -ch, s, e);
  const float lo = e + (fl - cl);
  two_prod(c.x, s, ph, pl);
  pl = __fmaf_rn(c.x, lo, __fmaf_rn(c.y, s, pl));
}

// q = K d = -(W A d) = -sum_f c_f (d_f - d_c); partials: d . q
__global__ void __launch_bounds__(256) k_cg_apply(const double* __restrict__ d, const float2* __restrict__ ce,
                                                  const float2* __restrict__ cn, const float2* __restrict__ cu,
                                                  double* __restrict__ q, CgDims D, double* __restrict__ partials) {
  double acc = 0;
  const long long rows = (long long)D.nz * D.ny;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {   // one x row per block step
    const int k = (int)(row / D.ny), j = (int)(row - (long long)k * D.ny);
    const long long base = row * D.nx;
    const long long dn_ = (j + 1 == D.ny ? (1 - D.ny) * (long long)D.nx : D.nx);
    const long long ds_ = (j == 0 ? (D.ny - 1) * (long long)D.nx : -(long long)D.nx);
    const bool has_up = k + 1 < D.nz, has_dn = k > 0;
    for (int i = threadIdx.x; i < D.nx; i += blockDim.x) {
      const long long idx = base + i;
      const long long w = idx + (i == 0 ? D.nx - 1 : -1), e = idx + (i + 1 == D.nx ? 1 - D.nx : 1);
      const double dc = d[idx];
      float ch, cl;
      d2ff_trunc(dc, ch, cl);
      float H = 0.f, Lo = 0.f;
      auto add = [&](double df, float2 c) {
        float fh, fl, ph, pl, s, t;
        d2ff_trunc(df, fh, fl);
        face_term(fh, fl, ch, cl, c, ph, pl);
        two_sum(H, ph, s, t);
        H = s;
        Lo += t + pl;
      };
      add(d[e], ce[idx]);
      add(d[w], ce[w]);
      add(d[idx + dn_], cn[idx]);
      add(d[idx + ds_], cn[idx + ds_]);
      if (has_up) add(d[idx + D.plane], cu[idx]);
      else add(0.0, cu[idx]);   // the face value 0 above the top (cu = 0 there with zero flux)
      if (has_dn) add(d[idx - D.plane], cu[idx - D.plane]);
      float s, t;
      two_sum(H, Lo, s, t);
      const double Kd = -ff2d_fast(s, t);
      q[idx] = Kd;
      acc += dc * Kd;
    }
  }
  block_sum2(acc, 0.0, partials);
}

// r = b = -W (S - mu), p = 0, t = -r/Wbar (the preconditioner's source); partials: S . S
__global__ void __launch_bounds__(256) k_cg_start(const double* __restrict__ rho, const double* __restrict__ S,
                                                  double mu, double* __restrict__ r, double* __restrict__ p,
                                                  double* __restrict__ t, const double* __restrict__ dz,
                                                  const CgLevel* __restrict__ lv, CgDims D,
                                                  double* __restrict__ partials) {
  double ss = 0;
  const long long rows = (long long)D.nz * D.ny;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const CgLevel L = lv[(int)(row / D.ny)];
    for (int i = threadIdx.x; i < D.nx; i += blockDim.x) {
      const long long idx = row * D.nx + i;
      const double s = S[idx];
      const double b = -(rho[idx] * L.dz) * (s - mu);
      r[idx] = b;
      p[idx] = 0.0;
      t[idx] = -b * L.iwbar;
      ss += s * s;
    }
  }
  block_sum2(ss, 0.0, partials);
}

// partials: W S, W (for the compatibility projection mu_W = sum W S / sum W)
__global__ void __launch_bounds__(256) k_cg_wmean(const double* __restrict__ rho, const double* __restrict__ S,
                                                  const double* __restrict__ dz, CgDims D,
                                                  double* __restrict__ partials) {
  double ws = 0, w = 0;
  const long long rows = (long long)D.nz * D.ny;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const double dzk = dz[(int)(row / D.ny)];
    for (int i = threadIdx.x; i < D.nx; i += blockDim.x) {
      const long long idx = row * D.nx + i;
      const double wk = rho[idx] * dzk;
      ws += wk * S[idx];
      w += wk;
    }
  }
  block_sum2(ws, w, partials);
}

// p += alpha d, r -= alpha q, t = -r/Wbar; partials: (r/(W ||S||))^2 (the relative residual of A p = S - mu)
__global__ void __launch_bounds__(256) k_cg_update(const double* __restrict__ rho, double alpha, float inv_snorm,
                                                   const double* __restrict__ d, const double* __restrict__ q,
                                                   double* __restrict__ p, double* __restrict__ r,
                                                   double* __restrict__ t, const CgLevel* __restrict__ lv, CgDims D,
                                                   double* __restrict__ partials) {
  float rr = 0.f;
  const long long rows = (long long)D.nz * D.ny;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const CgLevel L = lv[(int)(row / D.ny)];
    const float idz = (float)L.idz * inv_snorm;   // the norm comes out relative to ||S||
  for (int i = threadIdx.x; i < D.nx; i += blockDim.x) {
    const long long idx = row * D.nx + i;
    p[idx] += alpha * d[idx];
    const double rn = r[idx] - alpha * q[idx];
    r[idx] = rn;
    t[idx] = -rn * L.iwbar;
    // residual of A p = S - mu: r / (rho dz), to float accuracy (a stopping test), in the FP32 pipe
    float rh, rl, h, l;
    d2ff_trunc(rn, rh, rl);
    d2ff_trunc(rho[idx], h, l);
    const float ra = rh * idz * __frcp_rn(h);
    rr = __fmaf_rn(ra, ra, rr);
  }
  }
  block_sum2((double)rr, 0.0, partials);
}

// partials: z . r, z . q
__global__ void __launch_bounds__(256) k_cg_dots(const double* __restrict__ z, const double* __restrict__ r,
                                                 const double* __restrict__ q, CgDims D,
                                                 double* __restrict__ partials) {
  double zr = 0, zq = 0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < D.n;
       idx += (long long)gridDim.x * blockDim.x) {
    const double zv = z[idx];
    zr += zv * r[idx];
    if (q) zq += zv * q[idx];
  }
  block_sum2(zr, zq, partials);
}

// d = z + beta d (beta_is_zero: d = z, whatever d held)
__global__ void __launch_bounds__(256) k_cg_dir(const double* __restrict__ z, double beta, int beta_is_zero,
                                                double* __restrict__ d, long long n) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    d[idx] = beta_is_zero ? z[idx] : z[idx] + beta * d[idx];
}

// partials: sum p; then (second launch) p -= shift
__global__ void __launch_bounds__(256) k_cg_sum(const double* __restrict__ p, long long n,
                                                double* __restrict__ partials) {
  double s = 0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    s += p[idx];
  block_sum2(s, 0.0, partials);
}
__global__ void __launch_bounds__(256) k_cg_shift(double* __restrict__ p, double shift, long long n) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    p[idx] -= shift;
}

}  // namespace

// Host side ---------------------------------------------------------------------

int cg_blocks() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (sms > 0 ? sms : 1) * 8;
}

CgKernels cg_kernels(int nx, int ny, int nz, double dx, double dy, int top_dirichlet) {
  CgKernels K{};
  K.nx = nx;
  K.ny = ny;
  K.nz = nz;
  K.idx2 = 1.0 / (dx * dx);
  K.idy2 = 1.0 / (dy * dy);
  K.top_dirichlet = top_dirichlet;
  return K;
}

static CgDims dims_of(const CgKernels& K) {
  CgDims D{};
  D.nx = K.nx;
  D.ny = K.ny;
  D.nz = K.nz;
  D.plane = (long long)K.nx * K.ny;
  D.n = D.plane * K.nz;
  D.hx2 = 0.5 * K.idx2;
  D.hy2 = 0.5 * K.idy2;
  D.top_dirichlet = K.top_dirichlet;
  return D;
}

// the row kernels step over x rows, the flat ones over points
static unsigned grid_for(long long n, int nb) {
  long long g = (n + 255) / 256;
  if (g > nb) g = nb;
  return (unsigned)(g < 1 ? 1 : g);
}

// blocks of every CG kernel: one x row per block step (at most nb blocks)
unsigned cg_grid(const CgKernels& K, int nb) { return grid_for((long long)K.nz * K.ny * 256, nb); }

cudaError_t cg_launch(int op, const CgKernels& K, const CgArgs& a, int nb, cudaStream_t st) {
  const CgDims D = dims_of(K);
  const unsigned g = cg_grid(K, nb), gr = g;   // every kernel: the same grid, so the host sums g partials
  switch (op) {
    case CG_WMEAN: k_cg_wmean<<<gr, 256, 0, st>>>(a.rho, a.S, a.dz, D, a.partials); break;
    case CG_START:
      k_cg_start<<<gr, 256, 0, st>>>(a.rho, a.S, a.scalar, a.r, a.p, a.t, a.dz, a.lv, D, a.partials);
      break;
    case CG_FACES: k_cg_faces<<<gr, 256, 0, st>>>(a.rho, a.ce, a.cn, a.cu, a.lv, D); break;
    case CG_APPLY: k_cg_apply<<<gr, 256, 0, st>>>(a.d, a.ce, a.cn, a.cu, a.q, D, a.partials); break;
    case CG_UPDATE:
      k_cg_update<<<gr, 256, 0, st>>>(a.rho, a.scalar, (float)a.inv_snorm, a.d, a.q, a.p, a.r, a.t, a.lv, D,
                                      a.partials);
      break;
    case CG_DOTS: k_cg_dots<<<g, 256, 0, st>>>(a.z, a.r, a.q, D, a.partials); break;
    case CG_DIR: k_cg_dir<<<g, 256, 0, st>>>(a.z, a.scalar, a.flag, a.d, D.n); break;
    case CG_SUM: k_cg_sum<<<g, 256, 0, st>>>(a.p, D.n, a.partials); break;
    case CG_SHIFT: k_cg_shift<<<g, 256, 0, st>>>(a.p, a.scalar, D.n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}



}  // namespace pgb
