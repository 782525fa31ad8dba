// Internal launch interface between the C ABI (api.cu) and the kernel units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "fft_engine.cuh"

namespace pgb {

// Per-solve device statistics and control flags (zeroed at the start of a solve).
struct Stats {
  double sq_delta[4];     // ||delta_n||^2 of pass n (pass 0 = first solve, delta_0 = p0)
  double sq_p[4];         // ||p||^2 after pass n
  double rel_update[4];
  double sq_res[4];       // ||S - mu_W - L p_n||^2 of iterate n, formed in the forward x-pass of sweep n+1
  double sq_src[4];       // ||S||^2, summed in the same pass
  double rel_residual[4]; // sqrt(sq_res / sq_src)
  double err_est;         // bound on the relative error after the last executed pass
  double err_floor;       // limiting-accuracy term included in err_est (plan constant, see launch_accuracy_floor)
  double mu_w;            // weighted mean removed from the source (first solve)
  double pmean;           // mean of the current mixed iterate p0 + q (double-float accurate)
  float2 mu_ff;           // mu_w as a double-float pair (set after the first solve)
  double control_stage[5 * 64];   // per-block sums of the control reduction
  unsigned control_ticket;        // blocks of the control reduction that have finished
  int need_final;         // the refinement stopped after a sweep that stored q but not p: p = p0 + q still to write
  int p_written;          // the last executed pass stored the double iterate p
  int done;               // later passes become no-ops once set
  int sweeps;
  int converged;
  unsigned err;           // ERR_* bits
};

// Refinement control after pass `pass` (0 = first solve) from the norm sums of
// that pass: sd0 = sum delta^2, sp = sum p^2, sm = sum p (inverse x-pass), and
// sr = sum r^2, ss = sum S^2 of the residual the pass started from (its forward
// x-pass; unused for pass 0).  wrote_p: the pass's inverse x-pass stored the
// double iterate p.  One thread.
//
// Stopping rule (iterative refinement, successive corrections): with delta_n the
// correction of sweep n and e_n the error of the iterate after it,
// e_{n-1} = delta_n + e_n, so a sweep that contracts the error by phi <= 1/2 gives
//     ||e_n|| <= phi/(1 - phi) ||delta_n|| <= ||delta_n||.
// The estimate after sweep n is therefore rel_n = ||delta_n||/||p||, enlarged to
// rel_n phi/(1 - phi) when the contraction measured between the last two sweeps,
// phi = rel_n/rel_{n-1}, exceeds 1/2, and infinite when phi >= 1 (stagnation).
// The bound adds the limiting accuracy F of the double-float residual (floor,
// launch_accuracy_floor): the successive corrections measure the error that the
// sweeps can still remove, not the part that the residual's rounding leaves.
// Converged when the estimate is at most tol; otherwise the next sweep runs, up to
// max_sweeps.
__device__ __forceinline__ void control_decide(Stats* st, double sd0, double sp, double sm, double sr, double ss,
                                               int pass, int max_sweeps, double tol, long long npoints,
                                               int wrote_p, double floor) {
  st->pmean = sm / (double)npoints;
  if (pass == 0) {   // mu_W as a double-float pair, for the residual of the sweeps
    const float h = __double2float_rn(st->mu_w);
    st->mu_ff = make_float2(h, __double2float_rn(st->mu_w - (double)h));
  }
  const double sd = (pass == 0) ? sp : sd0;
  st->sq_delta[pass] = sd;
  st->sq_p[pass] = sp;
  const double rel = (sp > 0) ? sqrt(sd / sp) : 0.0;
  st->rel_update[pass] = (pass == 0) ? 1.0 : rel;
  st->sweeps = pass;
  if (pass == 0) {
    st->err_est = -1.0;
    if (max_sweeps == 0) {
      st->done = 1;
      st->converged = 1;
    }
    return;
  }
  st->sq_res[pass - 1] = sr;
  st->sq_src[pass - 1] = ss;
  st->rel_residual[pass - 1] = (ss > 0) ? sqrt(sr / ss) : 0.0;
  double est = rel;
  if (pass >= 2) {
    const double prev = st->rel_update[pass - 1];
    const double phi = (prev > 0) ? rel / prev : 0.0;
    if (phi >= 1.0) est = __longlong_as_double(0x7ff0000000000000LL);   // +inf: no contraction
    else if (phi > 0.5) est = rel * (phi / (1.0 - phi));
  }
  est += floor;
  st->err_floor = floor;
  st->err_est = est;
  if (est <= tol || sp == 0.0) {   // sp == 0: the solution is exactly zero
    st->done = 1;
    st->converged = 1;
  } else if (rel == 0.0 || pass >= max_sweeps) {   // an exactly zero correction changes nothing more
    st->done = 1;
    st->converged = 0;
  }
  st->p_written = wrote_p;
  if (st->done && !wrote_p) st->need_final = 1;
}

// Verification of iterate p_{pass-1} by the correction of sweep `pass` (solved, not applied):
// sd = ||delta_pass||^2 (Parseval on the solved spectrum), sr, ss the residual norms of the sweep's
// forward x-pass.  With contraction phi <= 1/2, ||e_{pass-1}|| <= ||delta||/(1 - phi) <= 2 ||delta||;
// above 1/2 the factor is 1/(1 - phi), +inf at phi >= 1; the limiting accuracy `floor` is added.
// On success the refinement ends on p_{pass-1}.  p_stored: the sweep's forward pass stored that
// iterate as the double output already.  One thread.
__device__ __forceinline__ void verify_decide(Stats* st, double sd, double sr, double ss, int pass, double tol,
                                              double floor, int p_stored) {
  const double sp = st->sq_p[pass - 1];       // ||p_{pass-1}||^2
  const double rel = (sp > 0) ? sqrt(sd / sp) : 0.0;
  const double prev = st->rel_update[pass - 1];
  const double phi = (pass >= 2 && prev > 0) ? rel / prev : 0.0;
  double est;
  if (phi >= 1.0) est = __longlong_as_double(0x7ff0000000000000LL);
  else est = rel * (phi > 0.5 ? 1.0 / (1.0 - phi) : 2.0);
  est += floor;
  st->sq_res[pass - 1] = sr;
  st->sq_src[pass - 1] = ss;
  st->rel_residual[pass - 1] = (ss > 0) ? sqrt(sr / ss) : 0.0;
  if (est <= tol || sp == 0.0) {
    // the refinement ends on p_{pass-1}: the correction just solved for is not applied
    st->rel_update[pass] = rel;
    st->sq_delta[pass] = sd;
    st->err_est = est;
    st->err_floor = floor;
    st->done = 1;
    st->converged = 1;
    st->sweeps = pass - 1;
    if (!st->p_written && !p_stored) st->need_final = 1;
  }
}

// Device-resident tables owned by a plan.
struct Tables {
  // vertical coefficients, level k
  const double* a_d; const double* c_d; const double* W_d;
  const float* a_f; const float* c_f;
  // double-float splits for the residual: a, c (hi, lo)
  const float2* a_ff; const float2* c_ff;
  // horizontal eigenvalues: lamx[kx], kx < nxh; lamy[ky], ky < ny
  const double* lamx_d; const double* lamy_d;
  const float* lamx_f; const float* lamy_f;
  // twiddles exp(-2 pi i m / n): x line (n = nx/2), R2C post (m = 0..nx/2 over nx), y line
  const double2* twx_d; const double2* twr_d; const double2* twy_d;
  const float2* twx_f; const float2* twr_f; const float2* twy_f;
  // limiting accuracy of the mixed refinement's error bound (one double, launch_accuracy_floor)
  const double* floor_d;
};

struct Geom {
  int nx, ny, nz, nxh, P;      // P: spectrum row pitch (complex elements), >= nxh
  long long plane;             // ny * P
  long long N;                 // nx * ny * nz
  double dx, dy;
  int lev0, lev1;              // levels [lev0, lev1) processed by a transform launch (a chunk)
};

// Output handling of the inverse x-pass.
enum XinvMode : int {
  XINV_PLAIN = 0,   // out[TO] = result
  XINV_P0 = 1,      // mixed first solve: p0 (float) + partial sums of p0^2; optional double output
  XINV_UPDATE = 2   // mixed sweep: q += delta, then q (float) and/or p (double) = p0 + q stored,
                    // partial sums of delta^2, p^2
};

struct XinvExtra {
  float* p0;            // P0: written; UPDATE: read
  float* q;             // UPDATE: the previous correction (read when q_valid)
  int q_valid;          // UPDATE: q holds a previous correction
  float* q_out;         // UPDATE: the new correction q + delta is stored here (nullable)
  double* p_out;        // P0 (when final) / UPDATE: double output field (nullable in UPDATE)
  double* partials;     // per-block partial sums (3 per block: delta^2, p^2, sum p)
  int part0;            // partial-sum slot of this launch's first block
  const double* res_partials;   // the forward x-pass's per-block sums (2 per block: r^2, S^2)
  int res_nblocks;              // their count (0 for the first solve)
  const int* done;      // skip when set (nullable)
  unsigned* err;        // ERR_* bits of the persistent kernels (nullable only when they are not used)
  // refinement control run by the launch's last CTA (persistent kernels; ctl_stats nullable = not fused)
  Stats* ctl_stats;
  int ctl_pass, ctl_max_sweeps;
  double ctl_tol;
  const double* ctl_floor;   // limiting accuracy added to the bound (one double)
  long long ctl_npoints;
};

// Inputs of the double-float refinement residual r = S - mu_W - L (p0 + q).
struct ResidualArgs {
  double* partials;      // per-block sums of r^2 and S^2 (2 per block), from slot part0 on
  int part0;
  double* p_out;         // nullable: the residual x-pass with q also stores the iterate p0 + q here (as
                         // the double the inverse x-pass would write), so that a verification stop
                         // needs no separate pass to form it
  const double* S;
  const float* p0;
  const float* q;        // nullable (first sweep)
  const float2* a_ff;
  const float2* c_ff;
  float2 cx, cy;
  const float2* mu_ff;
  int kmax;              // > 0: the static residual x-pass stores only the bins kx <= kmax (nothing reads
                         // the others); 0: every bin
  // Residual kept between sweep 1 and the verification's first try (static x-pass only): sweep 1 stores
  // its residual r0 in FP32 at r_out (row r at r_out + r r_ld floats); the first try, given r0 instead,
  // forms r0 - L q (S and p0's stencil are not read; p0 only for the stored iterate).
  float* r_out;          // nullable
  const float* r0;       // nullable
  long long r_ld;        // row stride of r_out / r0 in floats
};

// ---- launchers (stream-ordered, return cudaError_t of the launch) ----
cudaError_t launch_xfwd(int ti_is_double, int t_is_double, const void* in, void* spec, const Geom& g,
                        const FftPlan& fx, const Tables& tb, const int* done, cudaStream_t st);
// Forward x-pass of a refinement sweep whose input rows are the residual,
// computed in the load stage (no r array in memory).
cudaError_t launch_xfwd_residual(const ResidualArgs& R, void* spec, const Geom& g, const FftPlan& fx,
                                 const Tables& tb, const int* done, int* nblocks_out, cudaStream_t st);
cudaError_t launch_yfft(int t_is_double, int sign, void* spec, const Geom& g, const FftPlan& fy,
                        const Tables& tb, int tile, const int* done, cudaStream_t st);
// 2-D tensor map over 8-byte elements (dim0 contiguous, dim1 rows of row_stride_bytes);
// false when the driver entry point is unavailable or the shape is rejected.
bool encode_tensor_2d(CUtensorMap* tm, void* base, size_t elem_bytes, unsigned long long dim0,
                      unsigned long long dim1, unsigned long long row_stride_bytes, unsigned box0, unsigned box1);
// 3-D tensor map over 8-byte elements: dim0 contiguous, dim1 and dim2 with the given byte strides.
bool encode_tensor_3d(CUtensorMap* tm, void* base, unsigned long long dim0, unsigned long long dim1,
                      unsigned long long dim2, unsigned long long stride1_bytes, unsigned long long stride2_bytes,
                      unsigned box0, unsigned box1, unsigned box2);
// Persistent TMA y-pass; *used = false when the shape is not supported (caller falls back).
cudaError_t launch_yfft_tma(int t_is_double, int sign, void* spec, const Geom& g, const FftPlan& fy,
                            const Tables& tb, int tile, const int* done, Stats* stats, cudaStream_t st, bool* used);
cudaError_t launch_xinv(int t_is_double, int to_is_double, int mode, const void* spec, void* out,
                        const Geom& g, const FftPlan& fx, const Tables& tb, const XinvExtra& ex,
                        int* nblocks_out, cudaStream_t st);

struct ThomasArgs {
  void* spec;
  int t_is_double;        // storage/compute precision of the main kernel
  int adjoint;
  double scale;           // 1/(nx ny)
  int lowk_r2;            // columns with kx^2+ky'^2 <= lowk_r2 go to the low-k kernel (>= 0)
  int lowk_double;        // low-k kernel computes in double
  const int2* lowk_cols;  // (kx, ky) list, (0,0) first
  int n_lowk;
  double2* lowk_z;        // scratch nz * n_lowk
  double* lowk_w;         // scratch nz * n_lowk
  Stats* stats;
  const int* done;
  const double* target_mean;  // nullable: the (0,0) column then gives the solution mean -(*target_mean)
  int col_tile;               // requested columns per CTA (0 = default)
  int singular00;             // 1: zero flux at the top, so the (0,0) column is singular (projected, pinned)
  double* sqnorm;             // nullable: per-CTA w-weighted sums of |x|^2 of the solved spectrum (the
                              // two-threads-per-column kernel only); *sqnorm_blocks receives their count
  int* sqnorm_blocks;
  const double* lowk_inv;     // nullable: the plan's pivot table of the listed columns (double columns only)
  int kcut;                   // >= 0 (two-threads-per-column kernel): solve only the columns with kx <= kcut
                              // and |ky'| <= kcut (ky' signed); -1: every column
};
cudaError_t launch_thomas(const ThomasArgs& a, const Geom& g, const Tables& tb, cudaStream_t st);

// Refinement residual as its own pass (residual_stencil.cu): r = S - mu_W - L (p0 + q) as float
// into r_out, one z-marching tile kernel; per-CTA r^2, S^2 partials from R.part0.  nx % 64 == 0,
// ny % 8 == 0, all levels in one launch; *used = false otherwise.
bool residual_stencil_supported(int nx, int ny);
long long residual_stencil_blocks(int nx, int ny, int nz);
cudaError_t launch_residual_stencil(const ResidualArgs& R, float* r_out, const Geom& g, const int* done,
                                    int* nblocks_out, cudaStream_t st, bool* used);

// Fused spectral middle (spectral_fused.cu): forward y-pass, forward column solves and inverse
// y-pass of one pass in one persistent kernel over per-strip items.  Float spectra, ny in
// {256, 512, 1024}, nz <= 256.  The item list is built once per plan on the host (lowk_kx: kx of
// every listed low-|k| column, in list order); sched: spectral_fused_sched_words(nxh) zeroed words
// per launch.  *used = false when the shape or the arguments do not allow it.
bool spectral_fused_supported(int ny, int nz);
std::vector<int> spectral_fused_items(int nxh, int ny, int nz, const std::vector<int>& lowk_kx, int* nitems);
int spectral_fused_sched_words(int nxh);
cudaError_t launch_spectral_fused(const ThomasArgs& T, const Geom& g, const FftPlan& fy, const Tables& tb,
                                  const int* items, int nitems, unsigned* sched, cudaStream_t st, bool* used);

// q = p - p0 (float) from the stored double iterate, before a second or third sweep (skipped when done).
cudaError_t launch_q_rebuild(const double* p, const float* p0, float* q, long long n, const int* done,
                             cudaStream_t st);
cudaError_t launch_control(Stats* st_dev, const double* partials, int nblocks, const double* res_partials,
                           int res_nblocks, int pass, int max_sweeps, double tol, const double* floor,
                           long long npoints, int wrote_p, cudaStream_t st);
// Verification after the column solves of sweep n >= 2 (before its inverse transforms): the norm of
// the correction delta_n, from the solved half spectrum by Parseval (sq = per-CTA sums of
// w |x|^2, w = 1 for kx = 0 and nx/2, 2 otherwise; ||delta_n||^2 = nx ny sum w |x|^2), bounds the
// error of the current iterate p_{n-1}: ||e_{n-1}|| <= ||delta_n||/(1 - phi), taken as
// 2 ||delta_n|| (phi <= 1/2), or ||delta_n||/(1 - phi) with the measured contraction
// phi = ||delta_n||/||delta_{n-1}|| when that exceeds 1/2.  When the bound is at most tol the
// refinement stops on p_{n-1} (done; p still to be written when pass n-1 stored only q).  res_partials:
// the sweep's residual norms (its forward x-pass).  p_stored: that x-pass also stored p_{n-1} as p.
// inv_lcut2 > 0: the columns were solved only for the low wavenumbers (kx, |ky'| <= kcut) and the rest
// of ||delta_n||^2 is bounded by (W_max/W_min) ||r||^2/lambda_cut^2 (inv_lcut2 = 1/lambda_cut^2, the
// weight ratio from floor[1]); verify_cut in api.cu picks kcut.  from_r0: the sweep's residual was
// formed as r0 - L q from the previous sweep's FP32 residual r0 (ResidualArgs::r0); the bound then adds
// 2^-24 ||r0|| G/||p|| for r0's rounding and takes ||S|| from the previous sweep.
cudaError_t launch_verify(Stats* st_dev, const double* sq, int nsq, const double* res_partials, int res_nblocks,
                          int pass, double tol, const double* floor, double nxny, int p_stored, double inv_lcut2,
                          int from_r0, cudaStream_t st);
// p = p0 + q (double) when the refinement stopped after a sweep that stored only q (Stats::need_final).
cudaError_t launch_finalize(const float* p0, const float* q, double* p, long long n, const Stats* stats,
                            cudaStream_t st);
// Inside a captured CUDA graph: sets conditional handle h to 1 while the refinement is not done
// (*done == 0), else 0, so that the IF node that follows runs its body (a refinement sweep) only
// while the solve still needs it.
cudaError_t launch_set_if_not_done(cudaGraphConditionalHandle h, const int* done, cudaStream_t st);
// Zeroes `bytes` (a multiple of 4) at p with a kernel on stream st.
cudaError_t launch_zero_words(void* p, size_t bytes, cudaStream_t st);
// Four ints from src to dst by a one-thread kernel (dst may be mapped host memory).
cudaError_t launch_copy_status(const int* src, int* dst, cudaStream_t st);
// Conjugate gradients for a density varying in x, y and z (cg_kernels.cu).
enum CgOp { CG_WMEAN = 0, CG_START, CG_APPLY, CG_UPDATE, CG_DOTS, CG_DIR, CG_SUM, CG_SHIFT, CG_FACES };
struct CgLevel {      // per-level constants, so that no FP64 division runs per point
  double dz;          // dz_k
  double idz;         // 1/dz_k
  double hup;         // 0.5/h_{k+1/2}; at the top 2/dz_k with p = 0 on the face, else 0
  double hdn;         // 0.5/h_{k-1/2}; 0 at the bottom
  double iwbar;       // 1/(rho0_k dz_k), the preconditioner's weight
};
struct CgKernels {
  int nx, ny, nz;
  double idx2, idy2;
  int top_dirichlet;
};
struct CgArgs {
  const double* rho;    // [nz][ny][nx] density
  const double* S;      // source
  const double* dz;     // level thicknesses (device)
  const CgLevel* lv;    // per-level constants (device, nz entries)
  float2* ce;           // face coefficients of W A as float pairs: east, north, upper (CG_FACES writes them)
  float2* cn;
  float2* cu;
  double* p;            // iterate
  double* r;            // residual of K p = b
  double* d;            // search direction
  double* q;            // K d
  double* t;            // preconditioner source -r/Wbar
  const double* z;      // preconditioned residual
  double* partials;     // 2 doubles per block
  double scalar;        // mu, alpha, beta or shift
  double inv_snorm;     // 1/||S|| (CG_UPDATE: the residual norm comes out relative)
  int flag;             // CG_DIR: beta is zero
};
CgKernels cg_kernels(int nx, int ny, int nz, double dx, double dy, int top_dirichlet);
cudaError_t cg_launch(int op, const CgKernels& K, const CgArgs& a, int nb, cudaStream_t st);
int cg_blocks();
unsigned cg_grid(const CgKernels& K, int nb);

// dst[b][m][a] = src[a][m][b]: [nx][ny][nz] <-> [nz][ny][nx] field layouts (elem_bytes 4 or 8).
cudaError_t launch_swap_outer_inner(const void* src, void* dst, int A, int M, int B, int elem_bytes,
                                    cudaStream_t st);
cudaError_t launch_coefficients(const double* dz, const double* rho0, int nz, double* a_d, double* c_d,
                                double* W_d, float* a_f, float* c_f, float2* a_ff, float2* c_ff, int top_dirichlet,
                                cudaStream_t st);
// ---- persistent multi-domain solve of the mixed path (batch_persistent.cu) ----
// One domain as the batch hands it over: its plan's geometry, tables and options, its fields
// and its workspace (spectrum, p0, q, Stats).
struct BatchDomIn {
  Geom g;
  const Tables* tb;
  float2 cx, cy;            // double-float 1/dx^2, 1/dy^2
  int lowk_r2, n_lowk, singular00;
  const int2* lowk_cols;
  const double* lowk_inv;   // the plan's pivot table of the listed columns
  int max_sweeps, verify;
  double tol;
  const double* S;
  double* p;
  float2* spec;
  float* p0;
  float* q;
  Stats* stats;
};
// Device tables of one batch configuration (descriptors and item list, owned by the batch) and
// the ticket in the caller's workspace.
struct BatchPersistent {
  void* doms = nullptr;
  void* items = nullptr;
  int n = 0, nitems = 0, stall_dom = -1;
  size_t smem = 0;
  unsigned* ticket = nullptr;
};
// Shapes the persistent kernel takes: nx in {64, 128, 256, 384, 512}, ny in {64, 128, 256, 384, 512},
// 2 <= nz <= 128.
bool batch_persistent_supported(int nx, int ny, int nz);
// Workspace scratch (ticket, per-domain counters and partial sums) for the given domains.
size_t batch_persistent_scratch_bytes(const std::vector<BatchDomIn>& d);
// Builds the descriptors and the item list (host, synchronous copies); scratch: the workspace
// region of batch_persistent_scratch_bytes.  stall_dom >= 0: test hook, the first control item of
// that domain waits for a count that never arrives (its bounded wait runs out).  0 on success.
int batch_persistent_build(BatchPersistent* bp, const std::vector<BatchDomIn>& d, char* scratch, int stall_dom);
// The initialisation kernel (Stats, counters, ticket) and the persistent kernel, stream-ordered.
cudaError_t batch_persistent_launch(const BatchPersistent& bp, cudaStream_t st);
void batch_persistent_free(BatchPersistent* bp);

// Pivot reciprocals 1/u_k of the listed low-|k| columns ([n][nz], double), which depend only on the
// column's wavenumbers and the levels: built once per plan (and per poisson_plan_set_rho0) so that the
// double column solves run their recurrences without a division on the dependency chain.
cudaError_t launch_lowk_pivots(const int2* cols, int n, const double* a_d, const double* c_d, const double* lamx_d,
                               const double* lamy_d, int nz, int singular00, double* inv_tab, cudaStream_t st);
// Limiting accuracy F of the mixed refinement from the plan's coefficients (one block; nz <= 512):
// the relative error that the double-float residual's rounding leaves after any number of sweeps,
// added to every error bound.  Written to out[0]; out[1] = max_k W_k / min_k W_k (the bound on the
// vertical solve's non-normality that the low-wavenumber verification uses); out[2] = G, the factor
// by which a residual noise of 2-norm e reaches the solution (e G), so that F = u K ||p|| G/||p||.
cudaError_t launch_accuracy_floor(const double* a_d, const double* c_d, const double* W_d, int nz, int nx, int ny,
                                  double dx, double dy, int top_dirichlet, double* out, cudaStream_t st);
cudaError_t launch_grho(int kind /*0 double, 1 float, 2 double fields float math*/, const void* g, const void* p, const Geom& g_, const Tables& tb,
                        const double* dz, const double* rho0, double* partials, int nparts_max,
                        double* grho, cudaStream_t st);

// Persistent FP32 x-pass for the half lengths xpass_static_supported accepts; *used is
// false (and nothing is launched) when the shape or alignment does not allow it.
bool xpass_static_supported(int n_half);
cudaError_t launch_xfwd_static(int ti_is_double, const void* in, void* spec, const Geom& g, const FftPlan& fx,
                               const Tables& tb, const int* done, unsigned* err, cudaStream_t st, bool* used);
cudaError_t launch_xres_static(const ResidualArgs& R, void* spec, const Geom& g, const FftPlan& fx, const Tables& tb,
                               const int* done, unsigned* err, int* nblocks_out, cudaStream_t st, bool* used);
cudaError_t launch_xinv_static(int to_is_double, int mode, const void* spec, void* out, const Geom& g,
                               const FftPlan& fx, const Tables& tb, const XinvExtra& ex, int* nblocks_out,
                               cudaStream_t st, bool* used);

// Persistent FP32 y-pass with the compile-time FFT for power-of-two ny in [64, 2048].
bool ypass_static_supported(int ny);
// variant 0: two-slot ring + scratch tile; 1: two-slot ring, in place; 2: one tile, in place, two CTAs/SM.
cudaError_t launch_yfft_static(int sign, void* spec, const Geom& g, const FftPlan& fy, const Tables& tb, int tile,
                               int variant, const int* done, unsigned* err, cudaStream_t st, bool* used);

// Upper bound on the CTAs (and so partial-sum slots) of the x-pass launches of one field.
int xpass_blocks(const Geom& g, const FftPlan& fx, size_t csize);

// Elements per thread the FFT kernels are instantiated for.
bool fft_e_supported(int E);

}  // namespace pgb
