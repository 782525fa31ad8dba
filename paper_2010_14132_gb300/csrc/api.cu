// C ABI of the direct FFT pressure solver: plan construction (twiddles,
// eigenvalue and coefficient tables, workspace layout) and the launch sequence
// of each call.  Section 2.1: plan once, execute every timestep.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "../../include/poisson.h"
#include "kernels.cuh"

using namespace pgb;

namespace {

thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char* where, int line = 0) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s (api.cu:%d): %s", where, line, cudaGetErrorString(e));
  return POISSON_ERR_CUDA;
}
#define PGB_CUDA(call)                                             \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call, __LINE__);  \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool factor23(int n, int& a, int& b) {
  a = b = 0;
  if (n < 1) return false;
  while (n % 2 == 0) { n /= 2; ++a; }
  while (n % 3 == 0) { n /= 3; ++b; }
  return n == 1;
}

// Radix schedule and elements-per-thread for a line of length n = 2^a 3^b.
// e_pow2: elements per thread for pure powers of two (8 or 16).
bool make_fft_plan(int n, FftPlan& fp, int e_pow2 = 16) {
  int a, b;
  if (n < 2 || !factor23(n, a, b)) return false;
  std::memset(&fp, 0, sizeof(fp));
  fp.n = n;
  int s = 0;
  for (int i = 0; i < b; ++i) fp.radix[s++] = 3;
  for (int i = 0; i < a / 3; ++i) fp.radix[s++] = 8;
  if (a % 3 == 1) fp.radix[s++] = 2;
  if (a % 3 == 2) fp.radix[s++] = 4;
  if (s > kMaxStages) return false;
  fp.nstages = s;
  if (b == 0) fp.E = n < e_pow2 ? n : e_pow2;
  else fp.E = a >= 3 ? 24 : (a == 2 ? 12 : (a == 1 ? 6 : 3));
  return n % fp.E == 0 && fft_e_supported(fp.E);
}

int signed_k(int k, int n) { return k > n / 2 ? k - n : k; }

}  // namespace


// Optional per-phase CUDA-event timing (POISSON_OPT_PROFILE): events recorded on
// the launching stream around each kernel launch, summed on read.
struct PhaseProfiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> phase;   // phase of event pair i (events 2i, 2i+1)
  size_t used = 0;
};

struct poisson_plan {
  int nx = 0, ny = 0, nz = 0, nxh = 0, P = 0;
  double dx = 0, dy = 0;
  int dtype = 0;
  int bc = POISSON_BC_PERIODIC_XY_NEUMANN_Z;
  int layout = POISSON_LAYOUT_Z_Y_X;   // caller's field layout (the solver works on [nz][ny][nx])
  std::vector<double> dz, rho0;
  FftPlan fx{}, fy{};
  int lowk_r2 = 64, max_sweeps = 3, ytile = 0, ykernel = 4, xkernel = 0, xelems = 8, yelems = 16, lchunk = 0,
      coltile = 0, fused = 0, respass = 0, verify = 1;
  unsigned version = 0;   // bumped by every option change (invalidates captured batch graphs)
  // Set by a batch while it captures its graph: the stream into which each later refinement sweep is
  // captured as the body of a graph IF node (run only while the solve is not done); null otherwise.
  cudaStream_t cond_body = nullptr;
  // POISSON_OPT_GRAPH: the plan's own captured solves, keyed by their field and workspace pointers
  struct SolveGraph {
    const void* S;
    void* p;
    void* ws;
    unsigned version;
    unsigned long long used;
    cudaGraphExec_t exec;
  };
  static constexpr size_t kGraphs = 4;
  int use_graph = 1;
  std::vector<SolveGraph> graphs;
  unsigned long long graph_clock = 0;
  cudaStream_t gcap = nullptr, gbody = nullptr;
  double tol = 1e-10;
  Geom g{};
  Tables tb{};
  double* dz_d = nullptr;
  double* rho_d = nullptr;
  void* tables = nullptr;
  int2* lowk_d = nullptr;
  double* lowk_inv_d = nullptr;   // pivot reciprocals of the listed columns [n_lowk][nz] (launch_lowk_pivots)
  int n_lowk = 0;
  std::vector<int> lowk_kx;     // kx of every listed low-|k| column (host copy)
  int* mid_d = nullptr;         // item list of the fused spectral middle (device)
  int mid_nitems = 0;
  int sched_words = 0;          // per-pass scheduling counters of the fused middle
  float2 cx{}, cy{};
  // workspace layout
  size_t off_spec = 0, off_stats = 0, off_sched = 0, stats_bytes = 0, off_part = 0, off_rpart = 0, off_sqn = 0,
         off_r = 0, off_lz = 0, off_lw = 0, off_p0 = 0, off_q = 0,
         off_gp = 0, off_fa = 0, off_fb = 0, ws_bytes = 0;
  int xinv_blocks = 1, grho_nb = 1;
  PhaseProfiler prof;
  bool mixed() const { return dtype == POISSON_MIXED; }
  bool fp64() const { return dtype == POISSON_FP64; }
  int top_dirichlet() const { return bc == POISSON_BC_PERIODIC_XY_NEUMANN_BOTTOM_DIRICHLET_TOP ? 1 : 0; }
  size_t elem() const { return dtype == POISSON_FP32 ? 4 : 8; }
  size_t csize() const { return dtype == POISSON_FP64 ? 16 : 8; }
};

struct poisson_batch {
  static constexpr int kMaxBranches = 32;   // concurrent graph branches (POISSON_BATCH_OPT_BRANCHES)
  int n = 0;
  int dtype = 0;
  std::vector<poisson_plan*> plans;
  std::vector<size_t> off;
  size_t ws_bytes = 0;
  cudaStream_t cap = nullptr;
  cudaStream_t body = nullptr;   // captures the domains' conditional sweep bodies (one at a time)
  cudaStream_t branch[kMaxBranches] = {};
  cudaEvent_t fork = nullptr, join[kMaxBranches] = {};
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> capS;
  std::vector<void*> capP;
  std::vector<unsigned> capV;   // plan versions at capture
  void* capW = nullptr;
  int persistent = 0;           // POISSON_BATCH_OPT_PERSISTENT
  int stall_test = -1;          // POISSON_BATCH_OPT_STALL_TEST
  int branches = 24;            // POISSON_BATCH_OPT_BRANCHES
  BatchPersistent bp;           // descriptors and item list of the persistent kernel (when it is used)
};

namespace {

float2 split_host(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

int build_lowk(poisson_plan* pl) {
  std::vector<int2> cols;
  cols.push_back(make_int2(0, 0));
  const int r2 = pl->mixed() ? pl->lowk_r2 : 0;
  for (int ky = 0; ky < pl->ny; ++ky)
    for (int kx = 0; kx < pl->nxh; ++kx) {
      if (kx == 0 && ky == 0) continue;
      const int ks = signed_k(ky, pl->ny);
      if (kx * kx + ks * ks <= r2) cols.push_back(make_int2(kx, ky));
    }
  if (pl->lowk_d) cudaFree(pl->lowk_d);
  pl->lowk_d = nullptr;
  PGB_CUDA(cudaMalloc(&pl->lowk_d, cols.size() * sizeof(int2)));
  PGB_CUDA(cudaMemcpy(pl->lowk_d, cols.data(), cols.size() * sizeof(int2), cudaMemcpyHostToDevice));
  pl->n_lowk = (int)cols.size();
  pl->lowk_kx.clear();
  for (const int2& c : cols) pl->lowk_kx.push_back(c.x);
  if (pl->lowk_inv_d) cudaFree(pl->lowk_inv_d);
  pl->lowk_inv_d = nullptr;
  PGB_CUDA(cudaMalloc(&pl->lowk_inv_d, (size_t)pl->n_lowk * pl->nz * sizeof(double)));
  PGB_CUDA(launch_lowk_pivots(pl->lowk_d, pl->n_lowk, pl->tb.a_d, pl->tb.c_d, pl->tb.lamx_d, pl->tb.lamy_d, pl->nz,
                              !pl->top_dirichlet(), pl->lowk_inv_d, 0));
  PGB_CUDA(cudaStreamSynchronize(0));
  return POISSON_OK;
}

// Item list of the fused spectral middle (float spectra of a supported shape; rebuilt with the
// low-|k| list).
int build_mid(poisson_plan* pl) {
  if (pl->mid_d) cudaFree(pl->mid_d);
  pl->mid_d = nullptr;
  pl->mid_nitems = 0;
  if (pl->fp64() || !spectral_fused_supported(pl->ny, pl->nz)) return POISSON_OK;
  int n = 0;
  const std::vector<int> items = spectral_fused_items(pl->nxh, pl->ny, pl->nz, pl->lowk_kx, &n);
  if (n == 0) return POISSON_OK;
  PGB_CUDA(cudaMalloc(&pl->mid_d, items.size() * sizeof(int)));
  PGB_CUDA(cudaMemcpy(pl->mid_d, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice));
  pl->mid_nitems = n;
  return POISSON_OK;
}

void layout_workspace(poisson_plan* pl) {
  const long long N = pl->g.N;
  size_t off = 0;
  pl->off_spec = off;
  off = align256(off + (size_t)pl->nz * pl->g.plane * pl->csize());
  pl->off_stats = off;
  // the fused middle's scheduling counters (one set per pass of a solve) follow Stats, so one
  // zeroing kernel at the start of a solve clears both
  pl->sched_words = spectral_fused_sched_words(pl->nxh);
  pl->off_sched = off + ((sizeof(Stats) + 15) & ~(size_t)15);
  pl->stats_bytes = pl->off_sched - pl->off_stats + 4 * sizeof(unsigned) * (size_t)pl->sched_words;
  off = align256(off + pl->stats_bytes);
  pl->off_part = off;
  off = align256(off + 3 * sizeof(double) * (size_t)(pl->xinv_blocks + pl->nz));   // + one per level chunk
  pl->off_rpart = off;
  off = align256(off + 2 * sizeof(double) * (size_t)(pl->xinv_blocks + pl->nz));
  pl->off_sqn = off;   // per-CTA squared norms of a verification solve (column tiles of >= 16 columns)
  off = align256(off + sizeof(double) * (size_t)(pl->g.plane / 16 + 1 + pl->n_lowk));
  pl->off_lz = off;
  off = align256(off + sizeof(double2) * (size_t)pl->nz * pl->n_lowk);
  pl->off_lw = off;
  off = align256(off + sizeof(double) * (size_t)pl->nz * pl->n_lowk);
  if (pl->mixed()) {
    pl->off_p0 = off;
    off = align256(off + sizeof(float) * (size_t)N);
    pl->off_q = off;
    off = align256(off + sizeof(float) * (size_t)N);
    if (pl->respass && residual_stencil_supported(pl->nx, pl->ny)) {   // the sweep's residual r (float)
      pl->off_r = off;
      off = align256(off + sizeof(float) * (size_t)N);
    } else {
      pl->off_r = 0;
    }
  }
  pl->off_gp = off;
  off = align256(off + 2 * sizeof(double) * (size_t)(pl->nz - 1) * pl->grho_nb);
  if (pl->layout != POISSON_LAYOUT_Z_Y_X) {   // the caller's fields in the solver's layout
    pl->off_fa = off;
    off = align256(off + pl->elem() * (size_t)N);
    pl->off_fb = off;
    off = align256(off + pl->elem() * (size_t)N);
  }
  pl->ws_bytes = off;
}

// Device fields are read and written with 16-byte vector accesses (two points at a time).
bool field_aligned(const void* f) { return ((uintptr_t)f & 15) == 0; }

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

}  // namespace


namespace {

int prof_begin(poisson_plan* pl, int phase, cudaStream_t st) {
  if (!pl->prof.on) return -1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
  PhaseProfiler& P = pl->prof;
  if (2 * (P.used + 1) > P.pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      P.pool.push_back(e);
    }
  }
  if (P.phase.size() < P.used + 1) P.phase.resize(P.used + 1);
  const int slot = (int)P.used++;
  P.phase[slot] = phase;
  cudaEventRecord(P.pool[2 * slot], st);
  return slot;
}

void prof_end(poisson_plan* pl, int slot, cudaStream_t st) {
  if (slot >= 0) cudaEventRecord(pl->prof.pool[2 * slot + 1], st);
}

}  // namespace

extern "C" {

const char* poisson_status_string(int s) {
  switch (s) {
    case POISSON_OK: return "ok";
    case POISSON_ERR_INVALID_ARG: return "invalid argument";
    case POISSON_ERR_UNSUPPORTED: return "unsupported size";
    case POISSON_ERR_CUDA: return "CUDA error";
    case POISSON_ERR_WORKSPACE: return "bad workspace";
    case POISSON_ERR_NOT_CONVERGED: return "refinement did not reach its tolerance";
    case POISSON_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* poisson_last_error_detail(void) { return g_last_error; }

int poisson_plan_destroy(poisson_plan* pl) {
  if (!pl) return POISSON_OK;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : pl->prof.pool) cudaEventDestroy(e);
  for (auto& gr : pl->graphs) cudaGraphExecDestroy(gr.exec);
  if (pl->gcap) cudaStreamDestroy(pl->gcap);
  if (pl->gbody) cudaStreamDestroy(pl->gbody);
  if (pl->tables) cudaFree(pl->tables);
  if (pl->lowk_d) cudaFree(pl->lowk_d);
  if (pl->lowk_inv_d) cudaFree(pl->lowk_inv_d);
  if (pl->mid_d) cudaFree(pl->mid_d);
  delete pl;
  return POISSON_OK;
}

int poisson_plan_create(int nx, int ny, int nz, double dx, double dy, const double* dz, const double* rho0, int bc,
                        int dtype, poisson_plan** out) {
  if (!out) return POISSON_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dz || !rho0) return POISSON_ERR_INVALID_ARG;
  if (bc != POISSON_BC_PERIODIC_XY_NEUMANN_Z && bc != POISSON_BC_PERIODIC_XY_NEUMANN_BOTTOM_DIRICHLET_TOP)
    return POISSON_ERR_INVALID_ARG;
  if (dtype != POISSON_FP64 && dtype != POISSON_FP32 && dtype != POISSON_MIXED) return POISSON_ERR_INVALID_ARG;
  if (!(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy)) return POISSON_ERR_INVALID_ARG;
  for (int k = 0; k < nz; ++k)
    if (!(dz[k] > 0) || !(rho0[k] > 0) || !std::isfinite(dz[k]) || !std::isfinite(rho0[k]))
      return POISSON_ERR_INVALID_ARG;
  int a, b;
  if (nx < 4 || ny < 4 || nx > 4096 || ny > 4096 || nx % 2 != 0 || nz < 2 || nz > 512) return POISSON_ERR_UNSUPPORTED;
  if (!factor23(nx, a, b) || !factor23(ny, a, b)) return POISSON_ERR_UNSUPPORTED;

  poisson_plan* pl = new (std::nothrow) poisson_plan();
  if (!pl) return POISSON_ERR_CUDA;
  pl->nx = nx;
  pl->ny = ny;
  pl->nz = nz;
  pl->dx = dx;
  pl->dy = dy;
  pl->dtype = dtype;
  pl->bc = bc;
  pl->nxh = nx / 2 + 1;
  const int pad = dtype == POISSON_FP64 ? 8 : 16;  // 128-byte rows
  pl->P = (pl->nxh + pad - 1) / pad * pad;
  pl->dz.assign(dz, dz + nz);
  pl->rho0.assign(rho0, rho0 + nz);
  if (!make_fft_plan(nx / 2, pl->fx, pl->xelems) || !make_fft_plan(ny, pl->fy, pl->yelems)) {
    delete pl;
    return POISSON_ERR_UNSUPPORTED;
  }
  pl->g.nx = nx;
  pl->g.ny = ny;
  pl->g.nz = nz;
  pl->g.nxh = pl->nxh;
  pl->g.P = pl->P;
  pl->g.plane = (long long)ny * pl->P;
  pl->g.N = (long long)nx * ny * nz;
  pl->g.dx = dx;
  pl->g.dy = dy;
  pl->g.lev0 = 0;
  pl->g.lev1 = nz;
  pl->cx = split_host(1.0 / (dx * dx));
  pl->cy = split_host(1.0 / (dy * dy));

  // ---- host tables
  const int n = nx / 2;
  std::vector<double2> twx(n), twr(pl->nxh), twy(ny);
  for (int m = 0; m < n; ++m) twx[m] = make_double2(std::cos(2 * M_PI * m / n), -std::sin(2 * M_PI * m / n));
  for (int m = 0; m < pl->nxh; ++m) twr[m] = make_double2(std::cos(2 * M_PI * m / nx), -std::sin(2 * M_PI * m / nx));
  for (int m = 0; m < ny; ++m) twy[m] = make_double2(std::cos(2 * M_PI * m / ny), -std::sin(2 * M_PI * m / ny));
  std::vector<double> lx(pl->nxh), ly(ny);
  for (int k = 0; k < pl->nxh; ++k) {
    const double sn = std::sin(M_PI * k / nx);
    lx[k] = -(4.0 / (dx * dx)) * sn * sn;
  }
  for (int k = 0; k < ny; ++k) {
    // ky and ny - ky share one eigenvalue, bit for bit (the paired column solves use one pivot chain)
    const int kk = (k <= ny / 2) ? k : ny - k;
    const double sn = std::sin(M_PI * kk / ny);
    ly[k] = -(4.0 / (dy * dy)) * sn * sn;
  }

  // ---- one device block for all tables
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_a = take(nz * 8), o_c = take(nz * 8), o_W = take(nz * 8), o_af = take(nz * 4), o_cf = take(nz * 4),
               o_aff = take(nz * 8), o_cff = take(nz * 8), o_lxd = take(pl->nxh * 8),
               o_lyd = take(ny * 8), o_lxf = take(pl->nxh * 4), o_lyf = take(ny * 4), o_twxd = take(n * 16),
               o_twrd = take(pl->nxh * 16), o_twyd = take(ny * 16), o_twxf = take(n * 8), o_twrf = take(pl->nxh * 8),
               o_twyf = take(ny * 8), o_dz = take(nz * 8), o_rho = take(nz * 8), o_floor = take(32);
  cudaError_t e = cudaMalloc(&pl->tables, off);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaMalloc(tables)");
  }
  char* base = (char*)pl->tables;
  auto upd = [&](size_t o, const void* src, size_t bytes) {
    return cudaMemcpy(base + o, src, bytes, cudaMemcpyHostToDevice);
  };
  std::vector<float> lxf(pl->nxh), lyf(ny);
  std::vector<float2> twxf(n), twrf(pl->nxh), twyf(ny);
  for (int k = 0; k < pl->nxh; ++k) lxf[k] = (float)lx[k];
  for (int k = 0; k < ny; ++k) lyf[k] = (float)ly[k];
  for (int m = 0; m < n; ++m) twxf[m] = make_float2((float)twx[m].x, (float)twx[m].y);
  for (int m = 0; m < pl->nxh; ++m) twrf[m] = make_float2((float)twr[m].x, (float)twr[m].y);
  for (int m = 0; m < ny; ++m) twyf[m] = make_float2((float)twy[m].x, (float)twy[m].y);
  cudaError_t ce = cudaSuccess;
  if (ce == cudaSuccess) ce = upd(o_lxd, lx.data(), pl->nxh * 8);
  if (ce == cudaSuccess) ce = upd(o_lyd, ly.data(), ny * 8);
  if (ce == cudaSuccess) ce = upd(o_lxf, lxf.data(), pl->nxh * 4);
  if (ce == cudaSuccess) ce = upd(o_lyf, lyf.data(), ny * 4);
  if (ce == cudaSuccess) ce = upd(o_twxd, twx.data(), n * 16);
  if (ce == cudaSuccess) ce = upd(o_twrd, twr.data(), pl->nxh * 16);
  if (ce == cudaSuccess) ce = upd(o_twyd, twy.data(), ny * 16);
  if (ce == cudaSuccess) ce = upd(o_twxf, twxf.data(), n * 8);
  if (ce == cudaSuccess) ce = upd(o_twrf, twrf.data(), pl->nxh * 8);
  if (ce == cudaSuccess) ce = upd(o_twyf, twyf.data(), ny * 8);
  if (ce == cudaSuccess) ce = upd(o_dz, dz, nz * 8);
  if (ce == cudaSuccess) ce = upd(o_rho, rho0, nz * 8);
  Tables& tb = pl->tb;
  tb.a_d = (double*)(base + o_a);
  tb.c_d = (double*)(base + o_c);
  tb.W_d = (double*)(base + o_W);
  tb.a_f = (float*)(base + o_af);
  tb.c_f = (float*)(base + o_cf);
  tb.a_ff = (float2*)(base + o_aff);
  tb.c_ff = (float2*)(base + o_cff);
  tb.lamx_d = (double*)(base + o_lxd);
  tb.lamy_d = (double*)(base + o_lyd);
  tb.lamx_f = (float*)(base + o_lxf);
  tb.lamy_f = (float*)(base + o_lyf);
  tb.twx_d = (double2*)(base + o_twxd);
  tb.twr_d = (double2*)(base + o_twrd);
  tb.twy_d = (double2*)(base + o_twyd);
  tb.twx_f = (float2*)(base + o_twxf);
  tb.twr_f = (float2*)(base + o_twrf);
  tb.twy_f = (float2*)(base + o_twyf);
  tb.floor_d = (double*)(base + o_floor);
  pl->dz_d = (double*)(base + o_dz);
  pl->rho_d = (double*)(base + o_rho);
  if (ce == cudaSuccess)
    ce = launch_coefficients(pl->dz_d, pl->rho_d, nz, (double*)tb.a_d, (double*)tb.c_d, (double*)tb.W_d,
                             (float*)tb.a_f, (float*)tb.c_f, (float2*)tb.a_ff, (float2*)tb.c_ff, pl->top_dirichlet(), 0);
  if (ce == cudaSuccess)
    ce = launch_accuracy_floor(tb.a_d, tb.c_d, tb.W_d, nz, nx, ny, dx, dy, pl->top_dirichlet(), (double*)tb.floor_d, 0);
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  if (ce != cudaSuccess) {
    int rc = cuda_fail(ce, "plan tables");
    poisson_plan_destroy(pl);
    return rc;
  }
  int rc = build_lowk(pl);
  if (rc == POISSON_OK) rc = build_mid(pl);
  if (rc != POISSON_OK) {
    poisson_plan_destroy(pl);
    return rc;
  }
  {
    // x-pass block count (rows per CTA as chosen by the launcher)
    pl->xinv_blocks = xpass_blocks(pl->g, pl->fx, pl->csize());
    long long nb = ((long long)nx * ny + 255) / 256;
    pl->grho_nb = (int)(nb > 1024 ? 1024 : nb);
  }
  layout_workspace(pl);
  *out = pl;
  return POISSON_OK;
}

int poisson_plan_workspace_bytes(const poisson_plan* pl, size_t* bytes) {
  if (!pl || !bytes) return POISSON_ERR_INVALID_ARG;
  *bytes = pl->ws_bytes;
  return POISSON_OK;
}

int poisson_plan_set_option(poisson_plan* pl, int option, double value) {
  if (!pl) return POISSON_ERR_INVALID_ARG;
  pl->version++;
  switch (option) {
    case POISSON_OPT_LOWK_RADIUS2: {
      if (!(value >= 0) || value > 1e6) return POISSON_ERR_INVALID_ARG;
      pl->lowk_r2 = (int)value;
      int rc = build_lowk(pl);
      if (rc == POISSON_OK) rc = build_mid(pl);
      if (rc != POISSON_OK) return rc;
      layout_workspace(pl);
      return POISSON_OK;
    }
    case POISSON_OPT_MAX_SWEEPS:
      if (!(value >= 0 && value <= 3)) return POISSON_ERR_INVALID_ARG;
      pl->max_sweeps = (int)value;
      return POISSON_OK;
    case POISSON_OPT_TOLERANCE:
      if (!(value > 0 && value < 1)) return POISSON_ERR_INVALID_ARG;
      pl->tol = value;
      return POISSON_OK;
    case POISSON_OPT_Y_TILE:
      if (!(value >= 0 && value <= 64)) return POISSON_ERR_INVALID_ARG;
      pl->ytile = (int)value;
      return POISSON_OK;
    case POISSON_OPT_X_ELEMS:
    case POISSON_OPT_Y_ELEMS: {
      if (!(value == 8 || value == 16)) return POISSON_ERR_INVALID_ARG;
      FftPlan f{};
      const bool x = option == POISSON_OPT_X_ELEMS;
      if (!make_fft_plan(x ? pl->nx / 2 : pl->ny, f, (int)value)) return POISSON_ERR_UNSUPPORTED;
      if (x) {
        pl->xelems = (int)value;
        pl->fx = f;
        pl->xinv_blocks = xpass_blocks(pl->g, pl->fx, pl->csize());
        layout_workspace(pl);
      } else {
        pl->yelems = (int)value;
        pl->fy = f;
      }
      return POISSON_OK;
    }
    case POISSON_OPT_LEVEL_CHUNK:
      if (!(value >= 0 && value <= 4096)) return POISSON_ERR_INVALID_ARG;
      pl->lchunk = (int)value;
      return POISSON_OK;
    case POISSON_OPT_Y_KERNEL:
      if (!(value == 0 || value == 1 || value == 2 || value == 3 || value == 4)) return POISSON_ERR_INVALID_ARG;
      pl->ykernel = (int)value;
      return POISSON_OK;
    case POISSON_OPT_COL_TILE:
      if (!((value >= 0 && value <= 4 && value == (int)value) || value == 16 || value == 32 || value == 64 ||
            value == 128))
        return POISSON_ERR_INVALID_ARG;
      pl->coltile = (int)value;
      return POISSON_OK;
    case POISSON_OPT_X_KERNEL:
      if (!(value == 0 || value == 1)) return POISSON_ERR_INVALID_ARG;
      pl->xkernel = (int)value;
      return POISSON_OK;
    case POISSON_OPT_LAYOUT:
      if (!(value == POISSON_LAYOUT_Z_Y_X || value == POISSON_LAYOUT_X_Y_Z)) return POISSON_ERR_INVALID_ARG;
      pl->layout = (int)value;
      layout_workspace(pl);
      return POISSON_OK;
    case POISSON_OPT_SPECTRAL_FUSED:
      if (!(value == 0 || value == 1)) return POISSON_ERR_INVALID_ARG;
      pl->fused = (int)value;
      return POISSON_OK;
    case POISSON_OPT_VERIFY:
      if (!(value == 0 || value == 1 || value == 2)) return POISSON_ERR_INVALID_ARG;
      pl->verify = (int)value;
      return POISSON_OK;
    case POISSON_OPT_RESIDUAL_PASS:
      if (!(value == 0 || value == 1)) return POISSON_ERR_INVALID_ARG;
      pl->respass = (int)value;
      layout_workspace(pl);
      return POISSON_OK;
    case POISSON_OPT_PROFILE:
      if (!(value == 0 || value == 1)) return POISSON_ERR_INVALID_ARG;
      pl->prof.on = value != 0;
      pl->prof.used = 0;
      return POISSON_OK;
    case POISSON_OPT_GRAPH:
      if (!(value == 0 || value == 1)) return POISSON_ERR_INVALID_ARG;
      pl->use_graph = (int)value;
      return POISSON_OK;
    default:
      return POISSON_ERR_INVALID_ARG;
  }
}

int poisson_plan_profile_read(poisson_plan* pl, double* ms, int* launches, int nphases) {
  if (!pl || !ms || !launches || nphases < 0) return POISSON_ERR_INVALID_ARG;
  for (int i = 0; i < nphases; ++i) {
    ms[i] = 0;
    launches[i] = 0;
  }
  PhaseProfiler& P = pl->prof;
  for (size_t s = 0; s < P.used; ++s) {
    PGB_CUDA(cudaEventSynchronize(P.pool[2 * s + 1]));
    float t = 0;
    PGB_CUDA(cudaEventElapsedTime(&t, P.pool[2 * s], P.pool[2 * s + 1]));
    const int ph = P.phase[s];
    if (ph >= 0 && ph < nphases) {
      ms[ph] += t;
      launches[ph] += 1;
    }
  }
  P.used = 0;
  return POISSON_OK;
}

int poisson_plan_set_rho0(poisson_plan* pl, const double* rho0_dev, void* stream) {
  if (!pl || !rho0_dev) return POISSON_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  PGB_CUDA(cudaMemcpyAsync(pl->rho_d, rho0_dev, sizeof(double) * pl->nz, cudaMemcpyDeviceToDevice, st));
  const Tables& tb = pl->tb;
  PGB_CUDA(launch_coefficients(pl->dz_d, pl->rho_d, pl->nz, (double*)tb.a_d, (double*)tb.c_d, (double*)tb.W_d,
                               (float*)tb.a_f, (float*)tb.c_f, (float2*)tb.a_ff, (float2*)tb.c_ff,
                               pl->top_dirichlet(), st));
  PGB_CUDA(launch_accuracy_floor(tb.a_d, tb.c_d, tb.W_d, pl->nz, pl->nx, pl->ny, pl->g.dx, pl->g.dy,
                                 pl->top_dirichlet(), (double*)tb.floor_d, st));
  PGB_CUDA(launch_lowk_pivots(pl->lowk_d, pl->n_lowk, tb.a_d, tb.c_d, tb.lamx_d, tb.lamy_d, pl->nz,
                              !pl->top_dirichlet(), pl->lowk_inv_d, st));
  return POISSON_OK;
}

static int check_ws(const poisson_plan* pl, void* ws) {
  if (!ws) return POISSON_ERR_WORKSPACE;
  if (((uintptr_t)ws & 255) != 0) return POISSON_ERR_WORKSPACE;
  (void)pl;
  return POISSON_OK;
}

// y-pass: the persistent TMA kernel where the shape allows, else the plain one.
static cudaError_t ypass(poisson_plan* pl, const Geom& g, int sign, void* spec, const int* done, Stats* stats,
                         cudaStream_t st) {
  const bool t_double = pl->fp64();
  if ((pl->ykernel == 0 || pl->ykernel == 3 || pl->ykernel == 4) && !t_double) {
    bool used = false;
    const int variant = pl->ykernel == 3 ? 1 : (pl->ykernel == 4 ? 2 : 0);
    cudaError_t e = launch_yfft_static(sign, spec, g, pl->fy, pl->tb, pl->ytile, variant, done, &stats->err, st,
                                       &used);
    if (e != cudaSuccess || used) return e;
  }
  if (pl->ykernel == 0 || pl->ykernel == 2) {
    bool used = false;
    cudaError_t e = launch_yfft_tma(t_double, sign, spec, g, pl->fy, pl->tb, pl->ytile, done, stats, st, &used);
    if (e != cudaSuccess || used) return e;
  }
  return launch_yfft(t_double, sign, spec, g, pl->fy, pl->tb, pl->ytile, done, st);
}

// Levels per chunk of the transforms: x-pass and y-pass of a chunk run back to
// back, so the chunk's spectrum (about 32 MB by default) stays in L2 between them.
static int level_chunk(const poisson_plan* pl) {
  const int c = pl->lchunk <= 0 ? pl->nz : pl->lchunk;   // default: one chunk (all levels)
  return c < 1 ? 1 : (c > pl->nz ? pl->nz : c);
}

// Forward transform (chunked x-pass then y-pass) and column solve of one field.
// With a residual source R, *res_nblocks receives the number of per-block residual-norm
// partials the forward x-pass launches wrote (from R->part0 on).  pass: index of the pass
// within the solve (0 = first solve, n = sweep n).  *middle_fused is set when the fused
// spectral kernel ran the y-pass, the columns and the inverse y-pass (the inverse
// transform then runs its x-pass only).
static cudaError_t forward_columns(poisson_plan* pl, const void* in, int in_double, char* ws, cudaStream_t st,
                                   int adjoint, const int* done, const double* target_mean = nullptr,
                                   const ResidualArgs* R = nullptr, int* res_nblocks = nullptr, int pass = 0,
                                   bool* middle_fused = nullptr, double* sqnorm = nullptr,
                                   int* sqnorm_blocks = nullptr, bool* res_stored_p = nullptr, int kcut = -1) {
  const bool t_double = pl->fp64();
  void* spec = ws + pl->off_spec;
  Stats* stats = (Stats*)(ws + pl->off_stats);
  const int lc = level_chunk(pl);
  if (middle_fused) *middle_fused = false;
  if (res_stored_p) *res_stored_p = false;
  const bool try_fused = middle_fused && pl->fused && pl->mid_nitems > 0 && !adjoint && !t_double &&
                         lc >= pl->nz && pass >= 0 && pass < 4;
  cudaError_t e = cudaSuccess;
  int rparts = 0;
  for (int l0 = 0; l0 < pl->nz; l0 += lc) {
    Geom gc = pl->g;
    gc.lev0 = l0;
    gc.lev1 = l0 + lc < pl->nz ? l0 + lc : pl->nz;
    int ps = prof_begin(pl, POISSON_PHASE_XFWD, st);
    if (R) {
      bool used = false;
      ResidualArgs Rc = *R;
      Rc.part0 = R->part0 + rparts;
      int nb = 0;
      if (pl->respass && pl->off_r && pl->xkernel == 0 && lc >= pl->nz) {
        // the residual as its own pass into a float field, then the plain R2C x-pass of it
        float* r = (float*)(ws + pl->off_r);
        e = launch_residual_stencil(Rc, r, gc, done, &nb, st, &used);
        if (e == cudaSuccess && used) {
          bool xused = false;
          e = launch_xfwd_static(0, r, spec, gc, pl->fx, pl->tb, done, &stats->err, st, &xused);
          if (e == cudaSuccess && !xused) e = launch_xfwd(0, 0, r, spec, gc, pl->fx, pl->tb, done, st);
        }
      }
      bool stat = false;
      if (e == cudaSuccess && !used && pl->xkernel == 0) {
        e = launch_xres_static(Rc, spec, gc, pl->fx, pl->tb, done, &stats->err, &nb, st, &used);
        stat = used;
      }
      if (Rc.r0 && !stat) return cudaErrorNotSupported;   // the r0 - L q form exists in the static pass only
      if (res_stored_p && stat && Rc.q && Rc.p_out && lc >= pl->nz) *res_stored_p = true;
      Rc.p_out = nullptr;   // the other residual forms do not store the iterate
      if (e == cudaSuccess && !used) e = launch_xfwd_residual(Rc, spec, gc, pl->fx, pl->tb, done, &nb, st);
      rparts += nb;
    } else {
      bool used = false;
      if (!t_double && pl->xkernel == 0)
        e = launch_xfwd_static(in_double, in, spec, gc, pl->fx, pl->tb, done, &stats->err, st, &used);
      if (e == cudaSuccess && !used) e = launch_xfwd(in_double, t_double, in, spec, gc, pl->fx, pl->tb, done, st);
    }
    prof_end(pl, ps, st);
    if (e != cudaSuccess) return e;
    if (try_fused) continue;
    ps = prof_begin(pl, POISSON_PHASE_YFWD, st);
    Geom gy = gc;
    if (kcut >= 0) gy.nxh = kcut + 1;   // only the kx the low-wavenumber column solves need
    e = ypass(pl, gy, -1, spec, done, stats, st);
    prof_end(pl, ps, st);
    if (e != cudaSuccess) return e;
  }
  ThomasArgs A{};
  A.spec = spec;
  A.t_is_double = t_double;
  A.adjoint = adjoint;
  A.scale = 1.0 / ((double)pl->nx * pl->ny);
  A.lowk_r2 = pl->mixed() ? pl->lowk_r2 : 0;
  A.lowk_double = pl->mixed() || t_double;
  A.lowk_cols = pl->lowk_d;
  A.lowk_inv = A.lowk_double ? pl->lowk_inv_d : nullptr;
  A.singular00 = !pl->top_dirichlet();
  A.n_lowk = pl->n_lowk;
  A.lowk_z = (double2*)(ws + pl->off_lz);
  A.lowk_w = (double*)(ws + pl->off_lw);
  A.stats = stats;
  A.done = done;
  A.target_mean = target_mean;
  A.col_tile = pl->coltile;
  A.kcut = kcut;
  if (res_nblocks) *res_nblocks = rparts;
  if (sqnorm_blocks) *sqnorm_blocks = 0;
  if (try_fused) {
    bool used = false;
    unsigned* sched = (unsigned*)(ws + pl->off_sched) + (size_t)pass * pl->sched_words;
    int ps = prof_begin(pl, POISSON_PHASE_SPECTRAL, st);
    e = launch_spectral_fused(A, pl->g, pl->fy, pl->tb, pl->mid_d, pl->mid_nitems, sched, st, &used);
    prof_end(pl, ps, st);
    if (e != cudaSuccess) return e;
    if (used) {
      *middle_fused = true;
      return cudaSuccess;
    }
    ps = prof_begin(pl, POISSON_PHASE_YFWD, st);   // not launched: the separate y-pass after all
    e = ypass(pl, pl->g, -1, spec, done, stats, st);
    prof_end(pl, ps, st);
    if (e != cudaSuccess) return e;
  }
  A.sqnorm = sqnorm;
  A.sqnorm_blocks = sqnorm_blocks;
  const int ps = prof_begin(pl, POISSON_PHASE_COLUMNS, st);
  e = launch_thomas(A, pl->g, pl->tb, st);
  prof_end(pl, ps, st);
  return e;
}

// The low-wavenumber verification of sweep 1's iterate (POISSON_OPT_VERIFY = 1): the columns of the
// correction delta_2 with kx, |ky'| <= kcut = nx/8 are solved exactly (a y-pass of those kx only, the
// twisted column kernel restricted to them); every other column is (lambda_h + T)^{-1} of the
// residual's column with lambda_h >= lambda_cut and T = W^{-1} M similar to a positive semidefinite
// matrix through W^{1/2}, so its norm is at most sqrt(W_max/W_min)/lambda_cut times the residual
// column's.  ||delta_2||^2 <= ||delta_low||^2 + (W_max/W_min) ||r||^2/lambda_cut^2 is then an upper
// bound, and the verification test (verify_decide) takes it in place of the full norm.  -1 where the
// cut would not save work (small grids) or would leave low-|k| columns outside it.
static int verify_cut(const poisson_plan* pl, double* inv_lcut2) {
  *inv_lcut2 = 0.0;
  if (!pl->mixed() || pl->verify != 1 || pl->fused) return -1;
  const int kc = pl->nx / 8;
  int r = 0;
  while ((r + 1) * (r + 1) <= pl->lowk_r2) ++r;
  if (kc <= 8 || kc <= r || kc + 1 >= pl->nxh || 2 * kc + 1 >= pl->ny) return -1;
  const double sx = std::sin(M_PI * (kc + 1) / pl->nx), sy = std::sin(M_PI * (kc + 1) / pl->ny);
  const double lx = 4.0 / (pl->dx * pl->dx) * sx * sx, ly = 4.0 / (pl->dy * pl->dy) * sy * sy;
  const double lcut = lx < ly ? lx : ly;
  *inv_lcut2 = 1.0 / (lcut * lcut);
  return kc;
}

// Inverse transform (chunked y-pass then x-pass with the given epilogue);
// *nparts receives the number of partial-sum slots the x-pass launches wrote.
static cudaError_t inverse(poisson_plan* pl, char* ws, cudaStream_t st, const int* done, int to_double, int mode,
                           void* out, XinvExtra ex, int* nparts, bool* control_fused = nullptr,
                           bool skip_ypass = false) {
  if (control_fused) *control_fused = false;
  const bool t_double = pl->fp64();
  void* spec = ws + pl->off_spec;
  Stats* stats = (Stats*)(ws + pl->off_stats);
  const int lc = level_chunk(pl);
  int part = 0;
  cudaError_t e = cudaSuccess;
  for (int l0 = 0; l0 < pl->nz; l0 += lc) {
    Geom gc = pl->g;
    gc.lev0 = l0;
    gc.lev1 = l0 + lc < pl->nz ? l0 + lc : pl->nz;
    int ps = -1;
    if (!skip_ypass) {
      ps = prof_begin(pl, POISSON_PHASE_YINV, st);
      e = ypass(pl, gc, +1, spec, done, stats, st);
      prof_end(pl, ps, st);
      if (e != cudaSuccess) return e;
    }
    ex.part0 = part;
    int nb = 0;
    ps = prof_begin(pl, POISSON_PHASE_XINV, st);
    bool used = false;
    ex.err = &stats->err;
    XinvExtra exs = ex;
    // one chunk: the static kernel's last CTA runs the refinement control itself
    const bool fuse = control_fused && mode != XINV_PLAIN && lc >= pl->nz;
    if (!fuse) exs.ctl_stats = nullptr;
    if (!t_double && pl->xkernel == 0)
      e = launch_xinv_static(to_double, mode, spec, out, gc, pl->fx, pl->tb, exs, &nb, st, &used);
    if (used && fuse) *control_fused = true;
    if (e == cudaSuccess && !used) e = launch_xinv(t_double, to_double, mode, spec, out, gc, pl->fx, pl->tb, ex, &nb, st);
    prof_end(pl, ps, st);
    if (e != cudaSuccess) return e;
    part += nb;
  }
  if (nparts) *nparts = part;
  return e;
}

static int fill_info(poisson_plan* pl, char* ws, cudaStream_t st, poisson_info* info) {
  Stats s{};
  double floor = -1.0;
  PGB_CUDA(cudaMemcpyAsync(&s, ws + pl->off_stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
  if (pl->mixed()) PGB_CUDA(cudaMemcpyAsync(&floor, pl->tb.floor_d, sizeof(double), cudaMemcpyDeviceToHost, st));
  PGB_CUDA(cudaStreamSynchronize(st));
  std::memset(info, 0, sizeof(*info));
  info->accuracy_floor = floor;
  info->removed_weighted_mean = s.mu_w;
  if (s.err & ERR_WAIT_TIMEOUT) return POISSON_ERR_TIMEOUT;
  if (!pl->mixed()) {
    info->converged = 1;
    info->sweeps = 0;
    info->rel_update[0] = 1.0;
    info->error_estimate = -1.0;
    for (int i = 0; i < 4; ++i) info->rel_residual[i] = -1.0;
    return POISSON_OK;
  }
  info->sweeps = s.sweeps;
  info->converged = s.converged;
  for (int i = 0; i < 4; ++i) info->rel_update[i] = s.rel_update[i];
  for (int i = 0; i < 4; ++i) info->rel_residual[i] = s.sq_src[i] > 0 ? s.rel_residual[i] : -1.0;
  info->error_estimate = s.err_est;
  return s.converged ? POISSON_OK : POISSON_ERR_NOT_CONVERGED;
}

// [nx][ny][nz] (k fastest) <-> [nz][ny][nx] (i fastest)
static cudaError_t to_solver_layout(const poisson_plan* pl, const void* src, void* dst, cudaStream_t st) {
  return launch_swap_outer_inner(src, dst, pl->nx, pl->ny, pl->nz, (int)pl->elem(), st);
}
static cudaError_t from_solver_layout(const poisson_plan* pl, const void* src, void* dst, cudaStream_t st) {
  return launch_swap_outer_inner(src, dst, pl->nz, pl->ny, pl->nx, (int)pl->elem(), st);
}

// Capture of a refinement sweep as the body of a graph IF node (the capturing stream st gets a node
// that sets the condition from the device's done flag, then the IF node; the body is captured from the
// body stream until cond_end).  A certified solve then skips the sweep's kernels instead of launching
// them to return at once.
static cudaError_t cond_begin(cudaStream_t st, cudaStream_t body, const int* done) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = launch_set_if_not_done(h, done, st);
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, &edges, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, graph, deps, edges, nd, &np);
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(body, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
  return e;
}
static cudaError_t cond_end(cudaStream_t body) {
  cudaGraph_t g = nullptr;   // the IF node's body graph (owned by the node)
  return cudaStreamEndCapture(body, &g);
}

// A plan's captured solve for these pointers (captured now if the plan has none that is current, the
// least recently used one replaced beyond kGraphs), launched on st.  The sweeps after the first are IF
// nodes on the done flag (cond_body during the capture).
static int solve_graph(poisson_plan* pl, const void* S, void* p, void* ws, cudaStream_t st,
                       const std::function<int(cudaStream_t)>& solve_on) {
  poisson_plan::SolveGraph* hit = nullptr;
  for (auto& gr : pl->graphs)
    if (gr.S == S && gr.p == p && gr.ws == ws && gr.version == pl->version) hit = &gr;
  if (!hit) {
    if (!pl->gcap) PGB_CUDA(cudaStreamCreateWithFlags(&pl->gcap, cudaStreamNonBlocking));
    if (!pl->gbody) PGB_CUDA(cudaStreamCreateWithFlags(&pl->gbody, cudaStreamNonBlocking));
    PGB_CUDA(cudaStreamBeginCapture(pl->gcap, cudaStreamCaptureModeRelaxed));
    pl->cond_body = pl->gbody;
    const int rc = solve_on(pl->gcap);
    pl->cond_body = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(pl->gcap, &graph);
    if (rc != POISSON_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __LINE__);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate", __LINE__);
    // stale entries (older options) first, then the least recently used
    for (size_t i = 0; i < pl->graphs.size();)
      if (pl->graphs[i].version != pl->version) {
        cudaGraphExecDestroy(pl->graphs[i].exec);
        pl->graphs.erase(pl->graphs.begin() + i);
      } else {
        ++i;
      }
    if (pl->graphs.size() >= poisson_plan::kGraphs) {
      size_t lru = 0;
      for (size_t i = 1; i < pl->graphs.size(); ++i)
        if (pl->graphs[i].used < pl->graphs[lru].used) lru = i;
      cudaGraphExecDestroy(pl->graphs[lru].exec);   // freed once a launch in flight completes
      pl->graphs.erase(pl->graphs.begin() + lru);
    }
    pl->graphs.push_back({S, p, ws, pl->version, 0, exec});
    hit = &pl->graphs.back();
  }
  hit->used = ++pl->graph_clock;
  PGB_CUDA(cudaGraphLaunch(hit->exec, st));
  return POISSON_OK;
}

// The solve on fields in the solver's layout.
static int solve_fields(poisson_plan* pl, const void* S, void* p, char* ws, cudaStream_t st) {
  Stats* stats = (Stats*)(ws + pl->off_stats);
  PGB_CUDA(launch_zero_words(stats, pl->stats_bytes, st));
  const bool t_double = pl->fp64();
  XinvExtra ex{};
  ex.partials = (double*)(ws + pl->off_part);
  if (!pl->mixed()) {
    bool mid = false;
    PGB_CUDA(forward_columns(pl, S, t_double, ws, st, 0, nullptr, nullptr, nullptr, nullptr, 0, &mid));
    PGB_CUDA(inverse(pl, ws, st, nullptr, t_double, XINV_PLAIN, p, ex, nullptr, nullptr, mid));
  } else {
    const int* done = &stats->done;
    float* p0 = (float*)(ws + pl->off_p0);
    float* q = (float*)(ws + pl->off_q);
    int nb = 0;
    // first solve: double source, float transforms, double low-|k| columns
    bool mid = false;
    PGB_CUDA(forward_columns(pl, S, 1, ws, st, 0, nullptr, nullptr, nullptr, nullptr, 0, &mid));
    ex.p0 = p0;
    ex.p_out = pl->max_sweeps == 0 ? (double*)p : nullptr;
    ex.ctl_stats = stats;
    ex.ctl_max_sweeps = pl->max_sweeps;
    ex.ctl_tol = pl->tol;
    ex.ctl_floor = pl->tb.floor_d;
    ex.ctl_npoints = pl->g.N;
    ex.ctl_pass = 0;
    bool fused = false;
    PGB_CUDA(inverse(pl, ws, st, nullptr, 0, XINV_P0, p0, ex, &nb, &fused, mid));
    cudaError_t e = cudaSuccess;
    if (!fused) {
      int ps = prof_begin(pl, POISSON_PHASE_CONTROL, st);
      e = launch_control(stats, ex.partials, nb, nullptr, 0, 0, pl->max_sweeps, pl->tol, pl->tb.floor_d, pl->g.N,
                         ex.p_out != nullptr, st);
      prof_end(pl, ps, st);
      PGB_CUDA(e);
    }
    // Sweep 1 stores the correction q (and p only when it is the last sweep allowed); a later sweep
    // reads q and stores p.  If the refinement ends on sweep 1's iterate (the stopping rule after
    // sweep 1, or sweep 2's correction certifying it), k_finalize forms p = p0 + q.  A third sweep
    // first rebuilds q from the double iterate of the second.
    double* rpart = (double*)(ws + pl->off_rpart);
    // When sweep 2 starts with the low-wavenumber verification, sweep 1 keeps its residual r0 in FP32 in
    // the rows of p (row r's first nx floats; p is written in full later on every path) and the
    // verification forms r0 - L q from it instead of S - mu - L (p0 + q).
    double icut_unused = 0.0;
    const bool keep_r0 = pl->max_sweeps >= 2 && verify_cut(pl, &icut_unused) >= 0 && pl->xkernel == 0 &&
                         !pl->respass && level_chunk(pl) >= pl->nz && xpass_static_supported(pl->fx.n) &&
                         ((uintptr_t)p & 15) == 0;
    for (int sweep = 1; sweep <= pl->max_sweeps; ++sweep) {
      // residual computed inside the forward x-pass (its rows are never stored)
      ResidualArgs R{};
      R.partials = rpart;
      R.part0 = 0;
      R.S = (const double*)S;
      R.p0 = p0;
      R.q = sweep > 1 ? q : nullptr;
      R.a_ff = pl->tb.a_ff;
      R.c_ff = pl->tb.c_ff;
      R.cx = pl->cx;
      R.cy = pl->cy;
      R.mu_ff = &stats->mu_ff;
      R.r_ld = 2LL * pl->nx;
      if (sweep == 1 && keep_r0) R.r_out = (float*)p;
      int nres = 0, nsq = 0;
      // from the second sweep on, the correction's norm (Parseval on the solved spectrum) can already
      // certify the current iterate: then the sweep stops before its inverse transforms.  Sweep 2's
      // residual x-pass stores sweep 1's iterate p0 + q as p on the way, in case it does.
      double inv_lcut2 = 0.0;
      const int kcut = sweep == 2 ? verify_cut(pl, &inv_lcut2) : -1;
      if (kcut >= 0) {
        // first try: certify p_1 from the low-wavenumber columns of delta_2 and a bound on the rest; the
        // full sweep below then returns at once on the done flag (or runs, verifying again, if not)
        double* sqv = (double*)(ws + pl->off_sqn);
        ResidualArgs Rl = R;
        Rl.p_out = (double*)p;
        Rl.kmax = kcut;   // the residual's transform is read only up to kx = kcut
        if (keep_r0) Rl.r0 = (const float*)p;
        int nres_l = 0, nsq_l = 0;
        bool stored_l = false;
        PGB_CUDA(forward_columns(pl, nullptr, 0, ws, st, 0, done, &stats->pmean, &Rl, &nres_l, sweep, nullptr, sqv,
                                 &nsq_l, &stored_l, kcut));
        if (nsq_l > 0) {
          const int ps = prof_begin(pl, POISSON_PHASE_CONTROL, st);
          e = launch_verify(stats, sqv, nsq_l, rpart, nres_l, sweep, pl->tol, pl->tb.floor_d,
                            (double)pl->nx * pl->ny, stored_l ? 1 : 0, inv_lcut2, keep_r0 ? 1 : 0, st);
          prof_end(pl, ps, st);
          PGB_CUDA(e);
        }
      }
      // From sweep 2 on, inside a batch's graph capture, the sweep is the body of an IF node on the done
      // flag; elsewhere its kernels read the flag and return at once when the solve is already done.
      const bool cond = sweep >= 2 && pl->cond_body != nullptr;
      if (cond) PGB_CUDA(cond_begin(st, pl->cond_body, done));
      cudaStream_t ss = cond ? pl->cond_body : st;
      auto run_sweep = [&]() -> int {
        if (sweep > 2) {
          const int ps = prof_begin(pl, POISSON_PHASE_RESIDUAL, ss);
          const cudaError_t eq = launch_q_rebuild((const double*)p, p0, q, pl->g.N, done, ss);
          prof_end(pl, ps, ss);
          PGB_CUDA(eq);
        }
        double* sqn = (pl->verify && sweep >= 2) ? (double*)(ws + pl->off_sqn) : nullptr;
        R.p_out = (sqn && sweep == 2) ? (double*)p : nullptr;
        bool stored = false;
        PGB_CUDA(forward_columns(pl, nullptr, 0, ws, ss, 0, done, &stats->pmean, &R, &nres, sweep, &mid, sqn, &nsq,
                                 &stored));
        if (sqn && nsq > 0) {
          const int ps = prof_begin(pl, POISSON_PHASE_CONTROL, ss);
          e = launch_verify(stats, sqn, nsq, rpart, nres, sweep, pl->tol, pl->tb.floor_d, (double)pl->nx * pl->ny,
                            stored ? 1 : 0, 0.0, 0, ss);
          prof_end(pl, ps, ss);
          PGB_CUDA(e);
        }
        const bool last_allowed = sweep == pl->max_sweeps;
        XinvExtra eu = ex;
        eu.p0 = p0;
        eu.q = q;
        eu.q_valid = sweep > 1;
        eu.q_out = (sweep == 1 && !last_allowed) ? q : nullptr;
        eu.p_out = (sweep == 1 && !last_allowed) ? nullptr : (double*)p;
        eu.done = done;
        eu.ctl_pass = sweep;
        eu.res_partials = rpart;
        eu.res_nblocks = nres;
        PGB_CUDA(inverse(pl, ws, ss, done, 0, XINV_UPDATE, nullptr, eu, &nb, &fused, mid));
        if (!fused) {
          int ps = prof_begin(pl, POISSON_PHASE_CONTROL, ss);
          e = launch_control(stats, ex.partials, nb, rpart, nres, sweep, pl->max_sweeps, pl->tol, pl->tb.floor_d,
                             pl->g.N, eu.p_out != nullptr, ss);
          prof_end(pl, ps, ss);
          PGB_CUDA(e);
        }
        return POISSON_OK;
      };
      const int rc_sweep = run_sweep();
      if (cond) {   // end the body's capture even after an error, so that the stream is usable again
        const cudaError_t ce = cond_end(pl->cond_body);
        if (rc_sweep != POISSON_OK) return rc_sweep;
        PGB_CUDA(ce);
      } else if (rc_sweep != POISSON_OK) {
        return rc_sweep;
      }
    }
    if (pl->max_sweeps >= 2) {
      // p = p0 + q when the refinement ended on sweep 1's iterate (stopped after sweep 1, or verified by
      // sweep 2's correction); a no-op otherwise
      int ps = prof_begin(pl, POISSON_PHASE_CONTROL, st);
      e = launch_finalize(p0, q, (double*)p, pl->g.N, stats, st);
      prof_end(pl, ps, st);
      PGB_CUDA(e);
    }
  }
  return POISSON_OK;
}

int poisson_solve(poisson_plan* pl, const void* S, void* p, void* workspace, void* stream, poisson_info* info) {
  if (!pl || !S || !p) return POISSON_ERR_INVALID_ARG;
  if (!field_aligned(S) || !field_aligned(p)) return POISSON_ERR_INVALID_ARG;
  int rc = check_ws(pl, workspace);
  if (rc != POISSON_OK) return rc;
  const size_t fbytes = (size_t)pl->g.N * pl->elem();
  if (ranges_overlap(S, fbytes, p, fbytes)) return POISSON_ERR_INVALID_ARG;
  if (ranges_overlap(S, fbytes, workspace, pl->ws_bytes) || ranges_overlap(p, fbytes, workspace, pl->ws_bytes))
    return POISSON_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  auto solve_on = [&](cudaStream_t s) -> int {
    if (pl->layout == POISSON_LAYOUT_Z_Y_X) return solve_fields(pl, S, p, ws, s);
    void* Sa = ws + pl->off_fa;
    void* pb = ws + pl->off_fb;
    PGB_CUDA(to_solver_layout(pl, S, Sa, s));
    int r = solve_fields(pl, Sa, pb, ws, s);
    if (r == POISSON_OK) PGB_CUDA(from_solver_layout(pl, pb, p, s));
    return r;
  };
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {   // e.g. the legacy stream during another capture
    (void)cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;                  // plain launches then
  }
  if (pl->mixed() && pl->use_graph && !pl->prof.on && pl->max_sweeps >= 2 && cs == cudaStreamCaptureStatusNone) {
    rc = solve_graph(pl, S, p, workspace, st, solve_on);
  } else {
    rc = solve_on(st);
  }
  if (rc != POISSON_OK) return rc;
  if (info) return fill_info(pl, ws, st, info);
  return POISSON_OK;
}

int poisson_solve_adjoint(poisson_plan* pl, const void* gp, const void* p, void* gS, double* grho, void* workspace,
                          void* stream) {
  if (!pl || !gp || !gS) return POISSON_ERR_INVALID_ARG;
  if (grho && !p) return POISSON_ERR_INVALID_ARG;
  if (!field_aligned(gp) || !field_aligned(gS) || (p && !field_aligned(p))) return POISSON_ERR_INVALID_ARG;
  int rc = check_ws(pl, workspace);
  if (rc != POISSON_OK) return rc;
  const size_t fbytes = (size_t)pl->g.N * pl->elem();
  if (ranges_overlap(gp, fbytes, gS, fbytes)) return POISSON_ERR_INVALID_ARG;
  if (p && grho && ranges_overlap(p, fbytes, gS, fbytes)) return POISSON_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  Stats* stats = (Stats*)(ws + pl->off_stats);
  PGB_CUDA(launch_zero_words(stats, sizeof(Stats), st));
  const bool t_double = pl->fp64();
  const int io_double = pl->dtype != POISSON_FP32;
  const bool swap = pl->layout != POISSON_LAYOUT_Z_Y_X;
  void* fa = ws + pl->off_fa;
  void* gS_s = swap ? (void*)(ws + pl->off_fb) : gS;
  if (swap) PGB_CUDA(to_solver_layout(pl, gp, fa, st));
  PGB_CUDA(forward_columns(pl, swap ? fa : gp, io_double, ws, st, 1, nullptr));
  XinvExtra ex{};
  PGB_CUDA(inverse(pl, ws, st, nullptr, io_double, XINV_PLAIN, gS_s, ex, nullptr));
  if (grho) {
    const int kind = pl->fp64() ? 0 : (pl->dtype == POISSON_FP32 ? 1 : 2);
    if (swap) PGB_CUDA(to_solver_layout(pl, p, fa, st));   // gp's copy is no longer read
    PGB_CUDA(launch_grho(kind, gS_s, swap ? fa : p, pl->g, pl->tb, pl->dz_d, pl->rho_d, (double*)(ws + pl->off_gp),
                         pl->grho_nb, grho, st));
  }
  if (swap) PGB_CUDA(from_solver_layout(pl, gS_s, gS, st));
  return POISSON_OK;
}

// ---------------------------------------------------------------------------
// Preconditioned conjugate gradients for a density varying in x, y and z, with
// this plan's direct solve (its rho0 profile) as the preconditioner.
// ---------------------------------------------------------------------------
struct CgLayout {
  size_t off_r, off_d, off_q, off_t, off_z, off_part, off_lv, off_ce, off_cn, off_cu, bytes;
};
static CgLayout cg_layout(const poisson_plan* pl) {
  CgLayout L{};
  const size_t f = align256(sizeof(double) * (size_t)pl->g.N);
  size_t off = align256(pl->ws_bytes);
  L.off_r = off;
  off += f;
  L.off_d = off;
  off += f;
  L.off_q = off;
  off += f;
  L.off_t = off;
  off += f;
  L.off_z = off;
  off += f;
  L.off_part = off;
  off += align256(2 * sizeof(double) * (size_t)cg_blocks());
  L.off_lv = off;
  off += align256(sizeof(CgLevel) * (size_t)pl->nz);
  const size_t fc = align256(sizeof(float2) * (size_t)pl->g.N);   // face coefficients as float pairs
  L.off_ce = off;
  off += fc;
  L.off_cn = off;
  off += fc;
  L.off_cu = off;
  off += fc;
  L.bytes = off;
  return L;
}

int poisson_cg_workspace_bytes(const poisson_plan* pl, size_t* bytes) {
  if (!pl || !bytes) return POISSON_ERR_INVALID_ARG;
  *bytes = cg_layout(pl).bytes;
  return POISSON_OK;
}

// Sum the two-per-block partials of the last reduction on the host, in block order.
static int cg_sums(const double* partials_dev, unsigned nb, cudaStream_t st, double* s0, double* s1) {
  std::vector<double> h(2 * (size_t)nb);
  PGB_CUDA(cudaMemcpyAsync(h.data(), partials_dev, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  PGB_CUDA(cudaStreamSynchronize(st));
  double a = 0, b = 0;
  for (unsigned i = 0; i < nb; ++i) {
    a += h[2 * i];
    b += h[2 * i + 1];
  }
  *s0 = a;
  if (s1) *s1 = b;
  return POISSON_OK;
}

int poisson_cg_solve(poisson_plan* pl, const double* rho3, const double* S, double* p, double tol, int max_iter,
                     void* workspace, void* stream, poisson_cg_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!pl || !rho3 || !S || !p) return POISSON_ERR_INVALID_ARG;
  if (!field_aligned(rho3) || !field_aligned(S) || !field_aligned(p)) return POISSON_ERR_INVALID_ARG;
  if (pl->dtype == POISSON_FP32 || pl->layout != POISSON_LAYOUT_Z_Y_X) return POISSON_ERR_UNSUPPORTED;
  if (!(tol > 0) || max_iter < 1) return POISSON_ERR_INVALID_ARG;
  int rc = check_ws(pl, workspace);
  if (rc != POISSON_OK) return rc;
  const CgLayout L = cg_layout(pl);
  const size_t fbytes = sizeof(double) * (size_t)pl->g.N;
  if (ranges_overlap(S, fbytes, p, fbytes) || ranges_overlap(rho3, fbytes, p, fbytes) ||
      ranges_overlap(S, fbytes, workspace, L.bytes) || ranges_overlap(p, fbytes, workspace, L.bytes) ||
      ranges_overlap(rho3, fbytes, workspace, L.bytes))
    return POISSON_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const CgKernels K = cg_kernels(pl->nx, pl->ny, pl->nz, pl->dx, pl->dy, pl->top_dirichlet());
  const int nbmax = cg_blocks();
  const unsigned nb = cg_grid(K, nbmax);
  CgArgs a{};
  a.rho = rho3;
  a.S = S;
  a.dz = pl->dz_d;
  {
    // per-level constants; the preconditioner's weights come from the plan's device table (set_rho0)
    const int nz = pl->nz;
    std::vector<double> Wb(nz);
    PGB_CUDA(cudaMemcpyAsync(Wb.data(), pl->tb.W_d, sizeof(double) * nz, cudaMemcpyDeviceToHost, st));
    PGB_CUDA(cudaStreamSynchronize(st));
    std::vector<CgLevel> lv(nz);
    for (int k = 0; k < nz; ++k) {
      const double dzk = pl->dz[k];
      lv[k].dz = dzk;
      lv[k].idz = 1.0 / dzk;
      lv[k].hup = (k + 1 < nz) ? 0.5 / (0.5 * (dzk + pl->dz[k + 1])) : (pl->top_dirichlet() ? 1.0 / (0.5 * dzk) : 0.0);
      lv[k].hdn = (k > 0) ? 0.5 / (0.5 * (dzk + pl->dz[k - 1])) : 0.0;
      lv[k].iwbar = 1.0 / Wb[k];
    }
    CgLevel* lv_d = (CgLevel*)(ws + L.off_lv);
    PGB_CUDA(cudaMemcpyAsync(lv_d, lv.data(), sizeof(CgLevel) * nz, cudaMemcpyHostToDevice, st));
    PGB_CUDA(cudaStreamSynchronize(st));   // lv is a local vector
    a.lv = lv_d;
  }
  a.ce = (float2*)(ws + L.off_ce);
  a.cn = (float2*)(ws + L.off_cn);
  a.cu = (float2*)(ws + L.off_cu);
  PGB_CUDA(cg_launch(CG_FACES, K, a, nbmax, st));
  a.p = p;
  a.r = (double*)(ws + L.off_r);
  a.d = (double*)(ws + L.off_d);
  a.q = (double*)(ws + L.off_q);
  a.t = (double*)(ws + L.off_t);
  a.z = (const double*)(ws + L.off_z);
  a.partials = (double*)(ws + L.off_part);
  double* z = (double*)(ws + L.off_z);
  double s0 = 0, s1 = 0;
  // compatibility: with zero flux at the top remove mu_W = sum W S / sum W
  double mu = 0;
  if (!pl->top_dirichlet()) {
    PGB_CUDA(cg_launch(CG_WMEAN, K, a, nbmax, st));
    if ((rc = cg_sums(a.partials, nb, st, &s0, &s1)) != POISSON_OK) return rc;
    mu = s1 > 0 ? s0 / s1 : 0.0;
  }
  a.scalar = mu;
  PGB_CUDA(cg_launch(CG_START, K, a, nbmax, st));
  if ((rc = cg_sums(a.partials, nb, st, &s0, nullptr)) != POISSON_OK) return rc;
  const double snorm = std::sqrt(s0);
  double rel = snorm > 0 ? 1.0 : 0.0;
  a.inv_snorm = snorm > 0 ? 1.0 / snorm : 0.0;
  int it = 0;
  bool conv = snorm == 0;
  if (!conv) {
    // z = M r, d = z, rz = r . z
    if ((rc = solve_fields(pl, a.t, z, ws, st)) != POISSON_OK) return rc;
    a.q = nullptr;
    PGB_CUDA(cg_launch(CG_DOTS, K, a, nbmax, st));
    a.q = (double*)(ws + L.off_q);
    if ((rc = cg_sums(a.partials, nb, st, &s0, nullptr)) != POISSON_OK) return rc;
    double rz = s0;
    a.flag = 1;
    PGB_CUDA(cg_launch(CG_DIR, K, a, nbmax, st));
    a.flag = 0;
    for (it = 1; it <= max_iter; ++it) {
      PGB_CUDA(cg_launch(CG_APPLY, K, a, nbmax, st));
      if ((rc = cg_sums(a.partials, nb, st, &s0, nullptr)) != POISSON_OK) return rc;
      if (!(s0 > 0)) break;   // d in the null space (or a breakdown): nothing left to reduce
      const double alpha = rz / s0;
      a.scalar = alpha;
      PGB_CUDA(cg_launch(CG_UPDATE, K, a, nbmax, st));
      if ((rc = cg_sums(a.partials, nb, st, &s0, nullptr)) != POISSON_OK) return rc;
      rel = std::sqrt(s0);   // the update kernel's sum is already relative to ||S||
      if (rel <= tol) {
        conv = true;
        break;
      }
      if (it == max_iter) break;
      if ((rc = solve_fields(pl, a.t, z, ws, st)) != POISSON_OK) return rc;
      PGB_CUDA(cg_launch(CG_DOTS, K, a, nbmax, st));
      if ((rc = cg_sums(a.partials, nb, st, &s0, &s1)) != POISSON_OK) return rc;
      const double beta = -alpha * s1 / rz;   // Polak-Ribiere: z_new . (r_new - r_old) / (r_old . z_old)
      rz = s0;
      a.scalar = beta;
      PGB_CUDA(cg_launch(CG_DIR, K, a, nbmax, st));
    }
    if (it > max_iter) it = max_iter;
  }
  if (!pl->top_dirichlet()) {   // plain mean zero, as the direct solve
    PGB_CUDA(cg_launch(CG_SUM, K, a, nbmax, st));
    if ((rc = cg_sums(a.partials, nb, st, &s0, nullptr)) != POISSON_OK) return rc;
    a.scalar = s0 / (double)pl->g.N;
    PGB_CUDA(cg_launch(CG_SHIFT, K, a, nbmax, st));
  }
  if (info) {
    info->iterations = it;
    info->converged = conv ? 1 : 0;
    info->rel_residual = rel;
    info->removed_weighted_mean = mu;
  }
  return conv ? POISSON_OK : POISSON_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// Batched solve: per-domain plans; the launch sequence of all domains is
// captured once into a CUDA graph and replayed with one graph launch.
// ---------------------------------------------------------------------------
int poisson_batch_destroy(poisson_batch* b) {
  if (!b) return POISSON_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  batch_persistent_free(&b->bp);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->body) cudaStreamDestroy(b->body);
  for (int k = 0; k < poisson_batch::kMaxBranches; ++k) {
    if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto* p : b->plans) poisson_plan_destroy(p);
  delete b;
  return POISSON_OK;
}

int poisson_batch_create(int n, const int* nx, const int* ny, const int* nz, const double* dx, const double* dy,
                         const double* const* dz, const double* const* rho0, int dtype, poisson_batch** out) {
  if (!out) return POISSON_ERR_INVALID_ARG;
  *out = nullptr;
  if (n <= 0 || !nx || !ny || !nz || !dx || !dy || !dz || !rho0) return POISSON_ERR_INVALID_ARG;
  if (dtype != POISSON_FP32 && dtype != POISSON_MIXED) return POISSON_ERR_INVALID_ARG;
  poisson_batch* b = new (std::nothrow) poisson_batch();
  if (!b) return POISSON_ERR_CUDA;
  b->n = n;
  b->dtype = dtype;
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    poisson_plan* pl = nullptr;
    int rc = poisson_plan_create(nx[i], ny[i], nz[i], dx[i], dy[i], dz[i], rho0[i], POISSON_BC_PERIODIC_XY_NEUMANN_Z,
                                 dtype, &pl);
    if (rc != POISSON_OK) {
      poisson_batch_destroy(b);
      return rc;
    }
    b->plans.push_back(pl);
    b->off.push_back(off);
    off = align256(off + pl->ws_bytes);
  }
  b->ws_bytes = off;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->body, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int k = 0; k < poisson_batch::kMaxBranches && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    poisson_batch_destroy(b);
    return cuda_fail(e, "cudaStreamCreate");
  }
  *out = b;
  return POISSON_OK;
}

// Workspace offsets of the domains (plans' workspace sizes change with their options).
static void batch_layout(poisson_batch* b) {
  size_t off = 0;
  for (int i = 0; i < b->n; ++i) {
    b->off[i] = off;
    off = align256(off + b->plans[i]->ws_bytes);
  }
  b->ws_bytes = off;
}

// The persistent kernel takes the batch: mixed precision, every domain of a supported shape in the
// solver's own layout.
static bool batch_uses_persistent(const poisson_batch* b) {
  if (!b->persistent || b->dtype != POISSON_MIXED) return false;
  for (const poisson_plan* pl : b->plans)
    if (!batch_persistent_supported(pl->nx, pl->ny, pl->nz) || pl->layout != POISSON_LAYOUT_Z_Y_X) return false;
  return true;
}

static std::vector<BatchDomIn> batch_dom_inputs(const poisson_batch* b, const void* const* S, void* const* p,
                                                char* ws) {
  std::vector<BatchDomIn> d(b->n);
  for (int i = 0; i < b->n; ++i) {
    const poisson_plan* pl = b->plans[i];
    char* w = ws ? ws + b->off[i] : nullptr;
    BatchDomIn& in = d[i];
    in.g = pl->g;
    in.g.lev0 = 0;
    in.g.lev1 = pl->nz;
    in.tb = &pl->tb;
    in.cx = pl->cx;
    in.cy = pl->cy;
    in.lowk_r2 = pl->lowk_r2;
    in.n_lowk = pl->n_lowk;
    in.singular00 = !pl->top_dirichlet();
    in.lowk_cols = pl->lowk_d;
    in.lowk_inv = pl->lowk_inv_d;
    in.max_sweeps = pl->max_sweeps;
    in.verify = pl->verify;
    in.tol = pl->tol;
    in.S = S ? (const double*)S[i] : nullptr;
    in.p = p ? (double*)p[i] : nullptr;
    in.spec = w ? (float2*)(w + pl->off_spec) : nullptr;
    in.p0 = w ? (float*)(w + pl->off_p0) : nullptr;
    in.q = w ? (float*)(w + pl->off_q) : nullptr;
    in.stats = w ? (Stats*)(w + pl->off_stats) : nullptr;
  }
  return d;
}

int poisson_batch_set_option(poisson_batch* b, int option, double value) {
  if (!b) return POISSON_ERR_INVALID_ARG;
  if (option == POISSON_BATCH_OPT_PERSISTENT) {
    if (value != 0.0 && value != 1.0) return POISSON_ERR_INVALID_ARG;
    b->persistent = (int)value;
  } else if (option == POISSON_BATCH_OPT_STALL_TEST) {
    if (value != std::floor(value) || value < -1.0 || value >= (double)b->n) return POISSON_ERR_INVALID_ARG;
    b->stall_test = (int)value;
  } else if (option == POISSON_BATCH_OPT_BRANCHES) {
    if (value != std::floor(value) || value < 1.0 || value > (double)poisson_batch::kMaxBranches)
      return POISSON_ERR_INVALID_ARG;
    b->branches = (int)value;
  } else {
    return POISSON_ERR_INVALID_ARG;
  }
  if (b->exec) {   // the next solve re-captures
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return POISSON_OK;
}

int poisson_batch_plan(poisson_batch* b, int i, poisson_plan** out) {
  if (!b || !out || i < 0 || i >= b->n) return POISSON_ERR_INVALID_ARG;
  *out = b->plans[i];
  return POISSON_OK;
}

int poisson_batch_workspace_bytes(const poisson_batch* b, size_t* bytes) {
  if (!b || !bytes) return POISSON_ERR_INVALID_ARG;
  size_t off = 0;   // the domains' current workspace sizes (options can change them)
  for (int i = 0; i < b->n; ++i) off = align256(off + b->plans[i]->ws_bytes);
  if (batch_uses_persistent(b))   // the persistent kernel's counters and partial sums follow
    off = align256(off + batch_persistent_scratch_bytes(batch_dom_inputs(b, nullptr, nullptr, nullptr)));
  *bytes = off;
  return POISSON_OK;
}

int poisson_batch_solve(poisson_batch* b, const void* const* S, void* const* p, void* workspace, void* stream,
                        poisson_info* info) {
  if (!b || !S || !p) return POISSON_ERR_INVALID_ARG;
  if (!workspace || ((uintptr_t)workspace & 255)) return POISSON_ERR_WORKSPACE;
  for (int i = 0; i < b->n; ++i)
    if (!S[i] || !p[i] || !field_aligned(S[i]) || !field_aligned(p[i])) return POISSON_ERR_INVALID_ARG;
  bool same = b->exec && b->capW == workspace;
  if (same)
    for (int i = 0; i < b->n; ++i)
      same = same && b->capS[i] == S[i] && b->capP[i] == p[i] && b->capV[i] == b->plans[i]->version;
  if (!same) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    batch_layout(b);
    if (batch_uses_persistent(b)) {
      // one persistent kernel over every domain's work items, captured with its initialisation
      const std::vector<BatchDomIn> in = batch_dom_inputs(b, S, p, (char*)workspace);
      if (batch_persistent_build(&b->bp, in, (char*)workspace + b->ws_bytes, b->stall_test) != 0)
        return cuda_fail(cudaErrorInvalidValue, "batch_persistent_build", __LINE__);
      PGB_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
      const cudaError_t le = batch_persistent_launch(b->bp, b->cap);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
      if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le, "batch_persistent_launch", __LINE__);
      }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      b->capS.assign(S, S + b->n);
      b->capP.assign(p, p + b->n);
      b->capV.resize(b->n);
      for (int i = 0; i < b->n; ++i) b->capV[i] = b->plans[i]->version;
      b->capW = workspace;
    }
  }
  if (!same && !b->exec) {
    batch_persistent_free(&b->bp);
    // domains largest first, each to the least-loaded of the concurrent branches; a domain's load is its
    // points plus a fixed 2M for the latency-bound part of its launch chain (about 0.1 ms of a branch)
    std::vector<int> order(b->n);
    for (int i = 0; i < b->n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->plans[x]->g.N > b->plans[y]->g.N; });
    const int nbr = b->n < b->branches ? b->n : b->branches;
    std::vector<long long> load(nbr, 0);
    std::vector<int> branch_of(b->n, 0);
    for (int i : order) {
      int best = 0;
      for (int k = 1; k < nbr; ++k)
        if (load[k] < load[best]) best = k;
      branch_of[i] = best;
      load[best] += b->plans[i]->g.N + (1ll << 21);
    }
    PGB_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    int rc = POISSON_OK;
    cudaError_t ce = cudaEventRecord(b->fork, b->cap);
    for (int k = 0; k < nbr && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
    for (int i : order) {
      if (rc != POISSON_OK || ce != cudaSuccess) break;
      // a domain's refinement sweeps after the first become IF nodes on its done flag
      b->plans[i]->cond_body = b->body;
      rc = poisson_solve(b->plans[i], S[i], p[i], (char*)workspace + b->off[i], b->branch[branch_of[i]], nullptr);
      b->plans[i]->cond_body = nullptr;
    }
    for (int k = 0; k < nbr && ce == cudaSuccess; ++k) {
      ce = cudaEventRecord(b->join[k], b->branch[k]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->cap, b->join[k], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (ce != cudaSuccess && rc == POISSON_OK) rc = cuda_fail(ce, "batch capture branches", __LINE__);
    if (rc != POISSON_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    b->capS.assign(S, S + b->n);
    b->capP.assign(p, p + b->n);
    b->capV.resize(b->n);
    for (int i = 0; i < b->n; ++i) b->capV[i] = b->plans[i]->version;
    b->capW = workspace;
  }
  PGB_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  if (info) {
    int first = POISSON_OK;
    for (int i = 0; i < b->n; ++i) {
      int rc = fill_info(b->plans[i], (char*)workspace + b->off[i], (cudaStream_t)stream, &info[i]);
      if (rc != POISSON_OK && first == POISSON_OK) first = rc;
    }
    return first;
  }
  return POISSON_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Host-buffer pipeline: two device slots, three streams (copy in, compute,
// copy out) ordered by events, so that copies of neighbouring steps overlap
// the solve of the current one.
// ---------------------------------------------------------------------------
struct poisson_pipe {
  poisson_plan* plan = nullptr;
  size_t field_bytes = 0;
  void* ws = nullptr;
  void* dS[2] = {nullptr, nullptr};
  void* dp[2] = {nullptr, nullptr};
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  bool slot_used[2] = {false, false};
  long long submitted = 0, since_wait = 0;
  int first_status = POISSON_OK;
  // per-step (done, sweeps, converged, err) copied from the device statistics after each solve
  static constexpr int kRing = 1024;
  int4* status_ring = nullptr;   // page-locked and mapped, kRing entries
  int4* status_ring_dev = nullptr;   // the same ring as the device addresses it
};

int poisson_pipe_destroy(poisson_pipe* pp) {
  if (!pp) return POISSON_OK;
  if (pp->s_in) cudaStreamSynchronize(pp->s_in);
  if (pp->s_comp) cudaStreamSynchronize(pp->s_comp);
  if (pp->s_out) cudaStreamSynchronize(pp->s_out);
  for (int k = 0; k < 2; ++k) {
    if (pp->ev_in[k]) cudaEventDestroy(pp->ev_in[k]);
    if (pp->ev_comp[k]) cudaEventDestroy(pp->ev_comp[k]);
    if (pp->ev_out[k]) cudaEventDestroy(pp->ev_out[k]);
    if (pp->dS[k]) cudaFree(pp->dS[k]);
    if (pp->dp[k]) cudaFree(pp->dp[k]);
  }
  if (pp->ws) cudaFree(pp->ws);
  if (pp->status_ring) cudaFreeHost(pp->status_ring);
  if (pp->s_in) cudaStreamDestroy(pp->s_in);
  if (pp->s_comp) cudaStreamDestroy(pp->s_comp);
  if (pp->s_out) cudaStreamDestroy(pp->s_out);
  delete pp;
  return POISSON_OK;
}

int poisson_pipe_create(poisson_plan* pl, poisson_pipe** out) {
  if (!pl || !out) return POISSON_ERR_INVALID_ARG;
  *out = nullptr;
  poisson_pipe* pp = new (std::nothrow) poisson_pipe();
  if (!pp) return POISSON_ERR_CUDA;
  pp->plan = pl;
  pp->field_bytes = (size_t)pl->g.N * pl->elem();
  cudaError_t e = cudaMalloc(&pp->ws, pl->ws_bytes);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaMalloc(&pp->dS[k], pp->field_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&pp->dp[k], pp->field_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pp->ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pp->ev_comp[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pp->ev_out[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaHostAlloc(&pp->status_ring, sizeof(int4) * poisson_pipe::kRing, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&pp->status_ring_dev, pp->status_ring, 0);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pp->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pp->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pp->s_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    poisson_pipe_destroy(pp);
    return cuda_fail(e, "poisson_pipe_create", __LINE__);
  }
  *out = pp;
  return POISSON_OK;
}

int poisson_pipe_submit(poisson_pipe* pp, const void* S_host, void* p_host) {
  if (!pp || !S_host || !p_host) return POISSON_ERR_INVALID_ARG;
  const int k = (int)(pp->submitted & 1);
  // source slot k is free once the solve that read it two submissions ago is done; solution slot k
  // once that step's copy-out is done (so a copy-in and the previous copy-out run concurrently)
  if (pp->slot_used[k]) PGB_CUDA(cudaStreamWaitEvent(pp->s_in, pp->ev_comp[k], 0));
  PGB_CUDA(cudaMemcpyAsync(pp->dS[k], S_host, pp->field_bytes, cudaMemcpyHostToDevice, pp->s_in));
  PGB_CUDA(cudaEventRecord(pp->ev_in[k], pp->s_in));
  PGB_CUDA(cudaStreamWaitEvent(pp->s_comp, pp->ev_in[k], 0));
  if (pp->slot_used[k]) PGB_CUDA(cudaStreamWaitEvent(pp->s_comp, pp->ev_out[k], 0));
  const int st = poisson_solve(pp->plan, pp->dS[k], pp->dp[k], pp->ws, pp->s_comp, nullptr);
  if (st != POISSON_OK && pp->first_status == POISSON_OK) pp->first_status = st;
  static_assert(offsetof(Stats, err) == offsetof(Stats, done) + 3 * sizeof(int), "status fields not contiguous");
  // the step's status goes to the host ring by a one-thread kernel (stores into mapped host memory): a
  // copy here would queue on the copy engine behind the previous step's solution copy and hold the
  // compute stream, and with it the next solve, until that copy ends
  PGB_CUDA(launch_copy_status((const int*)((char*)pp->ws + pp->plan->off_stats + offsetof(Stats, done)),
                              (int*)&pp->status_ring_dev[pp->since_wait % poisson_pipe::kRing], pp->s_comp));
  pp->since_wait++;
  PGB_CUDA(cudaEventRecord(pp->ev_comp[k], pp->s_comp));
  PGB_CUDA(cudaStreamWaitEvent(pp->s_out, pp->ev_comp[k], 0));
  PGB_CUDA(cudaMemcpyAsync(p_host, pp->dp[k], pp->field_bytes, cudaMemcpyDeviceToHost, pp->s_out));
  PGB_CUDA(cudaEventRecord(pp->ev_out[k], pp->s_out));
  pp->slot_used[k] = true;
  pp->submitted++;
  return st;
}

int poisson_pipe_wait(poisson_pipe* pp) {
  if (!pp) return POISSON_ERR_INVALID_ARG;
  PGB_CUDA(cudaStreamSynchronize(pp->s_in));
  PGB_CUDA(cudaStreamSynchronize(pp->s_comp));
  PGB_CUDA(cudaStreamSynchronize(pp->s_out));
  int st = pp->first_status;
  const long long n = pp->since_wait < poisson_pipe::kRing ? pp->since_wait : poisson_pipe::kRing;
  for (long long i = 0; i < n && st == POISSON_OK; ++i) {
    const int4 r = pp->status_ring[i];   // (done, sweeps, converged, err)
    if ((unsigned)r.w & ERR_WAIT_TIMEOUT) st = POISSON_ERR_TIMEOUT;
    else if (pp->plan->mixed() && !r.z) st = POISSON_ERR_NOT_CONVERGED;
  }
  pp->first_status = POISSON_OK;
  pp->since_wait = 0;
  return st;
}
