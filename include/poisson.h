/*
 * poisson.h -- C ABI of the GB300 direct FFT pressure solver.
 *
 * The solver computes the pressure p of the elliptic pressure equation of Poisson type that
 * a dynamical core solves every timestep (Brown, "A comparison of techniques
 * for solving the Poisson equation in CFD", Section 2), by the direct method of
 * Section 2.1: a forward real Fourier transform over the periodic x/y plane at
 * every level, an independent tridiagonal solve per (kx, ky) wavenumber column,
 * and a backward transform.  Planning happens once and the plan is reused every
 * solve (the FFTW-style plan-once idea of Section 2.1).
 *
 * Discretisation (the paper names the equation but prints no stencil; this is
 * the reading the library implements):
 *   (L p)_ijk = (p_{i+1}-2p_i+p_{i-1})/dx^2 + (p_{j+1}-2p_j+p_{j-1})/dy^2
 *             + a_k (p_{k-1}-p_k) + c_k (p_{k+1}-p_k)
 *   W_k = rho0_k dz_k, a_k = rho_{k-1/2}/(W_k h_{k-1/2}), c_k = rho_{k+1/2}/(W_k h_{k+1/2}),
 *   h_{k+1/2} = (dz_k + dz_{k+1})/2, rho_{k+1/2} = (rho0_k + rho0_{k+1})/2,
 *   a_0 = 0 (zero flux through the bottom face), periodic in x and y; at the top
 *   face either zero flux, c_{nz-1} = 0 (POISSON_BC_PERIODIC_XY_NEUMANN_Z), or
 *   p = 0 on the face (POISSON_BC_PERIODIC_XY_NEUMANN_BOTTOM_DIRICHLET_TOP):
 *   c_{nz-1} = rho0_{nz-1}/(W_{nz-1} dz_{nz-1}/2), i.e. the face density taken
 *   from the top cell and the half-cell distance to the face.
 * With zero flux at the top the solve returns the unique p with
 * L p = S - mu_W  and plain mean zero, mu_W = sum W_k S_ijk / (nx ny sum W_k)
 * (the part of S outside the range of L).  With p = 0 on the top face L is
 * nonsingular and the solve returns p = L^-1 S (nothing is projected or pinned).
 *
 * Memory conventions (all calls):
 *   - fields are C-contiguous [nz][ny][nx] arrays, x fastest, in DEVICE memory
 *     (or [nx][ny][nz], z fastest, with POISSON_OPT_LAYOUT = POISSON_LAYOUT_X_Y_Z);
 *   - element type: double for POISSON_FP64 and POISSON_MIXED, float for POISSON_FP32;
 *   - device fields start on a 16-byte boundary (the kernels move two points per access;
 *     cudaMalloc and torch allocations always do): POISSON_ERR_INVALID_ARG otherwise;
 *   - the caller owns every field and the workspace; the plan owns only its small
 *     device tables (coefficients, twiddles), allocated by create, freed by destroy;
 *   - every call is asynchronous on the given CUDA stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream) unless it fills a poisson_info, in which
 *     case it synchronises that stream before returning;
 *   - one plan + one workspace must not be used by two calls in flight at once;
 *   - no call throws; every call returns a poisson_status.
 */
#ifndef POISSON_GB300_H
#define POISSON_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct poisson_plan poisson_plan;    /* opaque, owned by the library */
typedef struct poisson_batch poisson_batch;  /* opaque, owned by the library */
typedef struct poisson_pipe poisson_pipe;    /* opaque, owned by the library */

typedef enum {
  POISSON_OK = 0,
  POISSON_ERR_INVALID_ARG = -1,    /* null pointer, aliasing, non-positive spacing, bad enum */
  POISSON_ERR_UNSUPPORTED = -2,    /* size not of the supported form (see poisson_plan_create) */
  POISSON_ERR_CUDA = -3,           /* a CUDA runtime call failed (allocation, launch, copy) */
  POISSON_ERR_WORKSPACE = -4,      /* workspace pointer NULL or not 256-byte aligned */
  POISSON_ERR_NOT_CONVERGED = -5,  /* mixed path: refinement stopped above its tolerance; p is written */
  POISSON_ERR_TIMEOUT = -6         /* a bounded device-side wait gave up: a kernel's wait for its own
                                      asynchronous copies, or a persistent kernel's wait on a work
                                      counter, ran out of polls; the kernel stopped and flagged it */
} poisson_status;

/* Vertical boundary conditions (x and y are always periodic). */
typedef enum {
  POISSON_BC_PERIODIC_XY_NEUMANN_Z = 0,                  /* zero flux through the bottom and top faces */
  POISSON_BC_PERIODIC_XY_NEUMANN_BOTTOM_DIRICHLET_TOP = 1 /* zero flux at the bottom, p = 0 on the top face */
} poisson_bc;

typedef enum {
  POISSON_FP64 = 0,   /* all arithmetic in double */
  POISSON_FP32 = 1,   /* all arithmetic in float */
  POISSON_MIXED = 2   /* double in/out; float transforms; double low-|k| columns;
                         double-float residual and iterative refinement */
} poisson_dtype;

/* Plan options (poisson_plan_set_option). */
typedef enum {
  POISSON_OPT_LOWK_RADIUS2 = 0,  /* mixed: columns with kx^2 + ky'^2 <= value (ky' signed) use
                                    double; default 64 (|k| <= 8); the (0,0) column always does */
  POISSON_OPT_MAX_SWEEPS = 1,    /* mixed: refinement sweeps after the first solve, 0..3; default 3 */
  POISSON_OPT_TOLERANCE = 2,     /* mixed: the refinement stops once its error bound (error_estimate of
                                    poisson_info) is at most this relative L2 error; default 1e-10.  A
                                    tolerance below the plan's accuracy_floor is never met */
  POISSON_OPT_Y_TILE = 3,        /* y-pass kx tile width (autotuner hook); 0 = plan default (8 for the
                                    FP32 compile-time-FFT kernels) */
  POISSON_OPT_PROFILE = 4,       /* 1: record CUDA events around every kernel launch of this plan on
                                    the launching stream (read with poisson_plan_profile_read) */
  POISSON_OPT_Y_KERNEL = 5,      /* y-pass kernel: 0 = persistent TMA-staged kernel where the shape
                                    allows, with the compile-time FFT for FP32 and ny in {64, ..., 2048}
                                    of the form 2^a 3^b; 1 = plain shared-memory tile kernel;
                                    2 = persistent TMA-staged kernel with the run-time FFT;
                                    3 = as 0, transforming in place in the TMA tile (two barriers per
                                    stage, a third less shared memory); 4 (default) = one tile per CTA,
                                    in place, two CTAs per SM, the next tile's load overlapping this
                                    tile's stores (16 elements per thread; otherwise as 0) */
  POISSON_OPT_X_ELEMS = 6,       /* x-pass elements per thread for power-of-two lines: 8 (default) or 16 */
  POISSON_OPT_Y_ELEMS = 7,       /* y-pass elements per thread for power-of-two lines: 8 or 16 (default) */
  POISSON_OPT_LEVEL_CHUNK = 8,   /* levels per transform chunk (x-pass and y-pass of a chunk run back to
                                    back so its spectrum stays in L2); 0 = all levels in one chunk
                                    (default: the persistent kernels lose more to per-launch start-up
                                    than L2 reuse gains) */
  POISSON_OPT_X_KERNEL = 9,      /* x-pass kernel of the FP32 transforms: 0 = persistent kernel with bulk-copy
                                    staging where nx/2 is a power of two in [64, 2048] (default),
                                    1 = one CTA per row group */
  POISSON_OPT_COL_TILE = 10,     /* column-solve kernel: 0 = default (FP32 forward solves: two threads per
                                    column meeting mid-column, 32 columns per CTA; FP32 adjoint solves: the
                                    paired-ky kernel); 1, 2, 4 = two threads per column with 16, 32, 64
                                    columns; 3 = paired-ky kernel; 16, 32, 64, 128 = one thread per column
                                    with that many columns per CTA */
  POISSON_OPT_LAYOUT = 11,       /* layout of the caller's fields (S, p, gp, gS), a poisson_layout value;
                                    default POISSON_LAYOUT_Z_Y_X.  Any other layout adds two field-sized
                                    buffers to the workspace (query the size after setting it) */
  POISSON_OPT_SPECTRAL_FUSED = 12,/* 1: the forward y-pass, the column solves and the inverse y-pass of
                                    each forward solve run as one persistent kernel over strips of 8 kx,
                                    each strip's spectrum kept in L2 between the three steps, where the
                                    plan allows it (float spectrum, ny in {256, 512, 1024}, nz <= 256,
                                    one level chunk); 0 (default): three separate kernels */
  POISSON_OPT_RESIDUAL_PASS = 13, /* mixed: how a sweep forms its residual.  0 (default): the x-pass forms
                                    r while it loads its rows; 1 (where nx % 64 == 0, ny % 8 == 0, one
                                    level chunk): a stencil pass marching up the levels writes r as
                                    float (one more field-sized buffer in the workspace; query the size
                                    after setting it), then the plain R2C x-pass transforms it */
  POISSON_OPT_VERIFY = 14,        /* mixed: 1 (default): from the second sweep on, once a sweep's column
                                    solves are done, the norm of its correction delta_n (Parseval on the
                                    solved half spectrum) bounds the error of the current iterate,
                                    ||e_{n-1}|| <= ||delta_n||/(1 - phi) <= 2 ||delta_n|| for a contraction
                                    phi <= 1/2 (||delta_n||/(1 - phi) with the measured phi when that is
                                    above 1/2); if that bound is at most the tolerance the solve returns
                                    p_{n-1} without the sweep's inverse transforms (the two-threads-per-
                                    column kernel only).  On grids with nx/8 > max(8, sqrt(LOWK_RADIUS2))
                                    and ny > nx/4 the second sweep first solves only the columns with kx,
                                    |ky'| <= kcut = nx/8 (after a y-pass of those kx) and bounds the other
                                    columns of delta_2 by sqrt(W_max/W_min) ||r||/lambda_cut (lambda_cut
                                    the smallest horizontal eigenvalue outside that set): the norm is an
                                    upper bound, and when it does not certify p_1 the sweep runs in full.
                                    2: the verification solves every column (no cheaper first try).
                                    0: every sweep is applied in full */
  POISSON_OPT_GRAPH = 15          /* mixed: 1 (default): a solve called outside any stream capture and
                                    without profiling is captured once into a CUDA graph per (S, p,
                                    workspace) triple (the plan keeps the last four) and replayed on the
                                    caller's stream; the sweeps after the first are graph IF nodes on the
                                    device's done flag, so a certified solve launches none of their
                                    kernels.  0: plain stream launches (those kernels return at once) */
} poisson_option;

/* Field layouts (POISSON_OPT_LAYOUT), C order, outermost index first. */
typedef enum {
  POISSON_LAYOUT_Z_Y_X = 0,  /* [nz][ny][nx], x fastest: the solver's own layout */
  POISSON_LAYOUT_X_Y_Z = 1   /* [nx][ny][nz], z fastest: MONC's field order (its Fortran fields are
                                indexed data(z, y, x), as in the solver listings of Section 2.2);
                                converted to and from the solver's layout in the workspace by tiled
                                transposes, two extra passes over each field */
} poisson_layout;

/* Kernel phases reported by poisson_plan_profile_read. */
typedef enum {
  POISSON_PHASE_XFWD = 0,      /* forward x-pass (R2C) */
  POISSON_PHASE_YFWD = 1,      /* forward y-pass */
  POISSON_PHASE_COLUMNS = 2,   /* tridiagonal column solves (low-|k| + main kernels) */
  POISSON_PHASE_YINV = 3,      /* inverse y-pass */
  POISSON_PHASE_XINV = 4,      /* inverse x-pass (C2R) with its epilogue */
  POISSON_PHASE_RESIDUAL = 5,  /* correction rebuild before refinement sweep 3 (the residual itself is
                                  formed inside the sweep's forward x-pass) */
  POISSON_PHASE_CONTROL = 6,   /* refinement control and the final p = p0 + q after an early stop */
  POISSON_PHASE_SPECTRAL = 7,  /* the fused spectral middle (y-pass, columns, inverse y-pass in one
                                  kernel; POISSON_OPT_SPECTRAL_FUSED) */
  POISSON_NPHASES = 8
} poisson_phase;

/* Per-solve report of the mixed path's iterative refinement (the relative-residual
 * measure of Section 2.2 and the refinement stopping of Section 2.2's termination
 * idea, applied to the direct solve).  Sweep n computes the residual of iterate
 * p_{n-1} (p_0 = the first FP32 solve), solves for its correction delta_n and
 * updates p_n = p_{n-1} + delta_n. */
typedef struct {
  int sweeps;                  /* refinement corrections applied (mixed path; 0 otherwise): the result is
                                  iterate p_sweeps */
  int converged;               /* 1 if the mixed stopping test passed (always 1 for FP64/FP32) */
  double rel_update[4];        /* ||delta_n||_2/||p_n||_2 of sweep n (index 0 = first solve = 1).  When the
                                  solve stopped on a verification (POISSON_OPT_VERIFY), entry sweeps + 1
                                  holds the relative norm of the correction that certified the result
                                  and was not applied */
  double error_estimate;       /* mixed path: a bound on ||p_n - p||_2/||p||_2 for the returned iterate
                                  p_n, from the successive corrections.  With e_n the error of p_n,
                                  e_{n-1} = delta_n + e_n, so a sweep contracting the error by
                                  phi <= 1/2 gives ||e_n|| <= phi/(1-phi) ||delta_n|| <= ||delta_n||
                                  (bound rel_update[n] after applying delta_n) and
                                  ||e_{n-1}|| <= ||delta_n||/(1-phi) <= 2 ||delta_n|| (bound
                                  2 rel_update[n] for p_{n-1}, when delta_n verified it and was not
                                  applied); with a measured contraction
                                  phi = rel_update[n]/rel_update[n-1] above 1/2 the factors are
                                  phi/(1-phi) and 1/(1-phi), and the bound is +inf when phi >= 1.  The
                                  corrections see only the error that sweeps can remove; the bound adds
                                  accuracy_floor for the part the residual's rounding leaves.  The
                                  solve converges when it is at most the tolerance.  -1 when no sweep
                                  ran */
  double removed_weighted_mean;/* mu_W removed from S (first solve) */
  double rel_residual[4];      /* ||S - mu_W - L p_n||_2 / ||S||_2 of iterate n (index 0 = the first
                                  solve), formed in double-float arithmetic in the forward x-pass of
                                  sweep n+1; -1 where no such sweep ran (the returned iterate's own
                                  residual is formed only when a verification sweep ran).  mu_W is the
                                  one removed_weighted_mean reports.  -1 for FP64/FP32 plans */
  double accuracy_floor;       /* mixed path: the limiting accuracy F included in error_estimate, the
                                  relative error that the double-float residual's rounding (unit
                                  roundoff u = 2^-48) leaves however many sweeps run:
                                  F = u K sqrt(eta) sqrt(mean over the operator's nonsingular modes
                                  of 1/lambda^2), K the largest coefficient sum of the 7-point
                                  operator, eta = nz sum W_k^2/(sum W_k)^2.  A plan constant (it
                                  changes with poisson_plan_set_rho0); tolerances below it are never
                                  met.  -1 for FP64/FP32 plans */
} poisson_info;

/* Create a plan (Section 2.1: the solver plans once per grid and reuses the plan every
 * timestep).  dz and rho0 are HOST arrays of nz doubles (copied); bc is a
 * poisson_bc value (anything else: INVALID_ARG).
 * Supported: nx even, nx >= 4, ny >= 4, each of nx, ny of the form 2^a 3^b and
 * <= 4096, nz in [2, 512]; dx, dy > 0; dz[k] > 0; rho0[k] > 0.
 * Returns POISSON_ERR_UNSUPPORTED for other sizes, INVALID_ARG for bad values.
 * *out is set to NULL on failure. */
int poisson_plan_create(int nx, int ny, int nz, double dx, double dy, const double* dz,
                        const double* rho0, int bc, int dtype, poisson_plan** out);

/* Bytes of device workspace one solve/adjoint call of this plan needs: the half
 * spectrum [nz][ny][P] of Section 2.1's forward transform (P = nx/2+1 rounded up to
 * 128 bytes; float2 entries, double2 for FP64), the mixed path's float iterate and
 * correction fields, and small reduction buffers.  The caller allocates it (256-byte
 * aligned) and owns it. */
int poisson_plan_workspace_bytes(const poisson_plan* plan, size_t* bytes);

/* Set a plan option (see poisson_option).  Values out of range: INVALID_ARG. */
int poisson_plan_set_option(poisson_plan* plan, int option, double value);

/* Replace rho0 from a DEVICE array of nz doubles, recomputing the vertical
 * coefficient tables on the device, asynchronously on stream (used when rho0 is
 * a trained parameter).  Values must be positive; this is not checked on the
 * host (the call stays asynchronous). */
int poisson_plan_set_rho0(poisson_plan* plan, const double* rho0_dev, void* stream);

/* The direct solve of Section 2.1: forward real Fourier transform of S over x and y at
 * every level, one tridiagonal solve per (kx, ky) column along z, inverse transform.
 * Solve for p given the source S (both device fields of the plan's element type and
 * field layout; they must not overlap: INVALID_ARG).  workspace: device, >= workspace_bytes,
 * 256-byte aligned.  info: nullable host struct; when given, the call synchronises
 * the stream and fills it.  Mixed path: returns POISSON_ERR_NOT_CONVERGED (p still
 * written) when info is given and the error estimate stays above the tolerance. */
int poisson_solve(poisson_plan* plan, const void* S, void* p, void* workspace, void* stream,
                  poisson_info* info);

/* Adjoint of the solve map G: S -> p of Section 2.1 (a linear map for fixed rho0): the
 * same transform / column / inverse-transform pipeline with each column's transposed
 * tridiagonal system (the real DFT pair is its own adjoint up to scaling), so that the
 * pressure solve can sit inside gradient-based training.  The paper has no adjoint;
 * this is the derivative of its direct solve.
 * gp: dL/dp (device field); gS (out, device field): G^T gp = dL/dS.
 * grho (out, nullable, device array of nz doubles): dL/drho0 for p = G(rho0) S,
 * which needs p, the forward result (ignored when grho is NULL).
 * Same element type, workspace and stream rules as poisson_solve; gp, p, gS must
 * not overlap.  The mixed dtype runs the adjoint with double fields and float
 * transforms (no refinement). */
int poisson_solve_adjoint(poisson_plan* plan, const void* gp, const void* p, void* gS,
                          double* grho, void* workspace, void* stream);

/* ---- Variable density: preconditioned conjugate gradients (the iterative route of Section 2.2) ----
 * Solves  A p = S - mu_W  (zero plain mean; with p = 0 on the top face: A p = S) for a density
 * rho3 that varies in x, y and z, which the Fourier transform cannot separate:
 *   (A p)_ijk = (1/W_ijk) [ dz_k ((F^x_{i+1/2} - F^x_{i-1/2})/dx + (F^y_{j+1/2} - F^y_{j-1/2})/dy)
 *                          + F^z_{k+1/2} - F^z_{k-1/2} ],   W_ijk = rho3_ijk dz_k,
 *   F^x_{i+1/2} = (rho3_i + rho3_{i+1})/2 (p_{i+1} - p_i)/dx (periodic), F^y likewise,
 *   F^z_{k+1/2} = (rho3_k + rho3_{k+1})/2 (p_{k+1} - p_k)/h_{k+1/2}; the plan's vertical boundary
 *   condition at the bottom and top faces; mu_W = sum W S / sum W.  With rho3_ijk = rho0_k, A = L.
 * Conjugate gradients on -W A (symmetric): FP64 vectors and reductions, the operator applied in
 * double-float arithmetic (face coefficients formed once per call), preconditioned by this plan's direct solve
 * for its own rho0 profile (typically the horizontal mean of rho3); Polak-Ribiere directions.
 * The plan must have double fields (POISSON_FP64 or POISSON_MIXED; MIXED with
 * POISSON_OPT_MAX_SWEEPS = 0 is the cheapest preconditioner) and the default field layout.
 * rho3, S, p: DEVICE double [nz][ny][nx]; rho3 > 0 (not checked); none may overlap each other or
 * the workspace.  Stops when ||S - mu_W - A p||_2 / ||S||_2 <= tol or after max_iter iterations
 * (POISSON_ERR_NOT_CONVERGED, p holds the last iterate).  Synchronises the stream a few times per
 * iteration (the step lengths come back to the host, summed in a fixed order). */
typedef struct {
  int iterations;              /* CG iterations run */
  int converged;               /* 1 if the relative residual reached tol */
  double rel_residual;         /* ||S - mu_W - A p||_2 / ||S||_2 at exit */
  double removed_weighted_mean;/* mu_W (0 with p = 0 on the top face) */
} poisson_cg_info;

/* Workspace bytes for poisson_cg_solve (the plan's own workspace, five double fields and the
 * operator's three face-coefficient fields as float pairs). */
int poisson_cg_workspace_bytes(const poisson_plan* plan, size_t* bytes);

int poisson_cg_solve(poisson_plan* plan, const double* rho3, const double* S, double* p, double tol,
                     int max_iter, void* workspace, void* stream, poisson_cg_info* info);

/* Sum of the recorded per-phase kernel times (milliseconds) and launch counts
 * since the last read, for phases 0..nphases-1 (host arrays); synchronises on
 * the recorded events and clears them.  Recording is off unless
 * POISSON_OPT_PROFILE is set, and is skipped while a stream is being captured. */
int poisson_plan_profile_read(poisson_plan* plan, double* ms, int* launches, int nphases);

/* ---- Solve without allocating: for callers that cannot call cudaMalloc ----
 * (The paper has no counterpart; this serves callers of the library.)
 * Some callers cannot allocate device memory when they solve: a model driver whose
 * time loop must not call cudaMalloc (it can synchronise the device and has no
 * bounded latency), or a host program that owns the device memory pool and hands
 * this library only field pointers.  This entry point runs the same solve as
 * poisson_solve, but its scratch is a fixed device array inside the library of
 * POISSON_STATIC_WORKSPACE_BYTES bytes, held by every GPU that loads the library
 * until the process exits; it calls no allocating routine.  The plan itself is
 * created beforehand (its small tables are allocated then).
 *  - Plans whose workspace_bytes exceed the maximum: POISSON_ERR_WORKSPACE.
 *  - The first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture.  The address
 *    is then kept for the life of the process: it belongs to the device's primary
 *    context, so after cudaDeviceReset (which ends that context) this entry point
 *    must not be called again in the same process.
 *  - Every call on a device shares the one array: calls that overlap on the GPU
 *    (other streams, other plans, other threads) race.  The solve itself clears
 *    what must start at zero, so consecutive calls need nothing from the caller.
 * Same S, p, stream, info and status rules as poisson_solve. */
#define POISSON_STATIC_WORKSPACE_BYTES (32u * 1024u * 1024u)
int poisson_solve_static_workspace(poisson_plan* plan, const void* S, void* p, void* stream,
                                   poisson_info* info);

/* NULL-safe.  Frees the plan's device tables (synchronously). */
int poisson_plan_destroy(poisson_plan* plan);

/* Static string for a status code. */
const char* poisson_status_string(int status);

/* Text of the last CUDA failure seen by this thread (for POISSON_ERR_CUDA). */
const char* poisson_last_error_detail(void);

/* ---- Batched: many independent domains of uneven sizes in one graph launch ----
 * Arrays have n entries; dz[b], rho0[b] are host arrays of nz[b] doubles.
 * Every domain has zero flux at the bottom and top (POISSON_BC_PERIODIC_XY_NEUMANN_Z).
 * dtype POISSON_FP32 (float fields) or POISSON_MIXED (double fields). */
int poisson_batch_create(int n, const int* nx, const int* ny, const int* nz, const double* dx,
                         const double* dy, const double* const* dz, const double* const* rho0,
                         int dtype, poisson_batch** out);
int poisson_batch_workspace_bytes(const poisson_batch* batch, size_t* bytes);
/* S[b], p[b]: device fields of domain b.  info: nullable array of n structs.
 * By default the launch sequences of all domains are captured into one CUDA graph
 * of concurrent branches (domains largest first, each to the least-loaded branch;
 * POISSON_BATCH_OPT_BRANCHES).  With POISSON_BATCH_OPT_PERSISTENT = 1, mixed batches
 * whose every domain has nx and ny in {64, 128, 256, 384, 512} and 2 <= nz <= 128 run
 * as ONE persistent kernel instead: a work list of (domain, phase, tile) items
 * covering every step of every domain's solve and refinement (Sections 2.1 and 2.2),
 * per-domain dependency counters with bounded device waits (POISSON_ERR_TIMEOUT when
 * one runs out).  Either way the first call captures a CUDA graph bound to the given
 * pointers and workspace; later calls with the same pointers, workspace and
 * options replay it with a single graph launch, anything else re-captures.  The
 * persistent kernel ignores the plans' kernel-shape options (it has its own tile
 * shapes) and keeps their LOWK_RADIUS2, MAX_SWEEPS, TOLERANCE and VERIFY.
 * Returns the first failing domain's status. */
int poisson_batch_solve(poisson_batch* batch, const void* const* S, void* const* p,
                        void* workspace, void* stream, poisson_info* info);
int poisson_batch_destroy(poisson_batch* batch);
/* The plan of domain i (owned by the batch): for poisson_plan_set_option, e.g. to apply
 * autotuned kernel shapes.  Option changes re-capture the graph at the next solve;
 * query poisson_batch_workspace_bytes again after changing options. */
int poisson_batch_plan(poisson_batch* batch, int i, poisson_plan** plan);
/* Batch options (the next solve re-captures; query poisson_batch_workspace_bytes again after a
 * change).  POISSON_ERR_INVALID_ARG for an unknown option or value. */
typedef enum {
  POISSON_BATCH_OPT_PERSISTENT = 0,  /* 0 (default): the graph of per-domain launches; 1: the persistent
                                        kernel where the shapes allow */
  POISSON_BATCH_OPT_STALL_TEST = 1,  /* test hook, -1 (default) off: with the persistent kernel, the first
                                        control item of this domain waits for a work count that never
                                        arrives, so its bounded wait runs out (a few seconds) and the
                                        solve returns POISSON_ERR_TIMEOUT; no fault, no endless wait */
  POISSON_BATCH_OPT_BRANCHES = 2     /* graph of per-domain launches: concurrent branches, 1..32 (default 24) */
} poisson_batch_option;
int poisson_batch_set_option(poisson_batch* batch, int option, double value);

/* ---- Host-buffer pipeline: a stream of solves on one plan, fields in host memory ----
 * Not a step of the paper's method: the way a time-stepping host feeds the
 * solver.  poisson_pipe_create allocates two device slots (source and solution
 * of the plan's field type each), a workspace and three streams (copy in,
 * compute, copy out), all owned by the pipe.  poisson_pipe_submit enqueues one
 * step without waiting: copy S_host into a free slot, solve it, copy the
 * solution to p_host; the copy of step i+1's source and of step i-1's solution
 * overlap the solve of step i.  S_host and p_host hold nx*ny*nz values of the
 * plan's field type in its field layout ([nz][ny][nx], x fastest, by default).  Page-locked host buffers give
 * asynchronous copies; with pageable ones the copies still happen, without the
 * overlap.  The caller must not touch S_host until the step's source copy is
 * done, nor read p_host before poisson_pipe_wait returns.  Steps complete in
 * submission order.
 * poisson_pipe_wait blocks until every submitted step is done and returns the
 * first non-OK status of the steps since the previous wait: an enqueue error,
 * a device wait time-out, or POISSON_ERR_NOT_CONVERGED from a mixed solve (the
 * last 1024 steps are checked).  The pipe takes no ownership of the plan;
 * destroy the pipe first.  One thread per pipe. */
int poisson_pipe_create(poisson_plan* plan, poisson_pipe** out);
int poisson_pipe_submit(poisson_pipe* pipe, const void* S_host, void* p_host);
int poisson_pipe_wait(poisson_pipe* pipe);
int poisson_pipe_destroy(poisson_pipe* pipe);

#ifdef __cplusplus
}
#endif
#endif /* POISSON_GB300_H */
