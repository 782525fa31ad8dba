"""Plain FP64 CPU oracle for the direct FFT pressure solve.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call this
module: only the tests, the smoke check of ``__graft_entry__`` and the CPU
baseline / reference arm of ``bench.py`` use it.  It shares no code with the
CUDA path.

What it computes (Brown, "A comparison of techniques for solving the Poisson
equation in CFD", Section 2.1): a forward Fourier transform over the periodic
x/y plane at every level, an independent vertical tridiagonal solve per
(kx, ky) column, and a backward transform that gives the pressure.  The paper
names an elliptic equation of Poisson type (Section 2) and nabla^2 x = b
(Section 2.2) but prints no discretisation, so this module fixes one reading:

  * cell-centred finite-volume 7-point operator, periodic in x and y with
    uniform dx, dy; cell thicknesses dz[k]; reference density rho0[k] at cell
    centres, faces by arithmetic mean; homogeneous Neumann (zero flux) at the
    bottom face and, by default, at the top face;
        (L p) = (p[i+1]-2p[i]+p[i-1])/dx^2 + (p[j+1]-2p[j]+p[j-1])/dy^2
                + a_k (p[k-1]-p[k]) + c_k (p[k+1]-p[k]),
        W_k = rho_k dz_k,  a_k = rho_{k-1/2}/(W_k h_{k-1/2}),
        c_k = rho_{k+1/2}/(W_k h_{k+1/2}),  h_{k+1/2} = (dz_k+dz_{k+1})/2;
  * compatibility: the source is projected, Q_W S = S - mu_W with mu_W the
    W-weighted mean of S over all cells;
  * the solution is the unique p with L p = Q_W S and plain mean zero.

With bc="dirichlet_top" the top face instead carries p = 0: its flux is
rho_top (0 - p_{nz-1}) / (dz_{nz-1}/2) with rho_top = rho0[nz-1] (the paper gives
densities at centres only), so c_{nz-1} = rho_top / (W_{nz-1} dz_{nz-1}/2).  L is
then nonsingular and the solution is p = L^{-1} S: no projection, no pinning.

For the iterative alternative (Section 2.2) with a density that also varies in x
and y, apply_A_var and solve_var give the flux-form operator and a library sparse
direct solve of it on moderate grids.

The solve is exact (Section 3 describes the direct method as solving the
system exactly every time), so the oracle is that definition written out: a naive O(n^2) DFT per line built
from exactly index-reduced twiddles (matrix products are the library step), the
textbook Thomas recurrence per column, a dense bordered solve for the singular
(0,0) column, and the naive inverse DFT.  No blocking, fusion or reordering.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "vertical_coefficients", "horizontal_eigenvalues", "weighted_mean", "project_compatible",
    "apply_L", "residual", "dft_x", "dft_y", "idft_y", "idft_x", "thomas",
    "column_matrix", "singular_column_solve", "solve", "adjoint", "rho0_gradient",
    "relative_l2", "apply_A_var", "weights_var", "solve_var",
]


def _f64(x):
    return np.asarray(x, dtype=np.float64)


# ---------------------------------------------------------------------------
# Operator pieces (Section 2: the elliptic pressure equation, read as above)
# ---------------------------------------------------------------------------

BCS = ("neumann", "dirichlet_top")


def _check_bc(bc):
    if bc not in BCS:
        raise ValueError(f"bc must be one of {BCS}")


def vertical_coefficients(dz, rho0, bc="neumann"):
    """Return (W, a, c) of the density-weighted vertical operator.

    W_k = rho_k dz_k; a_k couples level k to k-1 (a_0 = 0: zero flux through the
    bottom face), c_k couples k to k+1.  Top face: c_{nz-1} = 0 for zero flux
    ("neumann"); for p = 0 on the face ("dirichlet_top") c_{nz-1} couples the top
    cell to the face value 0 over half a cell, with the top cell's density.
    """
    _check_bc(bc)
    dz = _f64(dz)
    rho0 = _f64(rho0)
    nz = dz.size
    W = rho0 * dz
    h = 0.5 * (dz[:-1] + dz[1:])              # centre-to-centre spacing at face k+1/2
    rho_face = 0.5 * (rho0[:-1] + rho0[1:])   # density at face k+1/2
    conductance = rho_face / h
    a = np.zeros(nz)
    c = np.zeros(nz)
    c[:-1] = conductance / W[:-1]
    a[1:] = conductance / W[1:]
    if bc == "dirichlet_top":
        c[-1] = rho0[-1] / (0.5 * dz[-1]) / W[-1]
    return W, a, c


def horizontal_eigenvalues(n, d, count=None):
    """Eigenvalues of the periodic second difference on n points of spacing d.

    For wavenumber m the eigenvector exp(2 pi i m j / n) gives
    (e^{-i t} - 2 + e^{i t})/d^2 = -(4/d^2) sin^2(pi m / n); the sin^2 form
    avoids the cancellation of 2cos(t)-2 at small m.
    """
    if count is None:
        count = n
    m = np.arange(count, dtype=np.float64)
    return -(4.0 / (d * d)) * np.sin(np.pi * m / n) ** 2


def weighted_mean(S, W):
    """mu_W = sum_{ijk} W_k S_ijk / (nx ny sum_k W_k)."""
    S = _f64(S)
    nz, ny, nx = S.shape
    level_sums = S.reshape(nz, -1).sum(axis=1)
    return float(np.dot(W, level_sums) / (nx * ny * W.sum()))


def project_compatible(S, W):
    """Q_W S = S - mu_W: the part of S in the range of L (sum W_k (Q_W S)_ijk = 0)."""
    return _f64(S) - weighted_mean(S, W)


def apply_L(p, dx, dy, a, c):
    """Matrix-free 7-point operator L p (periodic x/y).

    Bottom: no term below level 0 (a_0 = 0).  Top: c_{nz-1} (0 - p_{nz-1}), the
    coupling to the face value 0; it vanishes with zero flux (c_{nz-1} = 0).
    """
    p = _f64(p)
    Lx = (np.roll(p, -1, axis=2) - 2.0 * p + np.roll(p, 1, axis=2)) / (dx * dx)
    Ly = (np.roll(p, -1, axis=1) - 2.0 * p + np.roll(p, 1, axis=1)) / (dy * dy)
    Lz = np.zeros_like(p)
    Lz[1:] += a[1:, None, None] * (p[:-1] - p[1:])
    Lz[:-1] += c[:-1, None, None] * (p[1:] - p[:-1])
    Lz[-1] += c[-1] * (0.0 - p[-1])
    return Lx + Ly + Lz


def residual(S, p, dx, dy, dz, rho0, bc="neumann"):
    """r = Q_W S - L p (the quantity the relative-residual measure of Section 2.2 uses).

    With p = 0 on the top face nothing is projected: r = S - L p.
    """
    W, a, c = vertical_coefficients(dz, rho0, bc)
    rhs = project_compatible(S, W) if bc == "neumann" else _f64(S)
    return rhs - apply_L(p, dx, dy, a, c)


# ---------------------------------------------------------------------------
# Naive discrete Fourier transforms (Section 2.1: one dimension at a time)
# ---------------------------------------------------------------------------

def _twiddles(n, count, sign):
    """Matrix E[m, k] = exp(sign * 2 pi i ((m k) mod n) / n), m < n, k < count."""
    m = np.arange(n, dtype=np.int64)[:, None]
    k = np.arange(count, dtype=np.int64)[None, :]
    r = (m * k) % n
    t = 2.0 * np.pi * r.astype(np.float64) / n
    return np.cos(t), sign * np.sin(t)


def dft_x(S):
    """Real forward DFT along x: X[..., kx] = sum_i S[..., i] e^{-2 pi i kx i/nx}, kx = 0..nx//2."""
    S = _f64(S)
    nx = S.shape[-1]
    C, Sn = _twiddles(nx, nx // 2 + 1, -1.0)
    return (S @ C) + 1j * (S @ Sn)


def dft_y(X):
    """Complex forward DFT along y (axis -2): Y[.., ky, kx] = sum_j e^{-2 pi i ky j/ny} X[.., j, kx]."""
    ny = X.shape[-2]
    C, Sn = _twiddles(ny, ny, -1.0)
    F = C + 1j * Sn                    # symmetric: F[j, ky] = F[ky, j]
    return np.matmul(F, X)


def idft_y(Y):
    """Complex inverse DFT along y with the 1/ny factor."""
    ny = Y.shape[-2]
    C, Sn = _twiddles(ny, ny, +1.0)
    F = C + 1j * Sn
    return np.matmul(F, Y) / ny


def idft_x(X, nx):
    """Real inverse DFT along x from the half spectrum kx = 0..nx//2, with 1/nx.

    p[i] = (1/nx) sum_kx w_kx Re(X_kx e^{+2 pi i kx i/nx}); w = 1 for the
    self-conjugate bins kx = 0 and (nx even) kx = nx/2, 2 for all others.
    This is the full inverse DFT of the Hermitian extension of X, real part.
    """
    nh = nx // 2 + 1
    assert X.shape[-1] == nh
    w = np.full(nh, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[-1] = 1.0
    C, Sn = _twiddles(nx, nh, +1.0)    # (nx, nh): [i, kx]
    return (X.real @ (C * w).T - X.imag @ (Sn * w).T) / nx


# ---------------------------------------------------------------------------
# Column solves (Section 2.1: tridiagonal solve up and down each column)
# ---------------------------------------------------------------------------

def thomas(sub, diag, sup, rhs):
    """Textbook Thomas recurrence, vectorised over independent columns.

    Row k reads  sub[k] x[k-1] + diag[k] x[k] + sup[k] x[k+1] = rhs[k];
    all arrays have the level index first and broadcast over the rest.
    """
    n = rhs.shape[0]
    shape = np.broadcast_shapes(np.shape(diag[0]), np.shape(rhs[0]))
    cp = np.empty((n,) + shape, dtype=np.result_type(diag, sup))
    dp = np.empty((n,) + shape, dtype=np.result_type(diag, rhs))
    beta = diag[0] * np.ones(shape)
    cp[0] = sup[0] / beta
    dp[0] = rhs[0] / beta
    for k in range(1, n):
        beta = diag[k] - sub[k] * cp[k - 1]
        cp[k] = sup[k] / beta
        dp[k] = (rhs[k] - sub[k] * dp[k - 1]) / beta
    x = np.empty_like(dp)
    x[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return x


def column_matrix(a, c, lam):
    """Dense T = L_z + lam I for one column (a, c from vertical_coefficients)."""
    nz = a.size
    T = np.zeros((nz, nz))
    for k in range(nz):
        T[k, k] = -(a[k] + c[k]) + lam
        if k > 0:
            T[k, k - 1] = a[k]
        if k < nz - 1:
            T[k, k + 1] = c[k]
    return T


# Extended precision of the platform (x87 80-bit on x86-64, IEEE binary128 on aarch64):
# used for the columns whose FP64 rounding is amplified (see _column_solves).
XP = np.longdouble
# Columns with |lambda_x + lambda_y| below this fraction of the largest vertical coupling
# a_k + c_k are solved in XP.
WEAK_COLUMN_RATIO = 1e-3


def gauss_solve(A, B):
    """Dense Gaussian elimination with partial pivoting in A's dtype (B: one or more columns)."""
    A = np.array(A, copy=True)
    B = np.array(B, copy=True)
    n = A.shape[0]
    for k in range(n):
        piv = k + int(np.argmax(np.abs(A[k:, k])))
        if piv != k:
            A[[k, piv]] = A[[piv, k]]
            B[[k, piv]] = B[[piv, k]]
        f = A[k + 1:, k] / A[k, k]
        A[k + 1:, k:] -= f[:, None] * A[k, k:][None, :]
        B[k + 1:] -= f.reshape((-1,) + (1,) * (B.ndim - 1)) * B[k]
    X = np.empty_like(B)
    for k in range(n - 1, -1, -1):
        X[k] = (B[k] - A[k, k + 1:] @ X[k + 1:]) / A[k, k]
    return X


def singular_column_solve(a, c, rhs, transpose=False):
    """Unique zero-sum solution of T x = rhs for the singular (0,0) column.

    T = L_z has null vector 1 (T^T has null vector W); the bordered matrix
    [[T, 1], [1^T, 0]] is nonsingular and, for a compatible right-hand side,
    its solution is the zero-sum x with multiplier 0.  Dense Gaussian
    elimination with partial pivoting in extended precision (the bordered
    matrix's condition grows as the inverse of the smallest vertical eigenvalue,
    about 1e6 on 128 stretched levels, which FP64 would pass on to x).
    """
    nz = a.size
    T = np.zeros((nz, nz), dtype=XP)       # L_z with its diagonal -(a_k + c_k) formed in XP
    for k in range(nz):
        T[k, k] = -(XP(a[k]) + XP(c[k]))
        if k > 0:
            T[k, k - 1] = a[k]
        if k < nz - 1:
            T[k, k + 1] = c[k]
    if transpose:
        T = T.T
    B = np.zeros((nz + 1, nz + 1), dtype=XP)
    B[:nz, :nz] = T
    B[:nz, nz] = 1.0
    B[nz, :nz] = 1.0
    rhs = np.asarray(rhs)
    r = np.zeros((nz + 1, 2), dtype=XP)
    r[:nz, 0] = rhs.real
    if np.iscomplexobj(rhs):
        r[:nz, 1] = rhs.imag
    x = gauss_solve(B, r)[:nz].astype(np.float64)
    return x[:, 0] + 1j * x[:, 1] if np.iscomplexobj(rhs) else x[:, 0]


def _spectral_lambda(dx, dy, nx, ny):
    """lambda_x(kx) + lambda_y(ky) on the half spectrum, shape (ny, nx//2 + 1)."""
    lx = horizontal_eigenvalues(nx, dx, nx // 2 + 1)     # (nxh,)
    ly = horizontal_eigenvalues(ny, dy, ny)              # (ny,)
    return ly[:, None] + lx[None, :]


def _column_solves(sub, sup, a, c, lam, rhs, skip00):
    """Textbook Thomas on every column of rhs (nz, ny, nxh): T = L_z + lam I.

    sub/sup: the (nz,) couplings below/above the diagonal (a, c for T; c shifted,
    a shifted for T^T).  The diagonal -(a_k + c_k) + lam holds the column's row
    sum lam only to FP64 rounding of a_k + c_k, so a column with |lam| far below
    the couplings loses about eps (a + c)/|lam| of relative accuracy in FP64:
    those columns are solved again in extended precision.  skip00: the (0,0)
    column is solved elsewhere (zero-flux top); it gets a dominant stand-in here.
    """
    diag = -(a + c)[:, None, None] + lam[None, :, :]
    if skip00:
        diag[:, 0, 0] = -(a + c) - 1.0
    x = thomas(sub[:, None, None], diag, sup[:, None, None], rhs)
    weak = np.abs(lam) < WEAK_COLUMN_RATIO * np.max(a + c)
    if skip00:
        weak[0, 0] = False
    jj, ii = np.nonzero(weak)
    if jj.size:
        dxp = -(a.astype(XP) + c.astype(XP))[:, None] + lam[jj, ii].astype(XP)[None, :]
        sb, sp = sub.astype(XP)[:, None], sup.astype(XP)[:, None]
        col = rhs[:, jj, ii]
        re = thomas(sb, dxp, sp, col.real.astype(XP)).astype(np.float64)
        im = thomas(sb, dxp, sp, col.imag.astype(XP)).astype(np.float64)
        x[:, jj, ii] = re + 1j * im
    return x


def solve(S, dx, dy, dz, rho0, return_info=False, bc="neumann"):
    """p = the zero-mean solution of L p = Q_W S (Section 2.1 structure).

    Forward DFT in x then y at every level, textbook Thomas per (kx, ky)
    column with T = L_z + (lambda_x + lambda_y) I, bordered solve for the
    (0,0) column, inverse DFT in y then x.  With bc="dirichlet_top" every
    column, (0,0) included, is nonsingular: p = L^{-1} S by Thomas throughout.
    The direct method is exact (Section 3), so the oracle's own rounding must
    stay far below the tolerances it checks: columns whose diagonal dominance
    is weak are solved in extended precision (_column_solves).
    """
    S = _f64(S)
    nz, ny, nx = S.shape
    W, a, c = vertical_coefficients(dz, rho0, bc)
    neumann = bc == "neumann"
    mu_W = weighted_mean(S, W) if neumann else 0.0
    Shat = dft_y(dft_x(S - mu_W))                          # (nz, ny, nxh)
    phat = _column_solves(a, c, a, c, _spectral_lambda(dx, dy, nx, ny), Shat, skip00=neumann)
    if neumann:
        phat[:, 0, 0] = singular_column_solve(a, c, Shat[:, 0, 0])
    p = idft_x(idft_y(phat), nx)
    if return_info:
        return p, {"removed_weighted_mean": mu_W}
    return p


def adjoint(wgt, dx, dy, dz, rho0, bc="neumann"):
    """g = G^T wgt where G: S -> p is the map computed by solve().

    G = P_1 L^+ Q_W with P_1 the plain-mean projection.  The 2-D DFT matrix is
    symmetric and each column matrix is the same for +k and -k, so
    G^T = Q_W^T F^{-1} T_k^{-T} F P_1: forward DFT, transposed column solve,
    inverse DFT.  In the (0,0) column P_1 removes the plain mean of the
    transformed weights, the transposed singular column (null vector W) is
    solved by the bordered system, and Q_W^T v = v - W (sum v)/(nx ny sum W)
    removes the W direction.  With bc="dirichlet_top" G = L^{-1} and
    G^T = F^{-1} T_k^{-T} F in every column.
    """
    wgt = _f64(wgt)
    nz, ny, nx = wgt.shape
    W, a, c = vertical_coefficients(dz, rho0, bc)
    neumann = bc == "neumann"
    What = dft_y(dft_x(wgt))
    if neumann:
        What[:, 0, 0] -= What[:, 0, 0].mean()              # P_1
    # T^T: row k has T[k-1,k] = c_{k-1} below the diagonal and T[k+1,k] = a_{k+1} above
    sub_t = np.zeros(nz)
    sup_t = np.zeros(nz)
    sub_t[1:] = c[:-1]
    sup_t[:-1] = a[1:]
    mhat = _column_solves(sub_t, sup_t, a, c, _spectral_lambda(dx, dy, nx, ny), What, skip00=neumann)
    if neumann:
        mhat[:, 0, 0] = singular_column_solve(a, c, What[:, 0, 0], transpose=True)
    m = idft_x(idft_y(mhat), nx)
    if neumann:
        m -= W[:, None, None] * (m.sum() / (nx * ny * W.sum()))  # Q_W^T
    return m


def rho0_gradient(wgt, S, dx, dy, dz, rho0, p=None, g=None, bc="neumann"):
    """d(sum wgt*p)/d rho0_m for p = solve(S; rho0).

    Differentiating L p = Q_W S with 1^T p = 0 gives
        dl/drho_m = g^T (dQ_W/drho_m S - dL/drho_m p),  g = G^T wgt.
    dL/drho_m only touches the vertical coefficients a_k, c_k of rows m-1, m,
    m+1 (through W_m and the face densities at m-1/2, m+1/2).  With p = 0 on the
    top face there is no projection (Q_W = I) and c_{nz-1} = rho_{nz-1} /
    (W_{nz-1} dz_{nz-1}/2) also depends on rho_{nz-1}.
    """
    dz = _f64(dz)
    rho0 = _f64(rho0)
    S = _f64(S)
    nz, ny, nx = S.shape
    W, a, c = vertical_coefficients(dz, rho0, bc)
    if p is None:
        p = solve(S, dx, dy, dz, rho0, bc=bc)
    if g is None:
        g = adjoint(wgt, dx, dy, dz, rho0, bc=bc)
    h = 0.5 * (dz[:-1] + dz[1:])
    # per-level contractions  Ma_k = sum_ij g_k (p_{k-1}-p_k),  Mc_k = sum_ij g_k (p_{k+1}-p_k)
    Ma = np.zeros(nz)
    Mc = np.zeros(nz)
    Ma[1:] = np.einsum("kji,kji->k", g[1:], p[:-1] - p[1:])
    Mc[:-1] = np.einsum("kji,kji->k", g[:-1], p[1:] - p[:-1])
    Mc[-1] = np.einsum("ji,ji->", g[-1], 0.0 - p[-1])      # coupling to the top face value 0
    level_S = S.reshape(nz, -1).sum(axis=1)
    level_g = g.reshape(nz, -1).sum(axis=1)
    sumW = W.sum()
    mu_W = np.dot(W, level_S) / (nx * ny * sumW)
    grad = np.zeros(nz)
    for m in range(nz):
        da = np.zeros(nz)
        dc = np.zeros(nz)
        for k in range(nz):
            dW = dz[k] if k == m else 0.0
            if k > 0:   # a_k = rho_face[k-1] / (W_k h[k-1])
                dnum = 0.5 if m in (k - 1, k) else 0.0
                da[k] = dnum / (W[k] * h[k - 1]) - a[k] * dW / W[k]
            if k < nz - 1:   # c_k = rho_face[k] / (W_k h[k])
                dnum = 0.5 if m in (k, k + 1) else 0.0
                dc[k] = dnum / (W[k] * h[k]) - c[k] * dW / W[k]
            elif bc == "dirichlet_top":   # c_{nz-1} = rho_{nz-1} / (W_{nz-1} dz_{nz-1}/2)
                dnum = 1.0 if m == k else 0.0
                dc[k] = dnum / (W[k] * 0.5 * dz[k]) - c[k] * dW / W[k]
        dL_term = np.dot(da, Ma) + np.dot(dc, Mc)
        dQ_term = 0.0
        if bc == "neumann":
            # Q_W S = S - mu_W 1:  d/drho_m (-mu_W) contracted with g
            dmu = dz[m] * (level_S[m] - nx * ny * mu_W) / (nx * ny * sumW)
            dQ_term = -dmu * level_g.sum()
        grad[m] = dQ_term - dL_term
    return grad


def relative_l2(x, ref):
    """||x - ref||_2 / ||ref||_2 over all cells."""
    x = _f64(x)
    ref = _f64(ref)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


# ---------------------------------------------------------------------------
# Variable density (the case an iterative solver opens, Section 2.2): rho varies
# in x, y and z, so the Fourier transform no longer separates the operator.
# ---------------------------------------------------------------------------

def weights_var(dz, rho3):
    """W_ijk = rho_ijk dz_k, the cell weights of the variable-density operator."""
    return _f64(rho3) * _f64(dz)[:, None, None]


def apply_A_var(p, dx, dy, dz, rho3, bc="neumann"):
    """Flux-form 7-point operator of div(rho grad p)/rho on the same cells as L.

    (A p)_ijk = (1/W_ijk) [ dz_k ((F^x_{i+1/2} - F^x_{i-1/2})/dx + (F^y_{j+1/2} - F^y_{j-1/2})/dy)
                           + F^z_{k+1/2} - F^z_{k-1/2} ],
    with fluxes F^x_{i+1/2} = rho_{i+1/2} (p_{i+1} - p_i)/dx (periodic),
    F^y likewise, F^z_{k+1/2} = rho_{k+1/2} (p_{k+1} - p_k)/h_{k+1/2}, face
    densities by arithmetic mean of the two cells, zero flux through the bottom
    face and through the top face ("neumann") or F^z_top = rho_{nz-1} (0 - p_{nz-1})
    / (dz_{nz-1}/2) ("dirichlet_top").  With rho_ijk = rho0_k this is L.
    """
    _check_bc(bc)
    p = _f64(p)
    rho = _f64(rho3)
    dz = _f64(dz)
    nz = p.shape[0]
    Fx = 0.5 * (rho + np.roll(rho, -1, axis=2)) * (np.roll(p, -1, axis=2) - p) / dx   # at i+1/2
    Fy = 0.5 * (rho + np.roll(rho, -1, axis=1)) * (np.roll(p, -1, axis=1) - p) / dy   # at j+1/2
    h = 0.5 * (dz[:-1] + dz[1:])
    Fz = np.zeros((nz + 1,) + p.shape[1:])                                          # at k-1/2, k = 0..nz
    Fz[1:nz] = 0.5 * (rho[:-1] + rho[1:]) * (p[1:] - p[:-1]) / h[:, None, None]
    if bc == "dirichlet_top":
        Fz[nz] = rho[-1] * (0.0 - p[-1]) / (0.5 * dz[-1])
    div = (dz[:, None, None] * ((Fx - np.roll(Fx, 1, axis=2)) / dx + (Fy - np.roll(Fy, 1, axis=1)) / dy)
           + (Fz[1:] - Fz[:-1]))
    return div / weights_var(dz, rho)


def solve_var(S, dx, dy, dz, rho3, bc="neumann"):
    """p with A p = Q S (zero plain mean with zero flux at the top; A^-1 S with p = 0 there).

    Q S = S - sum(W S)/sum(W) removes the part of S outside the range of A.  The
    matrix is assembled column by column from apply_A_var and solved by a library
    sparse LU (with zero flux, after fixing one cell and then removing the mean):
    tiny and moderate grids only.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    S = _f64(S)
    shape = S.shape
    N = S.size
    nz, ny, nx = shape
    W = weights_var(dz, rho3)
    rhs = S.ravel().copy()
    if bc == "neumann":
        rhs -= (W * S).sum() / W.sum()
    # columns of A by probing with sums of unit vectors whose stencils never overlap: indices
    # of one colour differ by a multiple of m >= 3 (m divides a periodic extent, so the
    # wrap-around keeps the spacing)
    def colours(n, periodic):
        if not periodic:
            return 3
        return next((m for m in range(3, n + 1) if n % m == 0), n)

    mz, my, mx = colours(nz, False), colours(ny, True), colours(nx, True)
    rows, cols, vals = [], [], []
    idx = np.arange(N).reshape(shape)
    for ck in range(min(mz, nz)):
        for cj in range(min(my, ny)):
            for ci in range(min(mx, nx)):
                e = np.zeros(shape)
                sel = np.zeros(shape, dtype=bool)
                sel[ck::mz, cj::my, ci::mx] = True
                e[sel] = 1.0
                Ae = apply_A_var(e, dx, dy, dz, rho3, bc)
                for q in idx[sel]:
                    k, j, i = np.unravel_index(q, shape)
                    # the rows of q's stencil, each once (with 2 cells in a periodic direction
                    # the two neighbours there are one cell)
                    stencil = {(k + dk, (j + dj) % ny, (i + di) % nx)
                               for dk, dj, di in ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                                  (0, 0, 1), (0, 0, -1))
                               if 0 <= k + dk < nz}
                    for kk, jj, ii in stencil:
                        rows.append(idx[kk, jj, ii])
                        cols.append(q)
                        vals.append(Ae[kk, jj, ii])
    A = sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()
    A.sum_duplicates()
    if bc == "neumann":
        # constants span the null space: fix p at cell 0 (its row is implied by the others,
        # since the W-weighted rows of A sum to zero and Q S is compatible), then remove the mean
        A = A.tolil()
        A[0, :] = 0.0
        A[0, 0] = 1.0
        rhs[0] = 0.0
        x = spla.spsolve(A.tocsc(), rhs)
        x -= x.mean()
    else:
        x = spla.spsolve(A.tocsc(), rhs)
    return x.reshape(shape)
