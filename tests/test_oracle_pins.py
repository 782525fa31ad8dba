"""Pins for the FP64 CPU oracle, against facts that do not come from the oracle.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a wrong index, a transposed operand) fails at least one of them:

* the operator against exact discrete eigenfunctions (uniform grid) and against
  the continuous anelastic operator (1/rho) d/dz(rho dp/dz) on smoothly
  stretched grids (second-order convergence);
* the operator's structure: null vector, conservation, W-weighted symmetry;
* the transforms against numpy.fft (library special case) and the paper's
  forward-then-backward round-trip test (Section 2.1);
* the Thomas recurrence against a dense library solve;
* the full solve against eigenfunction closed forms, a brute-force dense
  bordered solve on tiny grids, and invariants (zero mean, residual, shift
  equivariance);
* the adjoint by the dot-product test and a dense transpose; the rho0 gradient
  by central finite differences.
* the p = 0 top-face option likewise: its own eigenfunctions, second-order
  convergence to the continuous problem, a dense nonsingular solve, the dense
  transposed solve and central differences of the rho0 gradient.
"""
import numpy as np
import pytest

import oracle as O
from paper_2010_14132_gb300 import workloads as wl


# ---------------------------------------------------------------------------
# operator
# ---------------------------------------------------------------------------

def test_vertical_coefficients_uniform_reduce_to_second_difference():
    h = 0.7
    W, a, c = O.vertical_coefficients(np.full(6, h), np.full(6, 1.3))
    assert np.allclose(W, 1.3 * h, rtol=1e-15)
    assert a[0] == 0.0 and c[-1] == 0.0
    assert np.allclose(a[1:], 1 / h**2, rtol=1e-14)
    assert np.allclose(c[:-1], 1 / h**2, rtol=1e-14)


def test_flux_symmetry_stretched():
    d = wl.anelastic_blobs(8, 8, 64, with_source=False)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0)
    # flux through face k+1/2 seen from below equals the one seen from above
    assert np.allclose(W[:-1] * c[:-1], W[1:] * a[1:], rtol=1e-14)


def _cos_mode(nx, ny, nz, ax, by, cz, phx=0.3, phy=-0.7):
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    return (np.cos(2 * np.pi * ax * i / nx + phx) * np.cos(2 * np.pi * by * j / ny + phy)
            * np.cos(np.pi * cz * (k + 0.5) / nz))


def _cos_mode_eig(nx, ny, nz, ax, by, cz, dx, dy, dz):
    return (-4 / dx**2 * np.sin(np.pi * ax / nx) ** 2 - 4 / dy**2 * np.sin(np.pi * by / ny) ** 2
            - 4 / dz**2 * np.sin(np.pi * cz / (2 * nz)) ** 2)


@pytest.mark.parametrize("mode", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (3, 2, 5), (8, 6, 3), (4, 3, 0)])
def test_operator_eigenfunctions_uniform(mode):
    nx, ny, nz, dx, dy, dz = 16, 12, 10, 0.9, 1.7, 0.6
    p = _cos_mode(nx, ny, nz, *mode)
    W, a, c = O.vertical_coefficients(np.full(nz, dz), np.full(nz, 2.0))
    Lp = O.apply_L(p, dx, dy, a, c)
    lam = _cos_mode_eig(nx, ny, nz, *mode, dx, dy, dz)
    assert np.abs(Lp - lam * p).max() <= 1e-13 * np.abs(lam)


def _smooth_grid(nz, H=3000.0, beta=1.5):
    """Cells of a smooth stretching z = H (e^{beta s}-1)/(e^beta-1), s uniform on [0,1]."""
    s = np.linspace(0, 1, nz + 1)
    zf = H * np.expm1(beta * s) / np.expm1(beta)
    return np.diff(zf)


def test_solution_converges_to_continuous_anelastic_problem():
    """Second-order convergence to the continuous anelastic problem on stretched levels.

    Exact solution p = cos(2 pi i/nx) cos(pi z/H): zero flux at z = 0 and H, and
    rho = 1.2 exp(-z/Hs).  The source uses the continuous vertical operator
    (1/rho) d/dz(rho dp/dz) plus the exact discrete horizontal eigenvalue, so only
    the vertical discretisation is under test.  Cell-centred finite volumes on a
    smooth stretching converge at second order; a wrong face density, centre
    spacing or weight leaves a first-order or O(1) error and fails the ratio test.
    """
    H, Hs, nx, dx = 3000.0, 2500.0, 8, 400.0
    i = np.arange(nx)
    lx = -(4 / dx**2) * np.sin(np.pi / nx) ** 2
    errs = []
    for nz in (32, 64, 128, 256):
        dz = _smooth_grid(nz, H)
        z = wl.cell_centres(dz)
        rho = 1.2 * np.exp(-z / Hs)
        f = np.cos(np.pi * z / H)
        Lf = -(np.pi / H) ** 2 * np.cos(np.pi * z / H) + (np.pi / H) / Hs * np.sin(np.pi * z / H)
        hx = np.cos(2 * np.pi * i / nx)[None, None, :] * np.ones((1, 2, 1))
        exact = f[:, None, None] * hx
        S = (Lf + lx * f)[:, None, None] * hx
        p = O.solve(S, dx, 1.0, dz, rho)
        errs.append(np.abs(p - exact).max() / np.abs(exact).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.5) and np.all(ratios < 4.3), (errs, ratios)


def test_operator_structure_stretched():
    d = wl.random_stretched(6, 5, 7, seed=11)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(d.S.shape)
    v = rng.standard_normal(d.S.shape)
    Wf = W[:, None, None]
    # constants are in the null space
    assert np.abs(O.apply_L(np.full(d.S.shape, 3.0), d.dx, d.dy, a, c)).max() < 1e-13
    # conservation: sum W (L v) = 0
    Lv = O.apply_L(v, d.dx, d.dy, a, c)
    assert abs((Wf * Lv).sum()) < 1e-12 * (Wf * np.abs(Lv)).sum()
    # W L is symmetric
    lhs = (u * Wf * Lv).sum()
    rhs = (Wf * O.apply_L(u, d.dx, d.dy, a, c) * v).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_projection():
    d = wl.random_stretched(5, 6, 4, seed=3)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0)
    S = d.S + 0.37
    Q = O.project_compatible(S, W)
    assert abs((W[:, None, None] * Q).sum()) < 1e-13 * np.abs(S).sum()
    assert np.allclose(O.project_compatible(S + 5.0, W), Q, atol=1e-13)
    assert np.allclose(O.project_compatible(Q, W), Q, atol=1e-14)


# ---------------------------------------------------------------------------
# transforms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nx,ny", [(4, 6), (12, 9), (16, 16), (6, 48), (7, 5)])
def test_dft_matches_numpy_fft(nx, ny):
    rng = np.random.default_rng(nx * 100 + ny)
    S = rng.standard_normal((3, ny, nx))
    X = O.dft_x(S)
    assert np.allclose(X, np.fft.rfft(S, axis=2), atol=1e-12)
    Y = O.dft_y(X)
    assert np.allclose(Y, np.fft.fft(np.fft.rfft(S, axis=2), axis=1), atol=1e-12)
    assert np.allclose(O.idft_y(Y), X, atol=1e-12)
    assert np.allclose(O.idft_x(X, nx), np.fft.irfft(X, n=nx, axis=2), atol=1e-12)


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 6, 12), (3, 9, 10), (2, 32, 32)])
def test_round_trip_identity(shape):
    """Forward then backward transform with the column solve disabled (Section 2.1 test)."""
    S = np.random.default_rng(1).standard_normal(shape)
    back = O.idft_x(O.idft_y(O.dft_y(O.dft_x(S))), shape[2])
    assert np.abs(back - S).max() < 1e-13


# ---------------------------------------------------------------------------
# column solves
# ---------------------------------------------------------------------------

def test_thomas_matches_dense_solve():
    rng = np.random.default_rng(5)
    nz = 9
    d = wl.random_stretched(4, 4, nz, seed=5)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0)
    for lam in (-1e-6, -0.3, -4.0):
        T = O.column_matrix(a, c, lam)
        rhs = rng.standard_normal(nz) + 1j * rng.standard_normal(nz)
        diag = np.diag(T).copy()
        x = O.thomas(a, diag, c, rhs)
        assert np.allclose(x, np.linalg.solve(T, rhs), rtol=1e-10, atol=0)
        # transposed operands
        sub_t = np.r_[0.0, c[:-1]]
        sup_t = np.r_[a[1:], 0.0]
        xt = O.thomas(sub_t, diag, sup_t, rhs)
        assert np.allclose(xt, np.linalg.solve(T.T, rhs), rtol=1e-10, atol=0)


def test_singular_column_solve():
    d = wl.random_stretched(4, 4, 8, seed=9)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0)
    T = O.column_matrix(a, c, 0.0)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(8)
    b -= W * (W @ b) / (W @ W)           # compatible: W^T b = 0
    x = O.singular_column_solve(a, c, b)
    assert abs(x.sum()) < 1e-13
    assert np.abs(T @ x - b).max() < 1e-12
    # pseudo-inverse solution differs only by a constant
    xp = np.linalg.lstsq(T, b, rcond=None)[0]
    assert np.allclose(x - x.mean(), xp - xp.mean(), atol=1e-11)


def _mp_column_solve(T, rhs, dps=40):
    """Reference solve of a small dense system in mpmath at dps digits (independent of numpy).

    T: a callable (mpmath module) -> mpmath matrix, so that entries such as -(a_k + c_k) + lam are
    formed at dps digits, or an array of exact entries."""
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(dps):
        A = T(mpmath) if callable(T) else mpmath.matrix([[mpmath.mpf(float(v)) for v in row] for row in T])
        b = mpmath.matrix([mpmath.mpf(float(v)) for v in rhs])
        x = mpmath.lu_solve(A, b)
        return np.array([float(v) for v in x])


def _mp_column(a, c, lam, border=False):
    """T = L_z + lam I (bordered by ones when border) with its entries formed in mpmath."""
    nz = a.size

    def build(mp):
        n = nz + 1 if border else nz
        A = mp.matrix(n, n)
        for k in range(nz):
            A[k, k] = -(mp.mpf(float(a[k])) + mp.mpf(float(c[k]))) + mp.mpf(float(lam))
            if k > 0:
                A[k, k - 1] = mp.mpf(float(a[k]))
            if k < nz - 1:
                A[k, k + 1] = mp.mpf(float(c[k]))
            if border:
                A[k, nz] = 1
                A[nz, k] = 1
        return A
    return build


@pytest.mark.parametrize("nz,lam", [(3, -6.0e-8), (17, -2.4e-8), (128, -1.5e-8)])
def test_weak_column_solve_is_accurate_to_fp64(nz, lam):
    """A column whose row sum lam is 1e5-1e6 times below its couplings (the lowest horizontal
    wavenumbers of the stretched, 50 m grids): the oracle's column solve matches a 40-digit solve
    to FP64 accuracy, where the plain FP64 recurrence loses eps (a + c)/|lam|."""
    dz = wl.stretched_levels(nz)
    rho = wl.exponential_density(dz)
    W, a, c = O.vertical_coefficients(dz, rho)
    rng = np.random.default_rng(nz)
    rhs = rng.standard_normal(nz)
    ref = _mp_column_solve(_mp_column(a, c, lam), rhs)
    lam_arr = np.array([[lam]])
    x = O.poisson_oracle._column_solves(a, c, a, c, lam_arr, rhs[:, None, None].astype(complex),
                                        skip00=False)[:, 0, 0].real
    err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    assert err <= 5e-15, err
    # the same recurrence carried in FP64 (the diagonal -(a + c) + lam rounded to double) is far worse
    x64 = O.thomas(a, -(a + c) + lam, c, rhs)
    err64 = np.linalg.norm(x64 - ref) / np.linalg.norm(ref)
    assert err64 > 20 * err + 1e-14, (err64, err)


def test_singular_column_solve_is_accurate_to_fp64():
    """The (0,0) column on 128 stretched, density-weighted levels (bordered matrix condition ~1e6)
    against a 40-digit bordered solve."""
    nz = 128
    dz = wl.stretched_levels(nz)
    rho = wl.exponential_density(dz)
    W, a, c = O.vertical_coefficients(dz, rho)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(nz)
    b -= W * (W @ b) / (W @ W)
    ref = _mp_column_solve(_mp_column(a, c, 0.0, border=True), np.r_[b, 0.0])[:nz]
    x = O.singular_column_solve(a, c, b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 5e-15


def test_gauss_solve_against_mpmath():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((7, 7))
    b = rng.standard_normal(7)
    x = O.poisson_oracle.gauss_solve(A.astype(O.poisson_oracle.XP), b.astype(O.poisson_oracle.XP)).astype(float)
    assert np.allclose(x, _mp_column_solve(A, b), rtol=1e-14, atol=0)


# ---------------------------------------------------------------------------
# full solve
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [(1, 0, 0), (0, 0, 1), (0, 0, 7), (3, 2, 5), (8, 6, 0), (5, 1, 9)])
def test_solve_eigenfunctions(mode):
    nx, ny, nz, dx, dy, dz = 16, 12, 10, 0.9, 1.7, 0.6
    p_exact = _cos_mode(nx, ny, nz, *mode)
    lam = _cos_mode_eig(nx, ny, nz, *mode, dx, dy, dz)
    p = O.solve(lam * p_exact, dx, dy, np.full(nz, dz), np.full(nz, 1.0))
    assert O.relative_l2(p, p_exact) < 1e-13


def test_solve_sum_of_modes_on_32_cube():
    n = 32
    modes = [(1, 2, 3), (0, 5, 1), (7, 0, 0), (16, 16, 31), (2, 0, 4)]
    p_exact = sum(_cos_mode(n, n, n, *m, phx=0.1 * q, phy=0.2 * q) for q, m in enumerate(modes))
    S = sum(_cos_mode_eig(n, n, n, *m, 1, 1, 1) * _cos_mode(n, n, n, *m, phx=0.1 * q, phy=0.2 * q)
            for q, m in enumerate(modes))
    p = O.solve(S, 1.0, 1.0, np.ones(n), np.ones(n))
    assert O.relative_l2(p, p_exact) < 1e-13


def _dense_L(shape, dx, dy, a, c):
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    e = np.zeros(N)
    for q in range(N):
        e[:] = 0
        e[q] = 1
        A[:, q] = O.apply_L(e.reshape(shape), dx, dy, a, c).ravel()
    return A


@pytest.mark.parametrize("dims,seed", [((4, 6, 5), 1), ((6, 4, 7), 2), ((5, 4, 3), 3), ((8, 6, 4), 4)])
def test_solve_matches_brute_force_bordered_system(dims, seed):
    nx, ny, nz = dims
    d = wl.random_stretched(nx, ny, nz, seed=seed)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0)
    A = _dense_L(d.S.shape, d.dx, d.dy, a, c)
    N = A.shape[0]
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = A
    B[:N, N] = 1
    B[N, :N] = 1
    rhs = np.r_[O.project_compatible(d.S, W).ravel(), 0.0]
    ref = np.linalg.solve(B, rhs)
    assert abs(ref[N]) < 1e-12       # compatible right-hand side: multiplier vanishes
    p = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
    assert O.relative_l2(p, ref[:N].reshape(d.S.shape)) < 1e-12


def test_solve_invariants_blob_workload():
    d = wl.anelastic_blobs(32, 24, 16, seed=2)
    p, info = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0, return_info=True)
    assert abs(p.mean()) < 1e-14 * np.abs(p).mean()
    r = O.residual(d.S, p, d.dx, d.dy, d.dz, d.rho0)
    assert np.linalg.norm(r) / np.linalg.norm(d.S) < 1e-12
    assert abs(info["removed_weighted_mean"]) < 1.0
    # periodic-shift equivariance in x and y
    ps = O.solve(np.roll(d.S, (3, 5), axis=(1, 2)), d.dx, d.dy, d.dz, d.rho0)
    assert O.relative_l2(ps, np.roll(p, (3, 5), axis=(1, 2))) < 1e-13


def test_solve_removes_incompatible_part():
    d = wl.random_stretched(6, 6, 5, seed=8)
    p1 = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
    p2 = O.solve(d.S + 2.5, d.dx, d.dy, d.dz, d.rho0)
    assert O.relative_l2(p2, p1) < 1e-13


# ---------------------------------------------------------------------------
# adjoint and rho0 gradient
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,seed", [((6, 4, 5), 1), ((8, 8, 6), 2), ((5, 6, 4), 3)])
def test_adjoint_dot_product_and_dense_transpose(dims, seed):
    nx, ny, nz = dims
    d = wl.random_stretched(nx, ny, nz, seed=seed)
    rng = np.random.default_rng(seed + 100)
    w = rng.standard_normal(d.S.shape)
    S = rng.standard_normal(d.S.shape)
    p = O.solve(S, d.dx, d.dy, d.dz, d.rho0)
    g = O.adjoint(w, d.dx, d.dy, d.dz, d.rho0)
    lhs = (w * p).sum()
    rhs = (g * S).sum()
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(w * p).sum() + np.abs(g * S).sum())
    # brute force: columns of G by solving unit sources
    N = d.S.size
    G = np.zeros((N, N))
    e = np.zeros(N)
    for q in range(N):
        e[:] = 0
        e[q] = 1
        G[:, q] = O.solve(e.reshape(d.S.shape), d.dx, d.dy, d.dz, d.rho0).ravel()
    assert O.relative_l2(g.ravel(), G.T @ w.ravel()) < 1e-12


def test_rho0_gradient_matches_central_differences():
    d = wl.random_stretched(6, 5, 6, seed=21)
    rng = np.random.default_rng(7)
    w = rng.standard_normal(d.S.shape)
    g = O.rho0_gradient(w, d.S, d.dx, d.dy, d.dz, d.rho0)

    def loss(rho):
        return (w * O.solve(d.S, d.dx, d.dy, d.dz, rho)).sum()

    fd = np.zeros(d.nz)
    for m in range(d.nz):
        eps = 1e-6 * d.rho0[m]
        rp = d.rho0.copy()
        rm = d.rho0.copy()
        rp[m] += eps
        rm[m] -= eps
        fd[m] = (loss(rp) - loss(rm)) / (2 * eps)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(g).max(), (g, fd)


def test_source_gradient_matches_central_differences():
    d = wl.random_stretched(5, 4, 5, seed=22)
    rng = np.random.default_rng(8)
    w = rng.standard_normal(d.S.shape)
    g = O.adjoint(w, d.dx, d.dy, d.dz, d.rho0)
    for q in rng.choice(d.S.size, 6, replace=False):
        Sp = d.S.copy().ravel()
        Sm = Sp.copy()
        Sp[q] += 1e-4
        Sm[q] -= 1e-4
        lp = (w * O.solve(Sp.reshape(d.S.shape), d.dx, d.dy, d.dz, d.rho0)).sum()
        lm = (w * O.solve(Sm.reshape(d.S.shape), d.dx, d.dy, d.dz, d.rho0)).sum()
        assert abs((lp - lm) / 2e-4 - g.ravel()[q]) < 1e-8 * np.abs(g).max()


# ---------------------------------------------------------------------------
# p = 0 on the top face (bc="dirichlet_top")
# ---------------------------------------------------------------------------

def _cos_mode_dt(nx, ny, nz, ax, by, cz, phx=0.3, phy=-0.7):
    """Discrete eigenfunction with zero flux at the bottom and a zero ghost mirror
    at the top face: cos(pi (2c+1)(k+1/2)/(2 nz)) vanishes midway between the top
    centre and its mirror image."""
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    return (np.cos(2 * np.pi * ax * i / nx + phx) * np.cos(2 * np.pi * by * j / ny + phy)
            * np.cos(np.pi * (2 * cz + 1) * (k + 0.5) / (2 * nz)))


def _cos_mode_dt_eig(nx, ny, nz, ax, by, cz, dx, dy, dz):
    return (-4 / dx**2 * np.sin(np.pi * ax / nx) ** 2 - 4 / dy**2 * np.sin(np.pi * by / ny) ** 2
            - 4 / dz**2 * np.sin(np.pi * (2 * cz + 1) / (4 * nz)) ** 2)


def test_dirichlet_top_coefficient_uniform():
    h = 0.7
    W, a, c = O.vertical_coefficients(np.full(6, h), np.full(6, 1.3), bc="dirichlet_top")
    assert a[0] == 0.0
    assert np.allclose(a[1:], 1 / h**2, rtol=1e-14)
    assert np.allclose(c[:-1], 1 / h**2, rtol=1e-14)
    # half a cell from the top centre to the face: twice the interior coupling
    assert np.isclose(c[-1], 2 / h**2, rtol=1e-14)
    with pytest.raises(ValueError):
        O.vertical_coefficients(np.full(6, h), np.full(6, 1.3), bc="dirichlet")


@pytest.mark.parametrize("mode", [(0, 0, 0), (1, 0, 0), (0, 0, 4), (3, 2, 5), (8, 6, 9), (4, 3, 0)])
def test_operator_eigenfunctions_dirichlet_top(mode):
    nx, ny, nz, dx, dy, dz = 16, 12, 10, 0.9, 1.7, 0.6
    p = _cos_mode_dt(nx, ny, nz, *mode)
    W, a, c = O.vertical_coefficients(np.full(nz, dz), np.full(nz, 2.0), bc="dirichlet_top")
    Lp = O.apply_L(p, dx, dy, a, c)
    lam = _cos_mode_dt_eig(nx, ny, nz, *mode, dx, dy, dz)
    assert np.abs(Lp - lam * p).max() <= 1e-13 * np.abs(lam)


@pytest.mark.parametrize("mode", [(0, 0, 0), (1, 0, 0), (0, 0, 7), (3, 2, 5), (8, 6, 0)])
def test_solve_eigenfunctions_dirichlet_top(mode):
    nx, ny, nz, dx, dy, dz = 16, 12, 10, 0.9, 1.7, 0.6
    p_exact = _cos_mode_dt(nx, ny, nz, *mode)
    lam = _cos_mode_dt_eig(nx, ny, nz, *mode, dx, dy, dz)
    p = O.solve(lam * p_exact, dx, dy, np.full(nz, dz), np.full(nz, 1.0), bc="dirichlet_top")
    assert O.relative_l2(p, p_exact) < 1e-13


def test_dirichlet_top_converges_to_continuous_anelastic_problem():
    """Second-order convergence with p = 0 at z = H and zero flux at z = 0.

    Exact solution p = cos(2 pi i/nx) cos(pi z/(2H)) with rho = 1.2 exp(-z/Hs) on
    smoothly stretched levels.  The top flux carries the top cell's density over
    half a cell; measuring the distance to the face as a whole cell instead
    converges at first order only.
    """
    H, Hs, nx, dx = 3000.0, 2500.0, 8, 400.0
    i = np.arange(nx)
    lx = -(4 / dx**2) * np.sin(np.pi / nx) ** 2
    q = np.pi / (2 * H)
    errs = []
    for nz in (32, 64, 128, 256):
        dz = _smooth_grid(nz, H)
        z = wl.cell_centres(dz)
        rho = 1.2 * np.exp(-z / Hs)
        f = np.cos(q * z)
        Lf = -q**2 * np.cos(q * z) + q / Hs * np.sin(q * z)
        hx = np.cos(2 * np.pi * i / nx)[None, None, :] * np.ones((1, 2, 1))
        S = (Lf + lx * f)[:, None, None] * hx
        p = O.solve(S, dx, 1.0, dz, rho, bc="dirichlet_top")
        exact = f[:, None, None] * hx
        errs.append(np.abs(p - exact).max() / np.abs(exact).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.4) and np.all(ratios < 4.3), (errs, ratios)


def test_dirichlet_top_operator_structure():
    d = wl.random_stretched(6, 5, 7, seed=12)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0, bc="dirichlet_top")
    rng = np.random.default_rng(1)
    u = rng.standard_normal(d.S.shape)
    v = rng.standard_normal(d.S.shape)
    Wf = W[:, None, None]
    # W L stays symmetric (the top coupling only adds to the diagonal)
    lhs = (u * Wf * O.apply_L(v, d.dx, d.dy, a, c)).sum()
    rhs = (Wf * O.apply_L(u, d.dx, d.dy, a, c) * v).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # a constant loses exactly the top-face flux
    Lone = O.apply_L(np.ones(d.S.shape), d.dx, d.dy, a, c)
    assert np.abs(Lone[:-1]).max() < 1e-13
    assert np.allclose(Lone[-1], -c[-1], rtol=1e-14)


@pytest.mark.parametrize("dims,seed", [((4, 6, 5), 1), ((6, 4, 7), 2), ((5, 4, 2), 3), ((8, 6, 4), 4)])
def test_dirichlet_top_matches_brute_force(dims, seed):
    nx, ny, nz = dims
    d = wl.random_stretched(nx, ny, nz, seed=seed)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0, bc="dirichlet_top")
    A = _dense_L(d.S.shape, d.dx, d.dy, a, c)
    S = d.S + 0.4          # no compatibility condition: a mean in S is solved for, not removed
    ref = np.linalg.solve(A, S.ravel()).reshape(d.S.shape)
    p = O.solve(S, d.dx, d.dy, d.dz, d.rho0, bc="dirichlet_top")
    assert O.relative_l2(p, ref) < 1e-12
    r = O.residual(S, p, d.dx, d.dy, d.dz, d.rho0, bc="dirichlet_top")
    assert np.linalg.norm(r) < 1e-12 * np.linalg.norm(S)


@pytest.mark.parametrize("dims,seed", [((6, 4, 5), 1), ((5, 6, 3), 3)])
def test_dirichlet_top_adjoint_dot_product_and_dense_transpose(dims, seed):
    nx, ny, nz = dims
    d = wl.random_stretched(nx, ny, nz, seed=seed)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0, bc="dirichlet_top")
    rng = np.random.default_rng(seed + 200)
    w = rng.standard_normal(d.S.shape)
    g = O.adjoint(w, d.dx, d.dy, d.dz, d.rho0, bc="dirichlet_top")
    A = _dense_L(d.S.shape, d.dx, d.dy, a, c)
    ref = np.linalg.solve(A.T, w.ravel())
    assert O.relative_l2(g.ravel(), ref) < 1e-12


def test_dirichlet_top_rho0_gradient_matches_central_differences():
    d = wl.random_stretched(6, 5, 6, seed=23)
    rng = np.random.default_rng(9)
    w = rng.standard_normal(d.S.shape)
    g = O.rho0_gradient(w, d.S, d.dx, d.dy, d.dz, d.rho0, bc="dirichlet_top")

    def loss(rho):
        return (w * O.solve(d.S, d.dx, d.dy, d.dz, rho, bc="dirichlet_top")).sum()

    fd = np.zeros(d.nz)
    for m in range(d.nz):
        eps = 1e-6 * d.rho0[m]
        rp = d.rho0.copy()
        rm = d.rho0.copy()
        rp[m] += eps
        rm[m] -= eps
        fd[m] = (loss(rp) - loss(rm)) / (2 * eps)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(g).max(), (g, fd)


# ---------------------------------------------------------------------------
# variable density (the operator the conjugate-gradient solver inverts)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", ["neumann", "dirichlet_top"])
def test_variable_operator_reduces_to_L_for_level_density(bc):
    d = wl.random_stretched(7, 6, 5, seed=31)
    rho3 = d.rho0[:, None, None] * np.ones(d.S.shape)
    W, a, c = O.vertical_coefficients(d.dz, d.rho0, bc)
    Ap = O.apply_A_var(d.S, d.dx, d.dy, d.dz, rho3, bc)
    assert np.abs(Ap - O.apply_L(d.S, d.dx, d.dy, a, c)).max() <= 1e-13 * np.abs(Ap).max()


@pytest.mark.parametrize("bc", ["neumann", "dirichlet_top"])
def test_variable_operator_structure(bc):
    d = wl.random_stretched(6, 5, 6, seed=32)
    rho3 = wl.perturbed_density(d.nx, d.ny, d.rho0, 0.4, seed=3)
    W = O.weights_var(d.dz, rho3)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(d.S.shape)
    v = rng.standard_normal(d.S.shape)
    Av = O.apply_A_var(v, d.dx, d.dy, d.dz, rho3, bc)
    Au = O.apply_A_var(u, d.dx, d.dy, d.dz, rho3, bc)
    # W A is symmetric and negative (semi)definite
    assert abs((u * W * Av).sum() - (W * Au * v).sum()) < 1e-12 * np.abs(u * W * Av).sum()
    assert (v * W * Av).sum() < 0
    if bc == "neumann":
        assert abs((W * Av).sum()) < 1e-12 * np.abs(W * Av).sum()                 # conservation
        assert np.abs(O.apply_A_var(np.full(d.S.shape, 2.0), d.dx, d.dy, d.dz, rho3)).max() < 1e-13


@pytest.mark.parametrize("dims", [(6, 5, 4), (4, 4, 2), (8, 6, 3)])
@pytest.mark.parametrize("bc", ["neumann", "dirichlet_top"])
def test_variable_solve_reduces_to_fft_solve(dims, bc):
    d = wl.random_stretched(*dims, seed=33)
    rho3 = d.rho0[:, None, None] * np.ones(d.S.shape)
    p = O.solve_var(d.S, d.dx, d.dy, d.dz, rho3, bc)
    assert O.relative_l2(p, O.solve(d.S, d.dx, d.dy, d.dz, d.rho0, bc=bc)) < 1e-12


def test_variable_solve_residual_and_mean():
    d = wl.random_stretched(12, 10, 6, seed=34)
    rho3 = wl.perturbed_density(d.nx, d.ny, d.rho0, 0.5, seed=4)
    p = O.solve_var(d.S, d.dx, d.dy, d.dz, rho3)
    W = O.weights_var(d.dz, rho3)
    r = d.S - (W * d.S).sum() / W.sum() - O.apply_A_var(p, d.dx, d.dy, d.dz, rho3)
    assert np.linalg.norm(r) < 1e-12 * np.linalg.norm(d.S)
    assert abs(p.mean()) < 1e-14 * np.abs(p).mean()


def test_variable_operator_converges_to_continuous_problem():
    """Second-order convergence to (1/rho) div(rho grad p) with rho varying in x and z.

    rho = exp(-z/Hs) (1 + 0.3 cos(kx x)), p = cos(kx x) cos(kz z), kz = pi/H (zero
    flux at z = 0 and H); the source is the continuous operator at the centres,
    made compatible by the discrete projection.  A face density that is not the
    two-cell mean, or a missing 1/rho weighting, spoils the ratio.
    """
    Lx, H, Hs = 4000.0, 3000.0, 2500.0
    kx, kz = 2 * np.pi / Lx, np.pi / H
    errs = []
    for n in (8, 16, 32, 64):
        nx, nz = 2 * n, n
        dx = Lx / nx
        dz = _smooth_grid(nz, H, beta=1.0)
        z = wl.cell_centres(dz)[:, None, None]
        x = ((np.arange(nx) + 0.5) * dx)[None, None, :] * np.ones((1, 2, 1))
        rho3 = np.exp(-z / Hs) * (1 + 0.3 * np.cos(kx * x)) * np.ones((nz, 2, nx))
        p_ex = np.cos(kx * x) * np.cos(kz * z) * np.ones((nz, 2, nx))
        dlnr_dx = -0.3 * kx * np.sin(kx * x) / (1 + 0.3 * np.cos(kx * x))
        Ap = (-(kx**2 + kz**2) * p_ex + dlnr_dx * (-kx * np.sin(kx * x) * np.cos(kz * z))
              + (-1 / Hs) * (-kz * np.cos(kx * x) * np.sin(kz * z)))
        p = O.solve_var(Ap, dx, 1.0, dz, rho3)
        ex = p_ex - p_ex.mean()
        errs.append(np.abs(p - ex).max() / np.abs(ex).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.4) and np.all(ratios < 4.6), (errs, ratios)


@pytest.mark.parametrize("nx,ny", [(8, 6), (12, 9), (10, 16)])
def test_dft_parseval_with_half_spectrum_weights(nx, ny):
    """sum |S|^2 = (1/(nx ny)) sum_k w_kx |S_hat|^2, with w = 1 for kx = 0 (and kx = nx/2 when nx is
    even) and 2 for the other stored bins: energy is kept by the real half-spectrum transform."""
    rng = np.random.default_rng(nx * ny)
    S = rng.standard_normal((3, ny, nx))
    Sh = O.dft_y(O.dft_x(S))
    w = np.full(nx // 2 + 1, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[-1] = 1.0
    lhs = (S ** 2).sum()
    rhs = (w[None, None, :] * np.abs(Sh) ** 2).sum() / (nx * ny)
    assert abs(lhs - rhs) <= 1e-12 * lhs
