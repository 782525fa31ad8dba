"""The oracle's pins catch plausible mistakes: each test plants one in the oracle (on the
CPU, by replacing one of its functions for the duration of the test) and checks that the
pin meant for it now fails.  Nothing here touches the CUDA path.
"""
import numpy as np
import pytest

import oracle
import oracle.poisson_oracle as P
import test_oracle_pins as pins

_true_vc = P.vertical_coefficients
_true_he = P.horizontal_eigenvalues
_true_tw = P._twiddles
_true_idft_x = P.idft_x
_true_apply_A_var = P.apply_A_var


def _plant(monkeypatch, name, fn):
    """Replace name in the oracle module and in the package namespace the tests use."""
    monkeypatch.setattr(P, name, fn)
    if hasattr(oracle, name):
        monkeypatch.setattr(oracle, name, fn)


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_face_density_from_one_cell_is_caught(monkeypatch):
    def vc(dz, rho0, bc="neumann"):
        W, a, c = _true_vc(dz, rho0, bc)
        rho0 = np.asarray(rho0, float)
        # face density taken from the lower cell instead of the two-cell mean
        a, c = a.copy(), c.copy()
        a[1:] *= rho0[:-1] / (0.5 * (rho0[:-1] + rho0[1:]))
        c[:-1] *= rho0[:-1] / (0.5 * (rho0[:-1] + rho0[1:]))
        return W, a, c
    _plant(monkeypatch, "vertical_coefficients", vc)
    # still conservative (both sides of a face use the same density), so only the convergence pin sees it
    pins.test_flux_symmetry_stretched()
    _fails(pins.test_solution_converges_to_continuous_anelastic_problem)


def test_centre_spacing_of_one_cell_is_caught(monkeypatch):
    def vc(dz, rho0, bc="neumann"):
        W, a, c = _true_vc(dz, rho0, bc)
        dz = np.asarray(dz, float)
        h = 0.5 * (dz[:-1] + dz[1:])
        a, c = a.copy(), c.copy()
        c[:-1] *= h / dz[:-1]          # the cell thickness used as the centre spacing
        a[1:] *= h / dz[1:]
        return W, a, c
    _plant(monkeypatch, "vertical_coefficients", vc)
    _fails(pins.test_solution_converges_to_continuous_anelastic_problem)


def test_weight_without_density_is_caught(monkeypatch):
    def vc(dz, rho0, bc="neumann"):
        W, a, c = _true_vc(dz, rho0, bc)
        rho0 = np.asarray(rho0, float)
        return W / rho0, a * rho0, c * rho0     # W = dz: the coefficients lose their 1/rho
    _plant(monkeypatch, "vertical_coefficients", vc)
    _fails(pins.test_solution_converges_to_continuous_anelastic_problem)


def test_dirichlet_distance_of_a_whole_cell_is_caught(monkeypatch):
    def vc(dz, rho0, bc="neumann"):
        W, a, c = _true_vc(dz, rho0, bc)
        if bc == "dirichlet_top":
            c = c.copy()
            c[-1] *= 0.5
        return W, a, c
    _plant(monkeypatch, "vertical_coefficients", vc)
    _fails(pins.test_dirichlet_top_coefficient_uniform)
    _fails(pins.test_dirichlet_top_converges_to_continuous_anelastic_problem)


def test_sign_of_the_horizontal_eigenvalue_is_caught(monkeypatch):
    _plant(monkeypatch, "horizontal_eigenvalues", lambda n, d, count=None: -_true_he(n, d, count))
    _fails(pins.test_solve_eigenfunctions, (3, 2, 5))


def test_conjugated_twiddles_are_caught(monkeypatch):
    _plant(monkeypatch, "_twiddles", lambda n, count, sign: _true_tw(n, count, -sign))
    _fails(pins.test_dft_matches_numpy_fft, 12, 9)


def test_missing_inverse_scaling_is_caught(monkeypatch):
    def idft_x(X, nx):
        return _true_idft_x(X, nx) * nx   # the 1/nx dropped
    _plant(monkeypatch, "idft_x", idft_x)
    _fails(pins.test_round_trip_identity, (5, 6, 12))


def test_plain_mean_projection_is_caught(monkeypatch):
    def wm(S, W):
        return float(np.asarray(S, float).mean())   # W ignored
    _plant(monkeypatch, "weighted_mean", wm)
    _fails(pins.test_projection)


def test_untransposed_adjoint_column_is_caught(monkeypatch):
    def adjoint(wgt, dx, dy, dz, rho0, bc="neumann"):
        # the forward solve used as its own adjoint: right only if every column matrix were symmetric
        return P.solve(wgt, dx, dy, dz, rho0, bc=bc)
    _plant(monkeypatch, "adjoint", adjoint)
    _fails(pins.test_adjoint_dot_product_and_dense_transpose, (6, 4, 5), 1)


def test_double_counted_stencil_entry_is_caught(monkeypatch):
    # the assembly mistake the convergence pin found once: a coupling counted twice
    def apply_A_var(p, dx, dy, dz, rho3, bc="neumann"):
        out = _true_apply_A_var(p, dx, dy, dz, rho3, bc)
        return out + (np.roll(p, -1, axis=1) - p) / (dy * dy) * 0.5
    _plant(monkeypatch, "apply_A_var", apply_A_var)
    _fails(pins.test_variable_solve_reduces_to_fft_solve, (6, 5, 4), "neumann")
