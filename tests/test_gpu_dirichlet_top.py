"""GPU parity with p = 0 on the top face (bc="dirichlet_top") against the FP64 oracle.

The top coupling c_{nz-1} enters the last pivot of every column (so the (0,0)
column is nonsingular and nothing is projected or pinned), the mirror recurrence
of the twisted column kernel starts from the top row's sum, and the residual of
the refinement sweeps couples the top level to the face value 0.  Tolerances as
for zero flux: FP64 <= 1e-12, FP32 <= 1e-5, mixed <= 1e-10 relative L2.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Plan

pytestmark = pytest.mark.gpu

BC = "dirichlet_top"
TOL = {"fp64": 1e-12, "fp32": 1e-5, "mixed": 1e-10}


def _solve(d, dtype, S=None, **opts):
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype, bc=BC, **opts)
    S = d.S if S is None else S
    St = torch.from_numpy(np.ascontiguousarray(S)).to("cuda", plan.field_dtype)
    p, info = plan.solve(St, info=True)
    torch.cuda.synchronize()
    return p.double().cpu().numpy(), info


def _check(d, dtype, S=None, tol=None, **opts):
    S = d.S if S is None else S
    p, info = _solve(d, dtype, S=S, **opts)
    ref = O.solve(S, d.dx, d.dy, d.dz, d.rho0, bc=BC)
    err = O.relative_l2(p, ref)
    assert np.isfinite(p).all()
    assert err <= (tol if tol is not None else TOL[dtype]), (dtype, d.name, err, info)
    return err, info


@pytest.mark.parametrize("nx,ny,nz", [(4, 4, 2), (6, 4, 3), (12, 48, 7), (64, 96, 16), (256, 128, 24),
                                      (128, 256, 33)])
@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
def test_sizes(nx, ny, nz, dtype):
    d = wl.random_stretched(nx, ny, nz, seed=nx + 2 * ny + 3 * nz)
    err, info = _check(d, dtype)
    assert info["removed_weighted_mean"] == 0.0


def test_anelastic_noise_mixed_converges():
    d = wl.anelastic_noise(512, 512, 64, seed=31)
    err, info = _check(d, "mixed")
    assert info["converged"] and 1 <= info["sweeps"] <= 3, info


@pytest.mark.parametrize("opts", [dict(col_tile=0), dict(col_tile=1), dict(col_tile=3), dict(col_tile=4),
                                  dict(col_tile=16), dict(col_tile=64), dict(x_kernel=1), dict(y_kernel=1),
                                  dict(lowk_radius2=0), dict(level_chunk=5)])
@pytest.mark.parametrize("dtype", ["fp32", "mixed"])
def test_kernel_shape_options(opts, dtype):
    d = wl.anelastic_noise(256, 128, 24, seed=33)
    _check(d, dtype, **opts)


def test_mixed_three_sweeps():
    d = wl.anelastic_noise(128, 96, 32, seed=34)
    p, info = _solve(d, "mixed", tolerance=1e-30)
    assert info["sweeps"] == 3, info
    assert O.relative_l2(p, O.solve(d.S, d.dx, d.dy, d.dz, d.rho0, bc=BC)) <= 1e-11


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
def test_constant_source_is_solved_not_removed(dtype):
    """With zero flux a constant source is projected away; with p = 0 at the top it
    drives a horizontally uniform profile that the solve must reproduce."""
    d = wl.random_stretched(32, 24, 12, seed=35)
    S = np.full(d.S.shape, 0.75)
    err, info = _check(d, dtype, S=S)
    p, _ = _solve(d, dtype, S=S)
    assert np.abs(p).max() > 0.0


@pytest.mark.parametrize("mode", [(0, 0, 0), (1, 0, 0), (0, 0, 9), (5, 3, 7), (16, 16, 2)])
@pytest.mark.parametrize("dtype", ["fp64", "mixed"])
def test_eigenfunctions_uniform(mode, dtype):
    """Closed form (no oracle): cos(pi (2c+1)(k+1/2)/(2 nz)) times horizontal cosines."""
    n, nz = 32, 24
    ax, by, cz = mode
    i = np.arange(n)[None, None, :]
    j = np.arange(n)[None, :, None]
    k = np.arange(nz)[:, None, None]
    p_exact = (np.cos(2 * np.pi * ax * i / n + 0.2) * np.cos(2 * np.pi * by * j / n - 0.4)
               * np.cos(np.pi * (2 * cz + 1) * (k + 0.5) / (2 * nz)))
    lam = (-4 * np.sin(np.pi * ax / n) ** 2 - 4 * np.sin(np.pi * by / n) ** 2
           - 4 * np.sin(np.pi * (2 * cz + 1) / (4 * nz)) ** 2)
    d = wl.Domain(n, n, nz, 1.0, 1.0, np.ones(nz), np.ones(nz), lam * p_exact, name="cos_mode_dirichlet_top")
    p, _ = _solve(d, dtype)
    assert O.relative_l2(p, p_exact) <= 1e-12


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("dims", [(64, 48, 16), (6, 4, 3), (12, 96, 2)])
def test_adjoint_and_rho_gradient(dtype, dims):
    nx, ny, nz = dims
    d = wl.random_stretched(nx, ny, nz, seed=sum(dims) + 1)
    w = np.random.default_rng(4).standard_normal(d.S.shape)
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype, bc=BC)
    to = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", plan.field_dtype)
    p = plan.solve(to(d.S))
    gS, grho = plan.adjoint(to(w), p=p, want_grho=True)
    torch.cuda.synchronize()
    g_ref = O.adjoint(w, d.dx, d.dy, d.dz, d.rho0, bc=BC)
    tol = {"fp64": 1e-12, "fp32": 1e-5, "mixed": 1e-5}[dtype]
    assert O.relative_l2(gS.double().cpu().numpy(), g_ref) <= tol
    r_ref = O.rho0_gradient(w, d.S, d.dx, d.dy, d.dz, d.rho0, bc=BC)
    err = np.abs(grho.cpu().numpy() - r_ref).max() / np.abs(r_ref).max()
    assert err <= {"fp64": 1e-10, "fp32": 1e-4, "mixed": 1e-4}[dtype], err


def test_set_rho0_keeps_the_top_coupling():
    d = wl.random_stretched(48, 32, 10, seed=36)
    rho_new = d.rho0 * np.linspace(1.0, 0.7, d.nz)
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="fp64", bc=BC)
    plan.set_rho0(torch.from_numpy(rho_new).cuda())
    p = plan.solve(torch.from_numpy(d.S).cuda())
    ref = O.solve(d.S, d.dx, d.dy, d.dz, rho_new, bc=BC)
    assert O.relative_l2(p.cpu().numpy(), ref) <= 1e-12
