"""GPU: preconditioned conjugate gradients for a density varying in x, y and z.

Checked against the oracle's sparse direct solve of the same flux-form operator
(moderate sizes), against the FFT solve when the density is a level profile
(the preconditioner is then exact), and by the oracle's operator on the GPU
solution (a residual that holds at any size).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Plan

pytestmark = pytest.mark.gpu


def _setup(dims, eps, seed, dtype="fp64", bc="neumann", **opts):
    d = wl.random_stretched(*dims, seed=seed)
    rho3 = wl.perturbed_density(d.nx, d.ny, d.rho0, eps, seed=seed + 1)
    rho_bar = rho3.mean(axis=(1, 2))
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, rho_bar, dtype=dtype, bc=bc, **opts)
    return d, rho3, plan


def _cg(plan, rho3, S, **kw):
    p, info = plan.cg_solve(torch.from_numpy(rho3).cuda(), torch.from_numpy(S).cuda(), **kw)
    torch.cuda.synchronize()
    return p.cpu().numpy(), info


@pytest.mark.parametrize("bc", ["neumann", "dirichlet_top"])
def test_level_density_converges_in_one_step(bc):
    d, _, plan = _setup((48, 32, 12), 0.0, 61, bc=bc)
    rho3 = d.rho0[:, None, None] * np.ones(d.S.shape)
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="fp64", bc=bc)
    p, info = _cg(plan, rho3, d.S, tol=1e-10)
    assert info["converged"] and info["iterations"] <= 2, info
    assert O.relative_l2(p, O.solve(d.S, d.dx, d.dy, d.dz, d.rho0, bc=bc)) <= 1e-10


@pytest.mark.parametrize("dims", [(32, 24, 12), (48, 32, 10), (12, 48, 7)])
@pytest.mark.parametrize("bc", ["neumann", "dirichlet_top"])
@pytest.mark.parametrize("dtype", ["fp64", "mixed"])
def test_matches_oracle_sparse_solve(dims, bc, dtype):
    opts = {"max_sweeps": 0} if dtype == "mixed" else {}
    d, rho3, plan = _setup(dims, 0.3, sum(dims), dtype=dtype, bc=bc, **opts)
    p, info = _cg(plan, rho3, d.S, tol=1e-12, max_iter=100)
    assert info["converged"], info
    ref = O.solve_var(d.S, d.dx, d.dy, d.dz, rho3, bc)
    assert O.relative_l2(p, ref) <= 1e-9, (O.relative_l2(p, ref), info)
    if bc == "neumann":
        W = O.weights_var(d.dz, rho3)
        assert abs(info["removed_weighted_mean"] - (W * d.S).sum() / W.sum()) <= 1e-12 * np.abs(d.S).max()
        assert abs(p.mean()) <= 1e-13 * np.abs(p).max()


def test_residual_at_a_larger_size():
    d, rho3, plan = _setup((256, 192, 48), 0.2, 62, dtype="mixed", max_sweeps=0)
    p, info = _cg(plan, rho3, d.S, tol=1e-10, max_iter=100)
    assert info["converged"], info
    W = O.weights_var(d.dz, rho3)
    r = d.S - (W * d.S).sum() / W.sum() - O.apply_A_var(p, d.dx, d.dy, d.dz, rho3)
    assert np.linalg.norm(r) / np.linalg.norm(d.S) <= 2e-10
    assert abs(info["rel_residual"] - np.linalg.norm(r) / np.linalg.norm(d.S)) <= 1e-10


def test_iterations_grow_with_the_perturbation():
    its = []
    for eps in (0.02, 0.2, 0.6):
        d, rho3, plan = _setup((64, 48, 16), eps, 63)
        _, info = _cg(plan, rho3, d.S, tol=1e-10, max_iter=200)
        assert info["converged"], (eps, info)
        its.append(info["iterations"])
    assert its[0] < its[1] < its[2], its


def test_not_converged_reports_the_last_iterate():
    d, rho3, plan = _setup((32, 24, 12), 0.5, 64)
    p, info = _cg(plan, rho3, d.S, tol=1e-14, max_iter=2)
    assert not info["converged"] and info["iterations"] == 2, info
    assert np.isfinite(p).all() and 0 < info["rel_residual"] < 1
