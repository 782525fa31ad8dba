"""Stored expected values (tests/golden/oracle_small_cases.json, written by
tests/golden/make_golden.py from the oracle only).

CPU: the stored solutions satisfy their defining equations with the oracle's
operator (residual and mean, independent of the solve that produced them), and the
oracle still reproduces them.  GPU: the CUDA path reproduces them.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "oracle_small_cases.json")))["cases"]

import importlib.util  # noqa: E402
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
MG = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(MG)


def _stored(case):
    return np.array(case["p"]).reshape(case["shape"])


@pytest.mark.parametrize("case", GOLDEN, ids=[c["name"] for c in GOLDEN])
def test_stored_solution_satisfies_its_equation(case):
    d, rho3 = MG.inputs(case)
    p = _stored(case)
    bc = case["bc"]
    if rho3 is None:
        r = O.residual(d.S, p, d.dx, d.dy, d.dz, d.rho0, bc=bc)
    else:
        W = O.weights_var(d.dz, rho3)
        rhs = d.S - ((W * d.S).sum() / W.sum() if bc == "neumann" else 0.0)
        r = rhs - O.apply_A_var(p, d.dx, d.dy, d.dz, rho3, bc)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(d.S)
    if bc == "neumann":
        assert abs(p.mean()) <= 1e-14 * np.abs(p).max()
    assert np.isclose(np.linalg.norm(p), case["l2"], rtol=1e-14)


@pytest.mark.parametrize("case", GOLDEN, ids=[c["name"] for c in GOLDEN])
def test_oracle_reproduces_stored_solution(case):
    assert O.relative_l2(MG.solve(case), _stored(case)) <= 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("case", GOLDEN, ids=[c["name"] for c in GOLDEN])
def test_gpu_reproduces_stored_solution(case):
    from paper_2010_14132_gb300.solver import Plan
    d, rho3 = MG.inputs(case)
    S = torch.from_numpy(d.S).cuda()
    if rho3 is None:
        plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="fp64", bc=case["bc"])
        p = plan.solve(S)
    else:
        plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, rho3.mean(axis=(1, 2)), dtype="fp64", bc=case["bc"])
        p, info = plan.cg_solve(torch.from_numpy(rho3).cuda(), S, tol=1e-13, max_iter=200)
        assert info["converged"], info
    torch.cuda.synchronize()
    assert O.relative_l2(p.cpu().numpy(), _stored(case)) <= 1e-11
