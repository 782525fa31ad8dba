"""The solve entry point that allocates nothing (poisson_solve_static_workspace).

It serves callers that cannot call cudaMalloc while they solve (a model driver's
time loop that must not allocate, or a host program that owns the device memory
pool and passes only field pointers).  Its scratch is a fixed device array inside
the library, so it must give the same answer as the ordinary entry point with a
caller-provided workspace, call after call.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import _native as N
from paper_2010_14132_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {N.POISSON_FP64: 1e-12, N.POISSON_FP32: 1e-5, N.POISSON_MIXED: 1e-10}


def _plan(d, dtype):
    return N.poisson_plan_create(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, N.POISSON_BC_PERIODIC_XY_NEUMANN_Z, dtype)


@pytest.mark.parametrize("dtype", [N.POISSON_FP64, N.POISSON_MIXED, N.POISSON_FP32])
def test_static_workspace_matches_caller_workspace(dtype):
    d = wl.anelastic_blobs(64, 48, 16, seed=91)
    plan = _plan(d, dtype)
    try:
        nbytes = N.poisson_plan_workspace_bytes(plan)
        assert nbytes <= N.POISSON_STATIC_WORKSPACE_BYTES
        tdt = torch.float32 if dtype == N.POISSON_FP32 else torch.float64
        S = torch.from_numpy(d.S).to("cuda", tdt)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        wptr = ws.data_ptr() + ((-ws.data_ptr()) % 256)
        stream = torch.cuda.current_stream().cuda_stream
        p_ref = torch.empty_like(S)
        N.poisson_solve(plan, S.data_ptr(), p_ref.data_ptr(), wptr, stream)
        outs = []
        for _ in range(2):   # two calls in a row share the static array
            p = torch.empty_like(S)
            st = N.poisson_solve_static_workspace(plan, S.data_ptr(), p.data_ptr(), stream)
            assert st in (N.POISSON_OK, N.POISSON_ERR_NOT_CONVERGED)
            outs.append(p)
        torch.cuda.synchronize()
        ref = p_ref.double().cpu().numpy()
        for p in outs:
            assert O.relative_l2(p.double().cpu().numpy(), ref) <= TOL[dtype]
        # and both agree with the oracle at the path's tolerance
        oref = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
        assert O.relative_l2(outs[1].double().cpu().numpy(), oref) <= TOL[dtype]
    finally:
        N.poisson_plan_destroy(plan)


def test_static_workspace_rejects_plans_above_the_maximum():
    d = wl.anelastic_noise(512, 512, 64, with_source=False)
    plan = _plan(d, N.POISSON_FP64)
    try:
        assert N.poisson_plan_workspace_bytes(plan) > N.POISSON_STATIC_WORKSPACE_BYTES
        S = torch.zeros((d.nz, d.ny, d.nx), dtype=torch.float64, device="cuda")
        p = torch.empty_like(S)
        st = N.poisson_solve_static_workspace(plan, S.data_ptr(), p.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)
        assert st == N.POISSON_ERR_WORKSPACE
    finally:
        N.poisson_plan_destroy(plan)
