"""GPU: the host-buffer pipeline (poisson_pipe_*) gives the device solve's results.

Each step's output must equal, bit for bit, plan.solve on the same source
(same kernels, same deterministic reductions), for page-locked and for pageable
host buffers, with more steps than device slots so that slots are reused.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Plan, Pipe

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["mixed", "fp32", "fp64"])
@pytest.mark.parametrize("pinned", [True, False])
def test_pipe_matches_device_solve(dtype, pinned):
    d = wl.anelastic_noise(128, 96, 24, seed=41)
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype)
    rng = np.random.default_rng(5)
    sources = []
    for i in range(5):
        S = rng.standard_normal(plan.shape)
        S -= S.mean()
        sources.append(torch.from_numpy(S).to(plan.field_dtype))
    if pinned:
        sources = [s.pin_memory() for s in sources]
    outs = [torch.empty(plan.shape, dtype=plan.field_dtype) for _ in sources]
    if pinned:
        outs = [o.pin_memory() for o in outs]
    pipe = Pipe(plan)
    for S, p in zip(sources, outs):
        pipe.submit(S, p)
    pipe.wait()
    for S, p in zip(sources, outs):
        ref = plan.solve(S.cuda()).cpu()
        assert torch.equal(p, ref)
    # and the first step against the oracle
    err = O.relative_l2(outs[0].double().numpy(), O.solve(sources[0].double().numpy(), d.dx, d.dy, d.dz, d.rho0))
    assert err <= {"fp64": 1e-12, "fp32": 1e-5, "mixed": 1e-10}[dtype]
    pipe.close()
    plan.close()


def test_pipe_rejects_device_tensors():
    d = wl.anelastic_noise(64, 64, 8, seed=42)
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed")
    pipe = Pipe(plan)
    S = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        pipe.submit(S, torch.empty(plan.shape, dtype=torch.float64))
    pipe.close()


def test_pipe_reports_each_steps_status():
    """The per-step status (done, sweeps, converged, error bits) reaches the host ring at wait(): a
    tolerance below the limiting accuracy is never met, so the mixed steps end NOT_CONVERGED; the
    same sources with the default tolerance converge."""
    from paper_2010_14132_gb300 import _native as N
    d = wl.anelastic_noise(128, 96, 24, seed=43)
    S = torch.from_numpy(np.ascontiguousarray(d.S)).pin_memory()
    outs = [torch.empty_like(S).pin_memory() for _ in range(3)]
    strict = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed", tolerance=1e-300)
    pipe = Pipe(strict)
    for p in outs:
        pipe.submit(S, p)
    with pytest.raises(N.PoissonError) as ei:
        pipe.wait()
    assert ei.value.status == N.POISSON_ERR_NOT_CONVERGED
    pipe.close()
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed")
    pipe = Pipe(plan)
    for p in outs:
        pipe.submit(S, p)
    pipe.wait()
    ref = plan.solve(S.cuda()).cpu()
    for p in outs:
        assert torch.equal(p, ref)
    pipe.close()
