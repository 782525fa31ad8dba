"""GPU: the field alignment contract of the C ABI (include/poisson.h, memory conventions).

The kernels read and write fields two points at a time (16-byte accesses), so every call that
takes device fields rejects a field that does not start on a 16-byte boundary with
POISSON_ERR_INVALID_ARG before anything is launched, and the same call on aligned fields works.
"""
import numpy as np
import pytest
import torch

from paper_2010_14132_gb300 import _native as N
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Batch, Plan

pytestmark = pytest.mark.gpu


def _offset_field(shape, dtype, offset_elems):
    """A contiguous device field whose data starts offset_elems elements into its allocation."""
    n = int(np.prod(shape))
    buf = torch.zeros(n + 4, dtype=dtype, device="cuda")
    return buf[offset_elems:offset_elems + n].view(shape)


@pytest.mark.parametrize("dtype", ["mixed", "fp32", "fp64"])
def test_unaligned_fields_are_rejected(dtype):
    d = wl.anelastic_noise(64, 64, 8, seed=61)
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype)
    fd = plan.field_dtype
    S = torch.from_numpy(np.ascontiguousarray(d.S)).to("cuda", fd)
    bad = 1 if fd == torch.float64 else 2   # 8 bytes past a 16-byte boundary
    S_bad = _offset_field(plan.shape, fd, bad)
    S_bad.copy_(S)
    p_bad = _offset_field(plan.shape, fd, bad)
    for src, out in ((S_bad, None), (S, p_bad)):
        with pytest.raises(N.PoissonError) as ei:
            plan.solve(src, out=out)
        assert ei.value.status == N.POISSON_ERR_INVALID_ARG
    with pytest.raises(N.PoissonError) as ei:
        plan.adjoint(S_bad)
    assert ei.value.status == N.POISSON_ERR_INVALID_ARG
    # aligned views at a 16-byte offset are fine and give the same answer
    good = 2 if fd == torch.float64 else 4
    S_ok = _offset_field(plan.shape, fd, good)
    S_ok.copy_(S)
    p_ok = _offset_field(plan.shape, fd, good)
    plan.solve(S_ok, out=p_ok)
    ref = plan.solve(S)
    torch.cuda.synchronize()
    assert torch.equal(p_ok, ref)


def test_unaligned_batch_field_is_rejected():
    doms = [wl.anelastic_noise(64, 64, 8, seed=62), wl.anelastic_noise(128, 64, 6, seed=63)]
    b = Batch(doms, dtype="mixed")
    S = [torch.from_numpy(np.ascontiguousarray(x.S)).cuda() for x in doms]
    outs = [torch.empty_like(x) for x in S]
    outs[1] = _offset_field(tuple(S[1].shape), torch.float64, 1)
    with pytest.raises(N.PoissonError) as ei:
        b.solve(S, outs)
    assert ei.value.status == N.POISSON_ERR_INVALID_ARG
