"""The fused spectral middle (one persistent kernel for the y-pass, the column solves
and the inverse y-pass of Section 2.1, strip by strip through L2) against the
separate kernels and the oracle.

The fused kernel runs the same compile-time FFT (16 elements per thread, the same
stage-ordered twiddles and swizzle) and the same two-threads-per-column solve as
the separate y-pass (y_kernel 4) and column (col_tile 0) kernels, so the two paths
agree bit for bit; the low-|k| double-precision columns share their code too.
Shapes cover strips cut by a ragged nx/2 + 1, short columns (nz = 2, 3), odd nz, the
p = 0 top face, and every ny the kernel is built for.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Plan

pytestmark = pytest.mark.gpu

# verify=0: the fused kernel does not form the column norms a verification needs, so both paths apply
# every sweep
SEPARATE = dict(y_kernel=4, y_elems=16, col_tile=0, level_chunk=0, verify=0)


def _solve(d, dtype, bc="neumann", **opts):
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype, bc=bc, **opts)
    fd = torch.float32 if dtype == "fp32" else torch.float64
    S = torch.from_numpy(np.ascontiguousarray(d.S)).to("cuda", fd)
    p, info = plan.solve(S, info=True)
    prof = None
    torch.cuda.synchronize()
    return p, info


def _phases(d, dtype, **opts):
    """Launch counts per phase of one solve (the library's own per-phase events)."""
    from paper_2010_14132_gb300 import _native as N
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype, **opts)
    fd = torch.float32 if dtype == "fp32" else torch.float64
    S = torch.from_numpy(np.ascontiguousarray(d.S)).to("cuda", fd)
    plan.solve(S)
    plan.set_option(N.POISSON_OPT_PROFILE, 1)
    N.poisson_plan_profile_read(plan._h)
    plan.solve(S)
    torch.cuda.synchronize()
    ph = N.poisson_plan_profile_read(plan._h)
    return {k: v[1] for k, v in ph.items()}


CASES = [
    (256, 256, 64, "noise"),      # 129 kx: 16 full strips and one of a single kx
    (96, 512, 17, "blobs"),       # 49 kx (ragged strip), odd nz
    (512, 1024, 32, "noise"),     # the bench's ny, 257 kx
    (144, 256, 2, "noise"),       # 73 kx (a strip of one kx), two levels
    (64, 512, 3, "blobs"),        # 33 kx, three levels
]


def _domain(nx, ny, nz, kind, seed):
    return (wl.anelastic_noise if kind == "noise" else wl.anelastic_blobs)(nx, ny, nz, seed=seed)


@pytest.mark.parametrize("dtype", ["fp32", "mixed"])
@pytest.mark.parametrize("case", CASES)
def test_fused_equals_separate_kernels_and_matches_oracle(case, dtype):
    nx, ny, nz, kind = case
    d = _domain(nx, ny, nz, kind, seed=41 + nz)
    pf, infof = _solve(d, dtype, spectral_fused=1, **SEPARATE)
    ps, infos = _solve(d, dtype, spectral_fused=0, **SEPARATE)
    assert torch.equal(pf, ps), float((pf - ps).abs().max())
    assert infof["sweeps"] == infos["sweeps"] and infof["error_estimate"] == infos["error_estimate"]
    ref = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
    err = O.relative_l2(pf.double().cpu().numpy(), ref)
    assert err <= (1e-5 if dtype == "fp32" else 1e-10), err
    if dtype == "mixed":
        assert infof["converged"] and infof["error_estimate"] >= err


@pytest.mark.parametrize("dtype", ["fp32", "mixed"])
def test_fused_dirichlet_top(dtype):
    d = wl.anelastic_blobs(128, 256, 24, seed=47)
    pf, _ = _solve(d, dtype, bc="dirichlet_top", spectral_fused=1, **SEPARATE)
    ps, _ = _solve(d, dtype, bc="dirichlet_top", spectral_fused=0, **SEPARATE)
    assert torch.equal(pf, ps)
    ref = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0, bc="dirichlet_top")
    assert O.relative_l2(pf.double().cpu().numpy(), ref) <= (1e-5 if dtype == "fp32" else 1e-10)


def test_fused_kernel_is_the_one_that_runs():
    """The option on a supported shape: one fused launch per pass, no separate y or column launches."""
    d = wl.anelastic_noise(256, 256, 32, seed=48)
    c = _phases(d, "mixed", max_sweeps=2, tolerance=1e-300, spectral_fused=1)
    assert c["spectral"] == 3 and c["yfwd"] == 0 and c["columns"] == 0 and c["yinv"] == 0, c
    c0 = _phases(d, "mixed", max_sweeps=2, tolerance=1e-300, spectral_fused=0, verify=2)
    assert c0["spectral"] == 0 and c0["yfwd"] == 3 and c0["columns"] == 3 and c0["yinv"] == 3, c0


def test_fused_lowk_radius_change_rebuilds_the_item_list():
    d = wl.anelastic_noise(256, 256, 40, seed=49)
    for r2 in (0, 4, 200):
        pf, info = _solve(d, "mixed", lowk_radius2=r2, spectral_fused=1, **SEPARATE)
        ps, _ = _solve(d, "mixed", lowk_radius2=r2, spectral_fused=0, **SEPARATE)
        assert torch.equal(pf, ps), r2
        assert info["converged"], (r2, info)
