"""GPU: fields in MONC's z-fastest order ([nx][ny][nz], layout "xyz").

The library converts such fields to its own [nz][ny][nx] order in the workspace,
runs the same kernels, and converts back, so every result must equal, bit for
bit, the transposed result of the default layout; one case is also checked
against the oracle directly.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Plan, Pipe

pytestmark = pytest.mark.gpu


def _plans(d, dtype, **kw):
    px = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype, **kw)
    pz = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype, layout="xyz", **kw)
    return px, pz


def _zfast(x):
    """[nz][ny][nx] -> [nx][ny][nz]"""
    return x.permute(2, 1, 0).contiguous()


@pytest.mark.parametrize("dims", [(4, 4, 2), (12, 48, 7), (96, 64, 33), (256, 128, 24), (64, 36, 40)])
@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("bc", ["neumann", "dirichlet_top"])
def test_solve_equals_default_layout(dims, dtype, bc):
    d = wl.random_stretched(*dims, seed=sum(dims) + 5)
    px, pz = _plans(d, dtype, bc=bc)
    assert pz.shape == (d.nx, d.ny, d.nz)
    assert pz.workspace_bytes() > px.workspace_bytes()
    S = torch.from_numpy(d.S).to("cuda", px.field_dtype)
    p_x = px.solve(S)
    p_z = pz.solve(_zfast(S))
    torch.cuda.synchronize()
    assert torch.equal(_zfast(p_x), p_z)


def test_solve_matches_oracle_zfast():
    d = wl.anelastic_noise(128, 96, 20, seed=51)
    _, pz = _plans(d, "mixed")
    p_z = pz.solve(_zfast(torch.from_numpy(d.S).cuda()))
    ref = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
    assert O.relative_l2(p_z.permute(2, 1, 0).cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
def test_adjoint_equals_default_layout(dtype):
    d = wl.random_stretched(48, 36, 14, seed=52)
    px, pz = _plans(d, dtype)
    S = torch.from_numpy(d.S).to("cuda", px.field_dtype)
    w = torch.from_numpy(np.random.default_rng(6).standard_normal(d.S.shape)).to("cuda", px.field_dtype)
    p_x = px.solve(S)
    g_x, r_x = px.adjoint(w, p=p_x, want_grho=True)
    p_z = pz.solve(_zfast(S))
    g_z, r_z = pz.adjoint(_zfast(w), p=p_z, want_grho=True)
    torch.cuda.synchronize()
    assert torch.equal(_zfast(g_x), g_z)
    assert torch.equal(r_x, r_z)


def test_pipe_with_zfast_fields():
    d = wl.anelastic_noise(64, 48, 12, seed=53)
    _, pz = _plans(d, "mixed")
    rng = np.random.default_rng(7)
    srcs = [torch.from_numpy(rng.standard_normal(pz.shape)).pin_memory() for _ in range(3)]
    outs = [torch.empty(pz.shape, dtype=torch.float64).pin_memory() for _ in srcs]
    pipe = Pipe(pz)
    for S, p in zip(srcs, outs):
        pipe.submit(S, p)
    pipe.wait()
    for S, p in zip(srcs, outs):
        assert torch.equal(p, pz.solve(S.cuda()).cpu())
