"""GPU: a mixed solve replayed from the plan's captured graph (POISSON_OPT_GRAPH, default on) equals the
same solve from plain stream launches, bit for bit, with its sweeps after the first as graph IF nodes.

* Certified after the first try (the later sweeps skipped), and with a tolerance only the full second
  sweep meets (the IF node's body runs), against plain launches and the oracle.
* The graph is reused for the same pointers, captured again for new pointers or after an option change
  (up to four pointer sets are kept), and the reported information matches.
* Fields in MONC's z-fastest order (the transposes are captured too).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import _native as N
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Plan

pytestmark = pytest.mark.gpu


def _pair(d, **opts):
    pg = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed", graph=1, **opts)
    pd = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed", graph=0, **opts)
    return pg, pd


def _info_core(i):
    return (i["sweeps"], i["converged"], i["error_estimate"], tuple(i["rel_update"]), tuple(i["rel_residual"]))


@pytest.mark.parametrize("tol", [1e-10, None])
def test_graph_replay_equals_plain_launches(tol):
    d = wl.anelastic_noise(384, 256, 64, seed=21)
    opts = {}
    if tol is None:   # between the first try's bound and the full verification's: sweep 2's IF body runs
        _, il = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed").solve(
            torch.from_numpy(np.ascontiguousarray(d.S)).cuda(), info=True)
        _, if_ = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed", verify=2).solve(
            torch.from_numpy(np.ascontiguousarray(d.S)).cuda(), info=True)
        assert il["error_estimate"] > if_["error_estimate"] * 1.001, (il, if_)
        opts["tolerance"] = (il["error_estimate"] * if_["error_estimate"]) ** 0.5
    pg, pd = _pair(d, **opts)
    S = torch.from_numpy(np.ascontiguousarray(d.S)).cuda()
    outs = [torch.empty_like(S) for _ in range(6)]
    infos = []
    # the same pointers three times (one capture), then new pointers (captures), then the first again
    for i in (0, 0, 0, 1, 2, 3, 4, 5, 0):
        _, inf = pg.solve(S, out=outs[i], info=True)
        infos.append(inf)
    ref, iref = pd.solve(S, info=True)
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)
    for inf in infos:
        assert _info_core(inf) == _info_core(iref), (inf, iref)
    assert O.relative_l2(ref.cpu().numpy(), O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)) <= iref["error_estimate"]
    # an option change is seen by the next replay
    N.poisson_plan_set_option(pg._h, N.POISSON_OPT_VERIFY, 2)
    N.poisson_plan_set_option(pd._h, N.POISSON_OPT_VERIFY, 2)
    a, ia = pg.solve(S, out=outs[0], info=True)
    b, ib = pd.solve(S, info=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and _info_core(ia) == _info_core(ib)


def test_graph_replay_z_fastest_layout():
    d = wl.anelastic_noise(256, 192, 24, seed=72)
    pg, pd = _pair(d, layout="xyz")
    Sz = torch.from_numpy(np.ascontiguousarray(d.S.transpose(2, 1, 0))).cuda()
    a = pg.solve(Sz)
    a2 = pg.solve(Sz, out=a.clone())
    b = pd.solve(Sz)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a2, b)


def test_graph_replay_after_set_rho0():
    """The plan's tables for rho0 are rebuilt in place (coefficients, limiting accuracy, low-|k| pivots),
    so a graph captured before poisson_plan_set_rho0 replays the solve for the new density: equal, bit for
    bit, to a plan created with that density."""
    d = wl.anelastic_noise(256, 192, 32, seed=73)
    S = torch.from_numpy(np.ascontiguousarray(d.S)).cuda()
    pg = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed", graph=1)
    out = torch.empty_like(S)
    pg.solve(S, out=out)                       # captures the graph for (S, out, workspace)
    rho_new = d.rho0 * (1.0 + 0.05 * np.cos(np.linspace(0.0, 3.0, d.nz)))
    pg.set_rho0(torch.from_numpy(rho_new).cuda())
    _, ig = pg.solve(S, out=out, info=True)    # replayed
    fresh = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, rho_new, dtype="mixed", graph=0)
    ref, ir = fresh.solve(S, info=True)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert _info_core(ig) == _info_core(ir)
    assert O.relative_l2(ref.cpu().numpy(), O.solve(d.S, d.dx, d.dy, d.dz, rho_new)) <= ir["error_estimate"]
