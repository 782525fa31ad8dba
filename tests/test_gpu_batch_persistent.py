"""The persistent multi-domain kernel of the mixed batch: every step of every
domain's direct solve (Section 2.1) and refinement (Section 2.2) in one launch over
a (domain, phase, tile) work list with per-domain dependency counters.

* Every supported nx and ny (64, 128, 256, 384 = 3 x 128, 512), square and
  non-square domains, dx == dy and dx != dy, nz from 2 (one level per column
  half) to odd, ragged and the largest (128) level counts: each domain against
  the oracle at the mixed tolerance, with the error bound covering the error.
* The same batch through the graph of per-domain launches: the same sweeps and
  fields equal to rounding (the two forms share every kernel's arithmetic; only the
  order of the norm sums differs).
* Replays are bit-identical (fixed-order sums, whatever CTA runs an item).
* The graph form gives the same bits whatever its number of concurrent branches.
* Bounded waits: the test hook makes one domain's first control item wait for a
  work count that never arrives; the wait runs out, the solve reports
  POISSON_ERR_TIMEOUT without a fault, and the next solve on the same context is
  correct again.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import _native as N
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Batch

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 2), (128, 128, 7), (256, 256, 33), (384, 384, 48), (512, 512, 20), (64, 512, 9),
          (512, 64, 5), (384, 128, 17), (128, 384, 3), (256, 512, 128)]


@pytest.fixture(scope="module")
def mixed_shapes():
    doms = [wl.anelastic_noise(nx, ny, nz, seed=200 + i) for i, (nx, ny, nz) in enumerate(SHAPES)]
    # dx != dy (the general horizontal residual term) and irregular levels and densities
    doms += [wl.random_stretched(128, 256, 12, seed=5), wl.random_stretched(384, 64, 6, seed=6)]
    refs = [O.solve(d.S, d.dx, d.dy, d.dz, d.rho0) for d in doms]
    return doms, refs


def _sources(doms):
    return [torch.from_numpy(np.ascontiguousarray(d.S)).to("cuda", torch.float64) for d in doms]


def test_every_shape_against_the_oracle(mixed_shapes):
    doms, refs = mixed_shapes
    b = Batch(doms, dtype="mixed", persistent=True)
    outs, infos = b.solve(_sources(doms), info=True)
    torch.cuda.synchronize()
    for d, p, ref, info in zip(doms, outs, refs, infos):
        err = O.relative_l2(p.cpu().numpy(), ref)
        assert err <= 1e-10, (d.name, err, info)
        assert info["converged"] and info["sweeps"] >= 1, (d.name, info)
        assert info["error_estimate"] >= err, (d.name, err, info)
        assert 0 < info["accuracy_floor"] <= info["error_estimate"]
        r = [x for x in info["rel_residual"] if x >= 0]
        assert r and all(b_ < a for a, b_ in zip(r, r[1:])), (d.name, info)


def test_persistent_equals_graph_of_launches(mixed_shapes):
    doms, _ = mixed_shapes
    S = _sources(doms)
    bp = Batch(doms, dtype="mixed", persistent=True)
    bg = Batch(doms, dtype="mixed", persistent=False)
    op, ip = bp.solve(S, info=True)
    og, ig = bg.solve(S, info=True)
    op2 = bp.solve(S)   # graph replay of the persistent launch
    torch.cuda.synchronize()
    for d, a, g, a2, ia, ib in zip(doms, op, og, op2, ip, ig):
        assert torch.equal(a, a2), d.name
        assert ia["sweeps"] == ib["sweeps"] and ia["converged"] == ib["converged"], (d.name, ia, ib)
        assert ia["removed_weighted_mean"] == pytest.approx(ib["removed_weighted_mean"], rel=1e-12, abs=1e-18)
        diff = (torch.linalg.vector_norm(a - g) / torch.linalg.vector_norm(g)).item()
        assert diff <= 1e-12, (d.name, diff)


def test_timeout_is_reported_and_the_context_stays_usable(mixed_shapes):
    doms, refs = mixed_shapes
    doms, refs = doms[:4], refs[:4]
    b = Batch(doms, dtype="mixed", persistent=True)
    S = _sources(doms)
    b.set_option(N.POISSON_BATCH_OPT_STALL_TEST, 1)
    with pytest.raises(N.PoissonError) as ei:
        b.solve(S, info=True)
    assert ei.value.status == N.POISSON_ERR_TIMEOUT
    torch.cuda.synchronize()   # the launch ended by itself
    b.set_option(N.POISSON_BATCH_OPT_STALL_TEST, -1)
    outs = b.solve(S)
    torch.cuda.synchronize()
    for d, p, ref in zip(doms, outs, refs):
        assert O.relative_l2(p.cpu().numpy(), ref) <= 1e-10, d.name


def test_branch_count_leaves_the_graph_form_bitwise_unchanged(mixed_shapes):
    doms, _ = mixed_shapes
    S = _sources(doms)
    b = Batch(doms, dtype="mixed", persistent=False)
    ref = [p.clone() for p in b.solve(S)]
    for nb in (1, 5, 32):
        b.set_option(N.POISSON_BATCH_OPT_BRANCHES, nb)
        outs = b.solve(S)
        torch.cuda.synchronize()
        for d, a, r in zip(doms, outs, ref):
            assert torch.equal(a, r), (nb, d.name)


def test_batch_options_are_checked():
    doms = [wl.anelastic_noise(64, 64, 4, seed=1)]
    b = Batch(doms, dtype="mixed")
    for opt, val in ((N.POISSON_BATCH_OPT_PERSISTENT, 2), (N.POISSON_BATCH_OPT_STALL_TEST, 1),
                     (N.POISSON_BATCH_OPT_STALL_TEST, 0.5), (N.POISSON_BATCH_OPT_BRANCHES, 0),
                     (N.POISSON_BATCH_OPT_BRANCHES, 33), (N.POISSON_BATCH_OPT_BRANCHES, 2.5), (7, 0)):
        with pytest.raises(N.PoissonError):
            b.set_option(opt, val)
