"""GPU: the precision ladder of the accuracy/time study (analogue of Table 1, Section 3).

The FP64 rung is checked against the FP64 CPU oracle first, so that the study's
reference is itself pinned; then each rung's distance from it must fall as the
ladder is climbed: FP32, mixed with 0 sweeps (FP32 transforms, FP64 low-|k|
columns), then 1, 2, 3 double-float refinement sweeps.
"""
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300 import tradeoff

pytestmark = pytest.mark.gpu


def test_precision_ladder_orders_accuracy():
    d = wl.anelastic_noise(192, 128, 40, seed=43)
    ref = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
    res = tradeoff.run(d, reps=3)
    rows = {r["solve"]: r for r in res["rows"]}
    assert [r["solve"] for r in res["rows"]] == [lab for lab, _, _ in tradeoff.rungs()]

    # the study's reference (the FP64 GPU solve) is the oracle's solution
    from paper_2010_14132_gb300.solver import Plan
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="fp64")
    p64 = plan.solve(torch.from_numpy(d.S).cuda()).cpu().numpy()
    assert O.relative_l2(p64, ref) <= 1e-12
    assert rows["fp64"]["rel_l2_diff"] == 0.0

    fp32 = rows["fp32"]["rel_l2_diff"]
    m0, m1, m2, m3 = (rows[f"mixed, {k} sweep{'s' if k != 1 else ''}"]["rel_l2_diff"] for k in range(4))
    assert 1e-8 < fp32 < 1e-4
    assert m0 < 1e-4
    assert m1 < 1e-2 * m0 and m1 <= 1e-10
    # sweeps 2 and 3 sit at the double-float residual's floor (~1e-12 here): no worse than sweep 1
    assert m2 <= m1 + 1e-12 and m3 <= m1 + 1e-12 and max(m2, m3) <= 1e-11
    for mode in ("mixed, stop rule", "mixed, stop rule, full-spectrum verification",
                 "mixed, stop rule, no verification"):
        assert rows[mode]["rel_l2_diff"] <= rows[mode]["error_estimate"] <= 1e-10, (mode, rows[mode])
    # k sweeps exactly, unless an update comes out exactly zero (then the rule stops early)
    assert rows["mixed, 0 sweeps"]["sweeps"] == 0 and rows["mixed, 1 sweep"]["sweeps"] == 1
    assert 1 <= rows["mixed, 2 sweeps"]["sweeps"] <= 2 and 1 <= rows["mixed, 3 sweeps"]["sweeps"] <= 3
    # the mean per-element difference orders the rungs the same way
    assert rows["mixed, 1 sweep"]["mean_abs_diff"] < rows["mixed, 0 sweeps"]["mean_abs_diff"]
    assert rows["mixed, 0 sweeps"]["mean_abs_diff"] <= rows["fp32"]["mean_abs_diff"] * 1.5
    for r in res["rows"]:
        assert r["ms_per_solve"] > 0


def test_cg_termination_residual_orders_accuracy_and_cost():
    """Table 1's form for the iterative solver: a tighter termination residual costs more
    iterations and lands closer to the converged solution; the direct solve for the level-mean
    density alone (the horizontal variation ignored) is further off than CG to 1e-4."""
    d = wl.anelastic_noise(128, 96, 24, seed=44)
    res = tradeoff.run_cg(d, 0.2, reps=1)
    cg = res["rows"][:-1]
    direct = res["rows"][-1]
    assert [r["tol"] for r in cg] == [1e-2, 1e-4, 1e-6, 1e-8]
    assert res["reference_rel_residual"] <= 1e-12
    for r in cg:
        assert r["rel_residual"] <= r["tol"], r
    its = [r["iterations"] for r in cg]
    diffs = [r["mean_abs_diff"] for r in cg]
    assert its == sorted(its) and its[-1] > its[0], its
    assert all(b < a for a, b in zip(diffs, diffs[1:])), diffs
    assert direct["iterations"] == 0 and direct["mean_abs_diff"] > diffs[1]
