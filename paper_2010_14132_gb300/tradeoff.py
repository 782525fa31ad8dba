"""Accuracy against time per solve: a synthetic analogue of the paper's Table 1.

Section 3 (Table 1) sets the iterative solver's termination residual against the
mean per-element difference from the direct FFT solution and the time per solve.
The direct solve has no termination residual, but it has a precision ladder:

    fp32                 FP32 transforms and FP32 columns on float fields
    mixed, k sweeps      FP32 transforms, FP64 low-|k| columns, then k double-float
                         residual refinement sweeps (k = 0..3), no early stop, no
                         verification
    mixed, stop rule     the default: sweeps until the error bound is below the
                         plan's tolerance, the next correction's low-wavenumber part
                         verifying an iterate before that correction is applied; also
                         with the full-spectrum verification and with none
    fp64                 FP64 throughout (the reference of the comparison)

For each rung this reports the time per solve (CUDA events on the solving
stream around back-to-back solves, inputs resident; with --tuned the autotuner's
kernel shapes), the mean |p - p_fp64| per
element (the paper's mean-difference column), the relative L2 difference, and the
sweeps and error bound the library reported.  The FP64 GPU solution is the
reference here; it matches the FP64 CPU oracle to 1e-12 relative L2 in the
parity tests.

    python -m paper_2010_14132_gb300.tradeoff [--nx 1024 --ny 1024 --nz 128 --reps 20] [--tuned]

With --cg EPS the study takes Table 1's own form for the library's iterative
solver: conjugate gradients for the density rho0(z) (1 + EPS g(x, y, z)),
preconditioned by the direct solve, run to termination residuals 1e-2 ... 1e-8.
Each row gives the iterations, the time per solve and the mean difference from a
1e-12 solution. A last row gives the direct solve for the level-mean density
alone: the error of ignoring the horizontal variation.

    python -m paper_2010_14132_gb300.tradeoff --cg 0.1
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import workloads as wl
from .solver import Plan


def _time_solve(plan, S, p, reps):
    """Mean device time per solve over `reps` back-to-back solves (median of three such runs)."""
    stream = torch.cuda.current_stream()
    for _ in range(3):
        plan.solve(S, out=p)
    times = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.solve(S, out=p)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / reps)
    return float(np.median(times))


def rungs():
    """(label, dtype, plan options) of the precision ladder, cheapest first."""
    out = [("fp32", "fp32", {})]
    for k in range(4):
        # a tolerance no bound reaches: exactly k sweeps
        out.append((f"mixed, {k} sweep{'s' if k != 1 else ''}", "mixed",
                    {"max_sweeps": k, "tolerance": 1e-300, "verify": 0}))
    out.append(("mixed, stop rule", "mixed", {}))
    out.append(("mixed, stop rule, full-spectrum verification", "mixed", {"verify": 2}))
    out.append(("mixed, stop rule, no verification", "mixed", {"verify": 0}))
    out.append(("fp64", "fp64", {}))
    return out


def run(domain, reps=20, device="cuda", tuned=False):
    d = domain
    S64 = torch.from_numpy(d.S).to(device)
    ref_plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="fp64", device=device)
    p64 = ref_plan.solve(S64)
    torch.cuda.synchronize()
    rows = []
    for label, dtype, opts in rungs():
        if tuned and dtype != "fp64":
            from .autotune import tuned_options
            opts = dict(tuned_options(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype), **opts)
        plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype, device=device, **opts)
        S = S64 if dtype != "fp32" else S64.to(torch.float32)
        p = torch.empty_like(S)
        ms = _time_solve(plan, S, p, reps if dtype != "fp64" else max(3, reps // 4))
        _, info = plan.solve(S, out=p, info=True)
        torch.cuda.synchronize()
        diff = p.to(torch.float64) - p64
        rows.append({
            "solve": label,
            "ms_per_solve": ms,
            "mpoints_s": d.npoints / (ms * 1e-3) / 1e6,
            "mean_abs_diff": float(diff.abs().mean()),
            "rel_l2_diff": float(torch.linalg.vector_norm(diff) / torch.linalg.vector_norm(p64)),
            "sweeps": info["sweeps"] if dtype == "mixed" else None,
            "error_estimate": info["error_estimate"] if dtype == "mixed" else None,
        })
        plan.close()
    ref_plan.close()
    return {"workload": d.name, "nx": d.nx, "ny": d.ny, "nz": d.nz,
            "p_mean_abs": float(p64.abs().mean()), "rows": rows}


def run_cg(domain, eps, tols=(1e-2, 1e-4, 1e-6, 1e-8), reps=3, device="cuda"):
    """Termination residual against mean difference and time (Table 1's columns) for the CG."""
    import time
    d = domain
    rho3 = wl.perturbed_density(d.nx, d.ny, d.rho0, eps, seed=8)
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, rho3.mean(axis=(1, 2)), dtype="mixed", device=device,
                max_sweeps=0)
    rho_t = torch.from_numpy(rho3).to(device)
    del rho3
    S = torch.from_numpy(d.S).to(device)
    ref, rinfo = plan.cg_solve(rho_t, S, tol=1e-12, max_iter=200)
    torch.cuda.synchronize()
    rows = []
    p = torch.empty_like(S)
    for tol in tols:
        plan.cg_solve(rho_t, S, out=p, tol=tol, max_iter=200)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            _, info = plan.cg_solve(rho_t, S, out=p, tol=tol, max_iter=200)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / reps
        diff = p - ref
        rows.append({"solve": f"CG to {tol:.0e}", "tol": tol, "iterations": info["iterations"],
                     "rel_residual": info["rel_residual"], "ms_per_solve": ms,
                     "mean_abs_diff": float(diff.abs().mean()),
                     "rel_l2_diff": float(torch.linalg.vector_norm(diff) / torch.linalg.vector_norm(ref))})
    # the direct solve alone (level-mean density): no iteration, the horizontal variation ignored
    plan.solve(S, out=p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.solve(S, out=p)
    e1.record()
    torch.cuda.synchronize()
    diff = p - ref
    rows.append({"solve": "direct solve, level-mean density", "tol": None, "iterations": 0, "rel_residual": None,
                 "ms_per_solve": e0.elapsed_time(e1) / reps, "mean_abs_diff": float(diff.abs().mean()),
                 "rel_l2_diff": float(torch.linalg.vector_norm(diff) / torch.linalg.vector_norm(ref))})
    plan.close()
    return {"workload": d.name, "nx": d.nx, "ny": d.ny, "nz": d.nz, "eps": eps,
            "reference_iterations": rinfo["iterations"], "reference_rel_residual": rinfo["rel_residual"],
            "p_mean_abs": float(ref.abs().mean()), "rows": rows}


def markdown_cg(res):
    lines = [f"Workload {res['workload']} ({res['nx']} x {res['ny']} x {res['nz']}), density rho0(z) "
             f"(1 + {res['eps']} g); reference: CG to 1e-12 ({res['reference_iterations']} iterations); "
             f"mean |p| = {res['p_mean_abs']:.3e}.", "",
             "| solve | iterations | relative residual | mean difference | rel. L2 difference | time per solve (ms) |",
             "|---|---|---|---|---|---|"]
    for r in res["rows"]:
        rr = "-" if r["rel_residual"] is None else f"{r['rel_residual']:.1e}"
        lines.append(f"| {r['solve']} | {r['iterations']} | {rr} | {r['mean_abs_diff']:.2e} | "
                     f"{r['rel_l2_diff']:.2e} | {r['ms_per_solve']:.2f} |")
    return "\n".join(lines)


def markdown(res):
    lines = [f"Workload {res['workload']} ({res['nx']} x {res['ny']} x {res['nz']}); "
             f"mean |p| of the FP64 solution = {res['p_mean_abs']:.3e}.", "",
             "| solve | time per solve (ms) | Mpoints/s | mean difference | rel. L2 difference | sweeps | error bound |",
             "|---|---|---|---|---|---|---|"]
    for r in res["rows"]:
        sw = "-" if r["sweeps"] is None else str(r["sweeps"])
        est = "-" if r["error_estimate"] is None or r["error_estimate"] < 0 else f"{r['error_estimate']:.1e}"
        diff = "reference" if r["solve"] == "fp64" else f"{r['mean_abs_diff']:.2e}"
        rel = "reference" if r["solve"] == "fp64" else f"{r['rel_l2_diff']:.2e}"
        lines.append(f"| {r['solve']} | {r['ms_per_solve']:.3f} | {r['mpoints_s']:.0f} | {diff} | {rel} | {sw} | {est} |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--nz", type=int, default=128)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--json", action="store_true", help="print JSON instead of a markdown table")
    ap.add_argument("--tuned", action="store_true", help="the autotuner's kernel shapes (as the bench)")
    ap.add_argument("--cg", type=float, default=None, metavar="EPS",
                    help="the conjugate-gradient study for the density rho0(z) (1 + EPS g)")
    a = ap.parse_args(argv)
    d = wl.anelastic_noise(a.nx, a.ny, a.nz, seed=a.seed)
    if a.cg is not None:
        res = run_cg(d, a.cg, reps=max(1, min(a.reps, 5)))
        print(json.dumps(res) if a.json else markdown_cg(res))
        return
    res = run(d, reps=a.reps, tuned=a.tuned)
    print(json.dumps(res) if a.json else markdown(res))


if __name__ == "__main__":
    main()
