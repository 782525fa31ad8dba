"""Run a few solves of one grid size, for profilers (ncu) and quick timing.

    python -m paper_2010_14132_gb300.profile_case --nx 1024 --ny 1024 --nz 32 --dtype mixed --reps 1

The grid uses the stretched/anelastic setup (dx = dy = 50 m, dz_k = 10*1.03^k m,
rho0 = 1.2 exp(-z/8000)) with a seeded N(0,1) source.  With --adjoint the
adjoint (and rho0 gradient) is run after each solve.  With --cg EPS each call is
instead a conjugate-gradient solve for the density rho0(z) (1 + EPS g(x, y, z)),
preconditioned by the plan's direct solve for the level-mean density (tolerance 1e-10).  Prints the mean time per
call measured with CUDA events.  The measured calls sit inside a CUDA profiler
range, so ``ncu --profile-from-start off`` captures them and not the set-up.
Kernel shapes default to the library's defaults; --tuned takes the autotuner's
choice for this size, and the explicit flags override either.
"""
from __future__ import annotations

import argparse
import sys

import torch

from . import workloads as wl
from .solver import Plan


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--nz", type=int, default=32)
    ap.add_argument("--dtype", default="mixed", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--tuned", action="store_true")
    ap.add_argument("--cg", type=float, default=None, metavar="EPS")
    ap.add_argument("--max-sweeps", dest="max_sweeps", type=int, default=None)
    for name in ("y_kernel", "y_tile", "y_elems", "x_elems", "level_chunk", "x_kernel", "col_tile", "spectral_fused", "residual_pass"):
        ap.add_argument("--" + name.replace("_", "-"), dest=name, type=int, default=None)
    args = ap.parse_args(argv)
    d = wl.anelastic_noise(args.nx, args.ny, args.nz, seed=3)
    opts = {}
    if args.tuned:
        from .autotune import tuned_options
        opts = tuned_options(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, args.dtype)
    for name in ("y_kernel", "y_tile", "y_elems", "x_elems", "level_chunk", "x_kernel", "col_tile", "spectral_fused", "residual_pass"):
        if getattr(args, name) is not None:
            opts[name] = getattr(args, name)
    if args.max_sweeps is not None:
        opts["max_sweeps"] = args.max_sweeps
    rho0, rho3 = d.rho0, None
    if args.cg is not None:
        rho3 = wl.perturbed_density(d.nx, d.ny, d.rho0, args.cg, seed=8)
        rho0 = rho3.mean(axis=(1, 2))
    # plain stream launches (POISSON_OPT_GRAPH = 0): the same kernels as the captured graph, each one
    # launched from the host, so that a profiler sees every launch as its own
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, rho0, dtype=args.dtype, graph=0, **opts)
    S = torch.from_numpy(d.S).cuda().to(plan.field_dtype)
    p = torch.empty_like(S)
    w = torch.randn_like(S) if args.adjoint else None
    rho_t = torch.from_numpy(rho3).cuda() if rho3 is not None else None

    def call():
        if rho_t is not None:
            plan.cg_solve(rho_t, S, out=p, tol=1e-10, max_iter=100)
        else:
            plan.solve(S, out=p)

    call()   # warm-up: kernel loading, workspace
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record()
    for _ in range(args.reps):
        call()
        if args.adjoint:
            plan.adjoint(w, p=p, want_grho=True)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(f"{args.nx}x{args.ny}x{args.nz} {args.dtype} {opts}: "
          f"{e0.elapsed_time(e1) / max(1, args.reps):.3f} ms per call")
    return 0


if __name__ == "__main__":
    sys.exit(main())
