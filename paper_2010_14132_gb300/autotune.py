"""Autotuner for the transform kernels' shape choices.

For one grid (nx, ny, nz, dtype) it times candidate settings of the y-pass
(TMA-staged or plain kernel, kx tile width, elements per thread) and of the
x-pass (persistent bulk-copy-staged kernel, or one CTA per row group with 8 or
16 elements per thread), using the library's own per-phase CUDA events
(POISSON_OPT_PROFILE) on the launching stream, and keeps the fastest setting of
each pass.  Results are cached in a JSON file keyed by GPU name, sizes and
dtype, so a plan is tuned once and the choice reused every solve (the
plan-once idea of Section 2.1).

    from paper_2010_14132_gb300.autotune import tuned_options
    opts = tuned_options(nx, ny, nz, dx, dy, dz, rho0, "mixed")
    plan = Plan(nx, ny, nz, dx, dy, dz, rho0, dtype="mixed", **opts)
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import _native as N
from .solver import Plan

CACHE = os.environ.get("POISSON_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "poisson_gb300_autotune.json"))

Y_CANDIDATES = [dict(y_kernel=k, y_tile=t, y_elems=e) for k in (0, 4, 3, 1, 2) for t in (2, 4, 8, 16) for e in (8, 16)]
X_CANDIDATES = [dict(x_kernel=k, x_elems=e) for k in (0, 1) for e in (8, 16)]
CHUNK_CANDIDATES = [dict(level_chunk=c) for c in (0, 1, 2, 4, 8, 16, 4096)]
COL_CANDIDATES = [dict(col_tile=c) for c in (0, 1, 4, 3, 16, 32)]
OPT_IDS = {"y_kernel": N.POISSON_OPT_Y_KERNEL, "y_tile": N.POISSON_OPT_Y_TILE, "y_elems": N.POISSON_OPT_Y_ELEMS,
           "x_elems": N.POISSON_OPT_X_ELEMS, "level_chunk": N.POISSON_OPT_LEVEL_CHUNK,
           "x_kernel": N.POISSON_OPT_X_KERNEL, "col_tile": N.POISSON_OPT_COL_TILE,
           "spectral_fused": N.POISSON_OPT_SPECTRAL_FUSED, "residual_pass": N.POISSON_OPT_RESIDUAL_PASS}


def _key(nx, ny, nz, dtype):
    name = torch.cuda.get_device_name()
    return f"{name}|{nx}x{ny}x{nz}|{dtype}"


def _load_cache():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(c):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
    except OSError:
        pass


def _time_phases(plan: Plan, S: torch.Tensor, p: torch.Tensor, reps: int):
    for _ in range(2):
        plan.solve(S, out=p)
    torch.cuda.synchronize()
    N.poisson_plan_set_option(plan._h, N.POISSON_OPT_PROFILE, 1)
    N.poisson_plan_profile_read(plan._h)
    for _ in range(reps):
        plan.solve(S, out=p)
    torch.cuda.synchronize()
    ph = N.poisson_plan_profile_read(plan._h)
    N.poisson_plan_set_option(plan._h, N.POISSON_OPT_PROFILE, 0)
    return {k: v[0] / reps for k, v in ph.items()}


def autotune(nx, ny, nz, dx, dy, dz, rho0, dtype="mixed", reps=3, verbose=False):
    """Measure the candidates (y-pass, x-pass, level chunk, column tile); return (best, table)."""
    plan = Plan(nx, ny, nz, dx, dy, dz, rho0, dtype=dtype)
    rng = np.random.default_rng(0)
    S = torch.from_numpy(rng.standard_normal((nz, ny, nx))).cuda().to(plan.field_dtype)
    S -= S.mean()
    p = torch.empty_like(S)
    table = []
    best_y, best_yt = {}, float("inf")
    for cand in Y_CANDIDATES:
        try:
            for k, v in cand.items():
                plan.set_option(OPT_IDS[k], v)
        except N.PoissonError:
            continue
        t = _time_phases(plan, S, p, reps)
        ty = t["yfwd"] + t["yinv"]
        table.append(("y", cand, ty))
        if verbose:
            print("y", cand, f"{ty:.3f} ms")
        if ty < best_yt:
            best_y, best_yt = dict(cand), ty
    for k, v in best_y.items():
        plan.set_option(OPT_IDS[k], v)
    best_x, best_xt = {}, float("inf")
    for cand in X_CANDIDATES:
        try:
            for k, v in cand.items():
                plan.set_option(OPT_IDS[k], v)
        except N.PoissonError:
            continue
        t = _time_phases(plan, S, p, reps)
        tx = t["xfwd"] + t["xinv"]
        table.append(("x", cand, tx))
        if verbose:
            print("x", cand, f"{tx:.3f} ms")
        if tx < best_xt:
            best_x, best_xt = dict(cand), tx
    for k, v in best_x.items():
        plan.set_option(OPT_IDS[k], v)
    # levels per transform chunk: timed on the whole solve (it trades L2 reuse against launch count)
    best_c, best_ct = {}, float("inf")
    for cand in CHUNK_CANDIDATES:
        for k, v in cand.items():
            plan.set_option(OPT_IDS[k], v)
        t = _time_phases(plan, S, p, reps)
        tt = sum(t.values())
        table.append(("chunk", cand, tt))
        if verbose:
            print("chunk", cand, f"{tt:.3f} ms")
        if tt < best_ct:
            best_c, best_ct = dict(cand), tt
    for k, v in best_c.items():
        plan.set_option(OPT_IDS[k], v)
    # columns per CTA of the column solve
    best_t, best_tt = {}, float("inf")
    for cand in COL_CANDIDATES:
        try:
            for k, v in cand.items():
                plan.set_option(OPT_IDS[k], v)
        except N.PoissonError:
            continue
        t = _time_phases(plan, S, p, reps)
        tt = t["columns"]
        table.append(("columns", cand, tt))
        if verbose:
            print("columns", cand, f"{tt:.3f} ms")
        if tt < best_tt:
            best_t, best_tt = dict(cand), tt
    plan.close()
    return {**best_y, **best_x, **best_c, **best_t}, table


def tuned_options(nx, ny, nz, dx, dy, dz, rho0, dtype="mixed", retune=False):
    """Cached autotune result for this GPU, size and dtype (tunes on first use)."""
    cache = _load_cache()
    key = _key(nx, ny, nz, dtype)
    if key in cache and not retune:
        return dict(cache[key])
    best, _ = autotune(nx, ny, nz, dx, dy, dz, rho0, dtype)
    cache[key] = best
    _save_cache(cache)
    return best
