"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative L2 over all cells, both sides pinned to zero mean):
FP64 path <= 1e-12, FP32 path <= 1e-5, mixed path (after refinement) <= 1e-10.
Inputs are the seeded synthetic workloads; sizes span several tiles, ragged
tails, radix-2/3 mixes and the degenerate cases of the method (the singular
(0,0) column, constant sources, pure vertical and pure horizontal modes).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_14132_gb300 import workloads as wl
from paper_2010_14132_gb300.solver import Plan, Batch, poisson_solve

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "mixed": 1e-10}


def gpu_solve(d, dtype, S=None, **opts):
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype=dtype, **opts)
    S = d.S if S is None else S
    St = torch.from_numpy(np.ascontiguousarray(S)).to("cuda", plan.field_dtype)
    p, info = plan.solve(St, info=True)
    torch.cuda.synchronize()
    return p.double().cpu().numpy(), info, plan


def assert_estimate_bounds(info, err):
    """A converged mixed solve's error bound is at least its error against the oracle."""
    if info.get("converged") and info.get("sweeps", 0) >= 1:
        assert info["error_estimate"] >= err, (info, err)


def check(d, dtype, tol=None, S=None, **opts):
    p, info, _ = gpu_solve(d, dtype, S=S, **opts)
    ref = O.solve(d.S if S is None else S, d.dx, d.dy, d.dz, d.rho0)
    err = O.relative_l2(p, ref)
    assert np.isfinite(p).all()
    assert err <= (tol if tol is not None else TOL[dtype]), (dtype, d.name, err, info)
    if dtype == "mixed":
        assert_estimate_bounds(info, err)
    return err, info


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def test_uniform_cube_32_fp64():
    err, info = check(wl.uniform_cube(32, seed=1), "fp64")
    assert abs(info["removed_weighted_mean"]) < 1e-15


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_anelastic_blobs_256x256x64(dtype):
    check(wl.anelastic_blobs(256, 256, 64, seed=2), dtype)


@pytest.fixture(scope="module")
def full_size():
    """The bench workload and the oracle's solution of it (computed once for the module)."""
    d = wl.anelastic_noise(1024, 1024, 128, seed=3)
    return d, O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)


def test_anelastic_noise_1024x1024x128_mixed_full_size(full_size):
    d, ref = full_size
    p, info, _ = gpu_solve(d, "mixed")
    err = O.relative_l2(p, ref)
    assert err <= TOL["mixed"], (err, info)
    assert info["converged"] and 1 <= info["sweeps"] <= 3, info
    # the stopping rule's bound meets the tolerance and bounds the measured error
    assert info["error_estimate"] <= 1e-10
    assert_estimate_bounds(info, err)
    # the residual of each iterate a sweep started from, relative to ||S||, falls sweep by sweep
    res = info["rel_residual"][:info["sweeps"]]
    assert all(r > 0 for r in res) and all(b < a for a, b in zip(res, res[1:])), info


def test_full_size_in_the_bench_launch_configuration(full_size):
    """The kernel shapes the bench times (the autotuner's choice on this GPU) at the full size."""
    from paper_2010_14132_gb300.autotune import tuned_options
    d, ref = full_size
    opts = tuned_options(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, "mixed")
    p, info, _ = gpu_solve(d, "mixed", **opts)
    err = O.relative_l2(p, ref)
    assert err <= TOL["mixed"], (err, opts, info)
    assert_estimate_bounds(info, err)


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
def test_anelastic_noise_small(dtype):
    check(wl.anelastic_noise(128, 96, 32, seed=31), dtype)


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
def test_gradient_workload_forward_512x512x64(dtype):
    d = wl.gradient_problem(512, 512, 64)
    check(d, dtype)


# ---------------------------------------------------------------------------
# sizes: radix 2/3 mixes, ragged tiles, minimum sizes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nx,ny,nz", [(4, 4, 2), (4, 6, 3), (6, 4, 5), (12, 48, 7), (96, 384, 9), (384, 96, 4),
                                      (48, 12, 33), (8, 16, 130), (18, 27, 6), (36, 8, 3), (64, 64, 512),
                                      (2048, 8, 4), (8, 4096, 2), (128, 8, 3), (256, 12, 5), (512, 6, 7),
                                      (1024, 12, 3), (4096, 4, 3)])
@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
@pytest.mark.parametrize("y_kernel", [0, 1, 2, 3, 4])
def test_sizes(nx, ny, nz, dtype, y_kernel):
    """Radix 2/3 mixes, ragged tiles, the smallest and largest line lengths.

    The horizontal spacing keeps every column well conditioned (smallest
    horizontal eigenvalue ~ (2 pi / 8)^2 against O(1) vertical coupling): with
    nz of 2-4 and kappa ~ 1e6 the FP64 oracle's textbook recurrence itself
    loses ~eps*kappa, which is not what these cases are about (conditioning is
    covered by the stretched workloads)."""
    h = 8.0 / max(nx, ny)
    d = wl.random_stretched(nx, ny, nz, seed=nx * 7 + ny * 3 + nz, dx=h, dy=1.3 * h)
    check(d, dtype, y_kernel=y_kernel)


@pytest.mark.parametrize("nx,ny,nz", [(384, 384, 48), (64, 128, 96), (512, 256, 32)])
def test_sizes_mixed(nx, ny, nz):
    d = wl.uneven_batch(1)[0]
    d = wl.Domain(nx, ny, nz, 50.0, 50.0, wl.stretched_levels(nz, 12.0, 1.02),
                  wl.exponential_density(wl.stretched_levels(nz, 12.0, 1.02), 1.1, 8500.0),
                  wl.normal_source((nz, ny, nx), seed=nx + ny + nz))
    check(d, "mixed")


@pytest.mark.parametrize("opts", [dict(x_elems=16), dict(y_elems=8), dict(x_elems=8, y_elems=8, y_tile=4),
                                  dict(y_kernel=1, y_tile=16, y_elems=8), dict(y_tile=2), dict(y_tile=16),
                                  dict(level_chunk=1), dict(level_chunk=5), dict(level_chunk=7, y_kernel=1),
                                  dict(level_chunk=4096), dict(x_kernel=1), dict(x_kernel=1, x_elems=16),
                                  dict(x_kernel=1, level_chunk=3), dict(y_kernel=2), dict(y_kernel=2, y_elems=8),
                                  dict(y_elems=8, y_tile=8), dict(y_elems=8, y_tile=2), dict(y_tile=8),
                                  dict(col_tile=16), dict(col_tile=32), dict(col_tile=64), dict(col_tile=128),
                                  dict(col_tile=1), dict(col_tile=3), dict(col_tile=4), dict(y_kernel=3),
                                  dict(y_kernel=3, y_tile=4), dict(y_kernel=3, y_elems=8, y_tile=8),
                                  dict(y_kernel=4, y_tile=8), dict(y_kernel=4, y_tile=4, y_elems=8)])
@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
def test_kernel_shape_options(opts, dtype):
    """Every autotuner candidate gives the same answer (tile shapes are not numerics)."""
    d = wl.anelastic_noise(256, 128, 24, seed=17)
    check(d, dtype, **opts)


# ---------------------------------------------------------------------------
# closed forms and degenerate cases (no oracle on the expected side)
# ---------------------------------------------------------------------------

def _cos_mode(nx, ny, nz, ax, by, cz):
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    return (np.cos(2 * np.pi * ax * i / nx + 0.3) * np.cos(2 * np.pi * by * j / ny - 0.7)
            * np.cos(np.pi * cz * (k + 0.5) / nz))


@pytest.mark.parametrize("mode", [(1, 0, 0), (0, 0, 1), (0, 0, 31), (16, 16, 0), (5, 3, 7), (0, 16, 2)])
@pytest.mark.parametrize("dtype", ["fp64", "mixed"])
def test_eigenfunctions_uniform_cube(mode, dtype):
    n = 32
    p_exact = _cos_mode(n, n, n, *mode)
    a, b, c = mode
    lam = -4 * np.sin(np.pi * a / n) ** 2 - 4 * np.sin(np.pi * b / n) ** 2 - 4 * np.sin(np.pi * c / (2 * n)) ** 2
    d = wl.Domain(n, n, n, 1.0, 1.0, np.ones(n), np.ones(n), lam * p_exact)
    p, info, _ = gpu_solve(d, dtype)
    # the FP64 bar (the float-rounded source itself moves the exact discrete solution
    # of the highest vertical mode by ~8e-13 from the closed form)
    assert O.relative_l2(p, p_exact) < (1e-12 if dtype == "fp64" else 1e-10)


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
def test_constant_source_gives_zero(dtype):
    d = wl.random_stretched(16, 12, 8, seed=5)
    S = np.full(d.S.shape, 3.25)
    p, info, _ = gpu_solve(d, dtype, S=S)
    assert np.abs(p).max() < {"fp64": 1e-12, "fp32": 1e-4, "mixed": 1e-9}[dtype]
    assert abs(info["removed_weighted_mean"] - 3.25) < 1e-6


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "mixed"])
def test_zero_mean_and_residual(dtype):
    d = wl.anelastic_blobs(64, 48, 24, seed=12)
    p, info, _ = gpu_solve(d, dtype)
    assert abs(p.mean()) <= 1e-12 * np.abs(p).max() * (1 if dtype != "fp32" else 1e6)
    r = O.residual(d.S, p, d.dx, d.dy, d.dz, d.rho0)
    bound = {"fp64": 1e-10, "fp32": 1e-3, "mixed": 1e-8}[dtype]
    assert np.linalg.norm(r) / np.linalg.norm(d.S) < bound


def test_periodic_shift_equivariance_fp64():
    d = wl.anelastic_blobs(64, 32, 16, seed=13)
    p1, _, plan = gpu_solve(d, "fp64")
    S2 = np.roll(d.S, (5, 11), axis=(1, 2))
    p2 = plan.solve(torch.from_numpy(S2).cuda()).cpu().numpy()
    assert O.relative_l2(p2, np.roll(p1, (5, 11), axis=(1, 2))) < 1e-13


def test_repeated_solves_are_bitwise_identical():
    d = wl.anelastic_noise(128, 128, 32, seed=14)
    plan = Plan(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype="mixed")
    St = torch.from_numpy(d.S).cuda()
    a = plan.solve(St).clone()
    b = plan.solve(St).clone()
    assert torch.equal(a, b)


# ---------------------------------------------------------------------------
# mixed-path options
# ---------------------------------------------------------------------------

def test_mixed_without_refinement_is_fp32_accurate():
    d = wl.anelastic_noise(256, 256, 64, seed=15)
    err, info = check(d, "mixed", tol=1e-5, max_sweeps=0)
    assert info["sweeps"] == 0


def test_mixed_lowk_radius_zero_still_converges():
    d = wl.anelastic_noise(256, 256, 64, seed=16)
    check(d, "mixed", lowk_radius2=0)


@pytest.mark.parametrize("x_kernel", [0, 1])
def test_mixed_three_sweeps(x_kernel):
    """A tolerance no estimate can meet runs all three sweeps: the later sweeps rebuild the
    correction from the stored double iterate, and every sweep keeps (or improves) accuracy."""
    d = wl.anelastic_noise(128, 96, 32, seed=18)
    p, info, _ = gpu_solve(d, "mixed", tolerance=1e-30, x_kernel=x_kernel)
    assert info["sweeps"] == 3 and not info["converged"], info
    ref = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
    assert O.relative_l2(p, ref) <= 1e-11
    # relative updates shrink sweep after sweep
    ru = info["rel_update"]
    assert ru[2] < ru[1] and ru[3] < ru[2] * 10, info


# ---------------------------------------------------------------------------
# batched solve (uneven sizes, one graph launch)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["fp32", "mixed"])
def test_batch_uneven_domains(dtype):
    doms = wl.uneven_batch(6, seed=70, nxy_choices=(64, 96, 128), nz_choices=(16, 24, 32))
    b = Batch(doms, dtype=dtype)
    fd = torch.float32 if dtype == "fp32" else torch.float64
    S = [torch.from_numpy(d.S).to("cuda", fd) for d in doms]
    outs, infos = b.solve(S, info=True)
    outs2 = b.solve(S)   # graph replay
    torch.cuda.synchronize()
    for d, p, p2 in zip(doms, outs, outs2):
        ref = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
        assert O.relative_l2(p.double().cpu().numpy(), ref) <= TOL[dtype]
        assert torch.equal(p, p2)


@pytest.mark.parametrize("dtype", ["fp32", "mixed"])
def test_batch_autotuned_shapes(dtype, tmp_path, monkeypatch):
    """Autotuned kernel shapes per domain give the same answers (concurrent graph branches)."""
    monkeypatch.setenv("POISSON_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    import importlib
    from paper_2010_14132_gb300 import autotune
    importlib.reload(autotune)
    doms = wl.uneven_batch(5, seed=71, nxy_choices=(64, 128), nz_choices=(16, 24))
    b = Batch(doms, dtype=dtype, tune=True, persistent=False)
    fd = torch.float32 if dtype == "fp32" else torch.float64
    S = [torch.from_numpy(d.S).to("cuda", fd) for d in doms]
    outs = b.solve(S)
    torch.cuda.synchronize()
    for d, p in zip(doms, outs):
        ref = O.solve(d.S, d.dx, d.dy, d.dz, d.rho0)
        assert O.relative_l2(p.double().cpu().numpy(), ref) <= TOL[dtype]


@pytest.fixture(scope="module")
def batch_64():
    """The 64-domain uneven batch and the oracle's solution of every domain (computed once)."""
    doms = wl.uneven_batch(64)
    refs = [O.solve(d.S, d.dx, d.dy, d.dz, d.rho0) for d in doms]
    return doms, refs


@pytest.mark.parametrize("dtype,persistent", [("fp32", False), ("mixed", True), ("mixed", False)])
def test_batch_64_uneven_domains_all_against_oracle(dtype, persistent, batch_64):
    """The 64-domain uneven batch (nx = ny in {64..512}, nz in {32..96}) in one graph launch (mixed: the
    persistent kernel over every domain's work items, or the graph of per-domain launches), every
    domain against the oracle at the dtype's tolerance."""
    doms, refs = batch_64
    b = Batch(doms, dtype=dtype, persistent=persistent)
    fd = torch.float32 if dtype == "fp32" else torch.float64
    S = [torch.from_numpy(d.S).to("cuda", fd) for d in doms]
    outs, infos = b.solve(S, info=True)
    torch.cuda.synchronize()
    worst = 0.0
    for d, p, ref, info in zip(doms, outs, refs, infos):
        err = O.relative_l2(p.double().cpu().numpy(), ref)
        worst = max(worst, err)
        assert err <= TOL[dtype], (d.name, err, info)
        if dtype == "mixed":
            assert info["converged"], (d.name, info)
            assert_estimate_bounds(info, err)
    assert worst > 0.0
