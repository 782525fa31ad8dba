"""PyTorch-facing API of the GB300 direct FFT pressure solver.

PyTorch provides device memory, streams and autograd plumbing only; every step
of the solve runs in the library's CUDA kernels through the C ABI
(``_native``).  There is no CPU path: creating a plan needs the built library
and solving needs CUDA tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _native as N

DTYPES = {"fp64": N.POISSON_FP64, "fp32": N.POISSON_FP32, "mixed": N.POISSON_MIXED}
LAYOUTS = {"zyx": N.POISSON_LAYOUT_Z_Y_X, "xyz": N.POISSON_LAYOUT_X_Y_Z}
BCS = {"neumann": N.POISSON_BC_PERIODIC_XY_NEUMANN_Z,
       "dirichlet_top": N.POISSON_BC_PERIODIC_XY_NEUMANN_BOTTOM_DIRICHLET_TOP}
FIELD_DTYPE = {"fp64": torch.float64, "fp32": torch.float32, "mixed": torch.float64}


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _require_cuda(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous tensor of shape {tuple(shape)}")


class Plan:
    """A planned solve for one grid (Section 2.1: plan once, reuse every timestep).

    nx, ny: periodic horizontal sizes (2^a 3^b, nx even); nz levels; dx, dy
    spacings; dz, rho0: per-level thickness and reference density (length nz).
    dtype: "fp64", "fp32" or "mixed" (double fields, float transforms, double
    low-|k| columns and double-float refinement).  bc: "neumann" (zero flux
    through the bottom and top faces; p is projected and pinned to zero mean) or
    "dirichlet_top" (zero flux at the bottom, p = 0 on the top face).  layout:
    "zyx" (fields of shape (nz, ny, nx), x fastest) or "xyz" (shape (nx, ny, nz),
    z fastest, MONC's order; converted inside the library's workspace).
    """

    def __init__(self, nx, ny, nz, dx, dy, dz, rho0, dtype="fp64", device=None, bc="neumann", layout="zyx",
                 lowk_radius2=None, max_sweeps=None, tolerance=None, y_tile=None, y_kernel=None,
                 x_elems=None, y_elems=None, level_chunk=None, x_kernel=None, col_tile=None,
                 spectral_fused=None, residual_pass=None, verify=None, graph=None):
        if dtype not in DTYPES:
            raise ValueError(f"dtype must be one of {sorted(DTYPES)}")
        if bc not in BCS:
            raise ValueError(f"bc must be one of {sorted(BCS)}")
        if layout not in LAYOUTS:
            raise ValueError(f"layout must be one of {sorted(LAYOUTS)}")
        self.bc = bc
        self.layout = layout
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dy = float(dx), float(dy)
        self.dz = np.asarray(dz, dtype=np.float64).copy()
        self.rho0 = np.asarray(rho0, dtype=np.float64).copy()
        if self.dz.shape != (self.nz,) or self.rho0.shape != (self.nz,):
            raise ValueError("dz and rho0 must have nz entries")
        self.dtype = dtype
        self.field_dtype = FIELD_DTYPE[dtype]
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self._h = N.poisson_plan_create(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.rho0,
                                            BCS[bc], DTYPES[dtype])
        if lowk_radius2 is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_LOWK_RADIUS2, lowk_radius2)
        if max_sweeps is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_MAX_SWEEPS, max_sweeps)
        if tolerance is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_TOLERANCE, tolerance)
        if y_tile is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_Y_TILE, y_tile)
        if y_kernel is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_Y_KERNEL, y_kernel)
        if x_elems is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_X_ELEMS, x_elems)
        if y_elems is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_Y_ELEMS, y_elems)
        if level_chunk is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_LEVEL_CHUNK, level_chunk)
        if x_kernel is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_X_KERNEL, x_kernel)
        if col_tile is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_COL_TILE, col_tile)
        if spectral_fused is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_SPECTRAL_FUSED, spectral_fused)
        if residual_pass is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_RESIDUAL_PASS, residual_pass)
        if verify is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_VERIFY, verify)
        if graph is not None:
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_GRAPH, graph)
        if layout != "zyx":
            N.poisson_plan_set_option(self._h, N.POISSON_OPT_LAYOUT, LAYOUTS[layout])
        self._ws = None

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            N.poisson_plan_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):  # pragma: no cover - interpreter shutdown ordering
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.layout == "zyx" else (self.nx, self.ny, self.nz)

    @property
    def npoints(self):
        return self.nx * self.ny * self.nz

    def workspace_bytes(self) -> int:
        return N.poisson_plan_workspace_bytes(self._h)

    def workspace(self) -> torch.Tensor:
        nb = self.workspace_bytes()
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        return self._ws

    def _ws_ptr(self) -> int:
        ws = self.workspace()
        ptr = ws.data_ptr()
        return ptr + ((-ptr) % 256)

    def set_option(self, option: int, value: float):
        N.poisson_plan_set_option(self._h, option, value)
        self._ws = None

    def set_rho0(self, rho0: torch.Tensor, stream=None):
        """Replace rho0 from a device float64 tensor (asynchronous on the stream)."""
        _require_cuda(rho0, torch.float64, (self.nz,), "rho0")
        N.poisson_plan_set_rho0(self._h, rho0.data_ptr(), _stream_handle(stream))
        self.rho0 = None  # now lives on the device only

    # -- calls ---------------------------------------------------------------
    def solve(self, S: torch.Tensor, out: torch.Tensor | None = None, info: bool = False, stream=None):
        """p with L p = S - mu_W and zero mean (L p = S with p = 0 on the top face).

        Returns p, or (p, info dict) if info."""
        _require_cuda(S, self.field_dtype, self.shape, "S")
        p = out if out is not None else torch.empty_like(S)
        _require_cuda(p, self.field_dtype, self.shape, "out")
        r = N.poisson_solve(self._h, S.data_ptr(), p.data_ptr(), self._ws_ptr(), _stream_handle(stream),
                            want_info=info)
        if info:
            st, d = r
            d["status"] = st
            return p, d
        return p

    def adjoint(self, gp: torch.Tensor, p: torch.Tensor | None = None, want_grho: bool = False,
                out: torch.Tensor | None = None, stream=None):
        """(G^T gp, d/drho0) for the solve map G; d/drho0 needs the forward p."""
        _require_cuda(gp, self.field_dtype, self.shape, "gp")
        gS = out if out is not None else torch.empty_like(gp)
        grho = None
        p_ptr = None
        if want_grho:
            if p is None:
                raise ValueError("the rho0 gradient needs the forward solution p")
            _require_cuda(p, self.field_dtype, self.shape, "p")
            grho = torch.empty(self.nz, dtype=torch.float64, device=gp.device)
            p_ptr = p.data_ptr()
        N.poisson_solve_adjoint(self._h, gp.data_ptr(), p_ptr, gS.data_ptr(),
                                grho.data_ptr() if grho is not None else None, self._ws_ptr(),
                                _stream_handle(stream))
        return gS, grho


    # -- variable density (preconditioned conjugate gradients) ------------------
    def cg_solve(self, rho3: torch.Tensor, S: torch.Tensor, out: torch.Tensor | None = None, tol: float = 1e-10,
                 max_iter: int = 50, stream=None):
        """p with A(rho3) p = S - mu_W for a density varying in x, y and z.

        Conjugate gradients in FP64, preconditioned by this plan's direct solve for
        its own rho0 profile (create the plan with the horizontal mean of rho3).
        Needs a "fp64" or "mixed" plan with the default layout.  Returns (p, info).
        """
        if self.layout != "zyx" or self.dtype == "fp32":
            raise ValueError("cg_solve needs a fp64 or mixed plan with the default layout")
        shape = (self.nz, self.ny, self.nx)
        _require_cuda(rho3, torch.float64, shape, "rho3")
        _require_cuda(S, torch.float64, shape, "S")
        p = out if out is not None else torch.empty_like(S)
        _require_cuda(p, torch.float64, shape, "out")
        nb = N.poisson_cg_workspace_bytes(self._h)
        if getattr(self, "_cg_ws", None) is None or self._cg_ws.numel() < nb + 256:
            self._cg_ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        ptr = self._cg_ws.data_ptr()
        ptr += (-ptr) % 256
        _, info = N.poisson_cg_solve(self._h, rho3.data_ptr(), S.data_ptr(), p.data_ptr(), tol, max_iter, ptr,
                                     _stream_handle(stream))
        return p, info


class PoissonSolve(torch.autograd.Function):
    """p = G(rho0) S as a differentiable op (gradients w.r.t. S and rho0).

    The backward pass calls the library's adjoint: forward transforms, the
    transposed tridiagonal solve, inverse transforms, and per-face reductions
    for the rho0 gradient.
    """

    @staticmethod
    def forward(ctx, S, rho0, plan: Plan):
        if rho0 is not None:
            plan.set_rho0(rho0.detach())
        p = plan.solve(S.detach())
        ctx.plan = plan
        ctx.need_rho = rho0 is not None and ctx.needs_input_grad[1]
        ctx.save_for_backward(p)
        return p

    @staticmethod
    def backward(ctx, gp):
        (p,) = ctx.saved_tensors
        gS, grho = ctx.plan.adjoint(gp.contiguous(), p=p, want_grho=ctx.need_rho)
        return gS, grho, None


def poisson_solve(S: torch.Tensor, plan: Plan, rho0: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable solve; pass rho0 (device float64, requires_grad) to train through it."""
    return PoissonSolve.apply(S, rho0, plan)


class Batch:
    """Many independent domains of uneven sizes, solved by one CUDA-graph launch.

    The graph runs the domains' launch sequences on concurrent branches (the
    default); with ``persistent=True``, mixed batches of supported shapes (nx, ny in
    {64, 128, 256, 384, 512}, nz <= 128) run as one persistent kernel over a
    (domain, phase, tile) work list instead.  With ``tune=True`` every distinct grid
    shape gets the autotuner's kernel shapes (measured once per GPU, shape and
    dtype, then cached), applied to the domains' plans (the graph form uses them).
    """

    def __init__(self, domains, dtype="mixed", device=None, tune=False, persistent=False):
        if dtype not in ("fp32", "mixed"):
            raise ValueError("batched solves support dtype 'fp32' or 'mixed'")
        self.dtype = dtype
        self.field_dtype = FIELD_DTYPE[dtype]
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.shapes = [(d.nz, d.ny, d.nx) for d in domains]
        with torch.cuda.device(self.device):
            self._h = N.poisson_batch_create([d.nx for d in domains], [d.ny for d in domains],
                                             [d.nz for d in domains], [d.dx for d in domains],
                                             [d.dy for d in domains], [d.dz for d in domains],
                                             [d.rho0 for d in domains], DTYPES[dtype])
        if tune:
            from .autotune import tuned_options, OPT_IDS
            with torch.cuda.device(self.device):
                for i, d in enumerate(domains):
                    opts = tuned_options(d.nx, d.ny, d.nz, d.dx, d.dy, d.dz, d.rho0, dtype)
                    ph = N.poisson_batch_plan(self._h, i)
                    for k, v in opts.items():
                        N.poisson_plan_set_option(ph, OPT_IDS[k], v)
        N.poisson_batch_set_option(self._h, N.POISSON_BATCH_OPT_PERSISTENT, 1 if persistent else 0)
        self._ws = None
        self._alloc_ws()

    def _alloc_ws(self):
        nb = N.poisson_batch_workspace_bytes(self._h)
        if self._ws is None or self._ws.numel() < nb + 256:
            self._ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)

    def set_option(self, option, value):
        """A batch option (POISSON_BATCH_OPT_*); the workspace grows if the new form needs more."""
        N.poisson_batch_set_option(self._h, option, value)
        self._alloc_ws()

    def _ws_ptr(self):
        ptr = self._ws.data_ptr()
        return ptr + ((-ptr) % 256)

    def solve(self, S_list, out_list=None, info=False, stream=None):
        if len(S_list) != len(self.shapes):
            raise ValueError("one source per domain")
        for S, shp in zip(S_list, self.shapes):
            _require_cuda(S, self.field_dtype, shp, "S")
        outs = out_list if out_list is not None else [torch.empty_like(S) for S in S_list]
        r = N.poisson_batch_solve(self._h, [S.data_ptr() for S in S_list], [p.data_ptr() for p in outs],
                                  self._ws_ptr(), _stream_handle(stream), want_info=info)
        if info:
            return outs, r[1]
        return outs

    def close(self):
        if getattr(self, "_h", None):
            N.poisson_batch_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Pipe:
    """A stream of solves on one plan with fields in host memory (the library's pipeline).

    submit(S, p) enqueues one step (copy S in, solve, copy the solution to p) and
    returns at once; copies of neighbouring steps overlap the solve.  S and p are
    CPU tensors of the plan's field dtype and shape, page-locked for overlap
    (``tensor.pin_memory()``).  wait() blocks until all submitted steps are done and
    raises on the first failed step.  Keep S unchanged and do not read p until wait().
    """

    def __init__(self, plan: Plan):
        self.plan = plan
        with torch.cuda.device(plan.device):
            self._h = N.poisson_pipe_create(plan._h)
        self._keep = []

    def submit(self, S: torch.Tensor, p: torch.Tensor):
        for t, name in ((S, "S"), (p, "p")):
            if t.is_cuda or t.dtype != self.plan.field_dtype or tuple(t.shape) != self.plan.shape \
                    or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CPU tensor of dtype {self.plan.field_dtype} "
                                 f"and shape {self.plan.shape}")
        self._keep.append((S, p))
        N.poisson_pipe_submit(self._h, S.data_ptr(), p.data_ptr())

    def wait(self):
        try:
            N.poisson_pipe_wait(self._h)
        finally:
            self._keep.clear()

    def close(self):
        if getattr(self, "_h", None):
            N.poisson_pipe_destroy(self._h)
            self._h = None
        self._keep = []

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
