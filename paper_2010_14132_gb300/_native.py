"""ctypes binding of the C ABI in include/poisson.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Pointers are
plain integers (device addresses), streams are cudaStream_t handles as
integers.  A missing library raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpoisson_gb300.so")

POISSON_OK = 0
POISSON_ERR_INVALID_ARG = -1
POISSON_ERR_UNSUPPORTED = -2
POISSON_ERR_CUDA = -3
POISSON_ERR_WORKSPACE = -4
POISSON_ERR_NOT_CONVERGED = -5
POISSON_ERR_TIMEOUT = -6

POISSON_BC_PERIODIC_XY_NEUMANN_Z = 0
POISSON_BC_PERIODIC_XY_NEUMANN_BOTTOM_DIRICHLET_TOP = 1
POISSON_FP64, POISSON_FP32, POISSON_MIXED = 0, 1, 2
POISSON_OPT_LOWK_RADIUS2, POISSON_OPT_MAX_SWEEPS, POISSON_OPT_TOLERANCE, POISSON_OPT_Y_TILE = 0, 1, 2, 3
POISSON_OPT_PROFILE = 4
POISSON_OPT_Y_KERNEL = 5
POISSON_OPT_X_ELEMS = 6
POISSON_OPT_Y_ELEMS = 7
POISSON_OPT_LEVEL_CHUNK = 8
POISSON_OPT_X_KERNEL = 9
POISSON_OPT_COL_TILE = 10
POISSON_OPT_LAYOUT = 11
POISSON_OPT_SPECTRAL_FUSED = 12
POISSON_OPT_RESIDUAL_PASS = 13
POISSON_OPT_VERIFY = 14
POISSON_OPT_GRAPH = 15
POISSON_BATCH_OPT_PERSISTENT = 0
POISSON_BATCH_OPT_STALL_TEST = 1
POISSON_BATCH_OPT_BRANCHES = 2
POISSON_LAYOUT_Z_Y_X = 0
POISSON_LAYOUT_X_Y_Z = 1
PHASES = ("xfwd", "yfwd", "columns", "yinv", "xinv", "residual", "control", "spectral")

# every symbol include/poisson.h declares
EXPORTED = (
    "poisson_plan_create", "poisson_plan_workspace_bytes", "poisson_plan_set_option", "poisson_plan_set_rho0",
    "poisson_solve", "poisson_solve_adjoint", "poisson_plan_destroy", "poisson_status_string",
    "poisson_last_error_detail", "poisson_batch_create", "poisson_batch_workspace_bytes", "poisson_batch_solve",
    "poisson_batch_destroy", "poisson_plan_profile_read", "poisson_solve_static_workspace",
    "poisson_pipe_create", "poisson_pipe_submit", "poisson_pipe_wait", "poisson_pipe_destroy",
    "poisson_batch_plan", "poisson_cg_workspace_bytes", "poisson_cg_solve", "poisson_batch_set_option",
)

# size of the fixed device array poisson_solve_static_workspace uses as scratch
POISSON_STATIC_WORKSPACE_BYTES = 32 * 1024 * 1024


class PoissonInfo(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int),
        ("converged", C.c_int),
        ("rel_update", C.c_double * 4),
        ("error_estimate", C.c_double),
        ("removed_weighted_mean", C.c_double),
        ("rel_residual", C.c_double * 4),
        ("accuracy_floor", C.c_double),
    ]

    def as_dict(self):
        return {
            "sweeps": self.sweeps, "converged": bool(self.converged),
            "rel_update": list(self.rel_update), "error_estimate": self.error_estimate,
            "removed_weighted_mean": self.removed_weighted_mean,
            "rel_residual": list(self.rel_residual), "accuracy_floor": self.accuracy_floor,
        }


class PoissonCgInfo(C.Structure):
    _fields_ = [
        ("iterations", C.c_int),
        ("converged", C.c_int),
        ("rel_residual", C.c_double),
        ("removed_weighted_mean", C.c_double),
    ]

    def as_dict(self):
        return {"iterations": self.iterations, "converged": bool(self.converged),
                "rel_residual": self.rel_residual, "removed_weighted_mean": self.removed_weighted_mean}


class PoissonError(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = ""
        try:
            lib = load()
            detail = lib.poisson_status_string(status).decode()
            if status == POISSON_ERR_CUDA:
                detail += ": " + lib.poisson_last_error_detail().decode()
        except Exception:  # pragma: no cover - message only
            pass
        super().__init__(f"{where} failed with status {status} ({detail})")
        self.status = status


_lib = None


def load():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"solver library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    dp = C.POINTER(C.c_double)
    L.poisson_plan_create.argtypes = [i, i, i, d, d, dp, dp, i, i, C.POINTER(vp)]
    L.poisson_plan_workspace_bytes.argtypes = [vp, C.POINTER(sz)]
    L.poisson_plan_set_option.argtypes = [vp, i, d]
    L.poisson_plan_set_rho0.argtypes = [vp, vp, vp]
    L.poisson_solve.argtypes = [vp, vp, vp, vp, vp, C.POINTER(PoissonInfo)]
    L.poisson_solve_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.poisson_plan_destroy.argtypes = [vp]
    L.poisson_status_string.argtypes = [i]
    L.poisson_status_string.restype = C.c_char_p
    L.poisson_last_error_detail.argtypes = []
    L.poisson_last_error_detail.restype = C.c_char_p
    L.poisson_batch_create.argtypes = [i, C.POINTER(i), C.POINTER(i), C.POINTER(i), dp, dp, C.POINTER(dp),
                                       C.POINTER(dp), i, C.POINTER(vp)]
    L.poisson_batch_workspace_bytes.argtypes = [vp, C.POINTER(sz)]
    L.poisson_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), vp, vp, C.POINTER(PoissonInfo)]
    L.poisson_batch_destroy.argtypes = [vp]
    L.poisson_plan_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int), i]
    L.poisson_solve_static_workspace.argtypes = [vp, vp, vp, vp, C.POINTER(PoissonInfo)]
    L.poisson_pipe_create.argtypes = [vp, C.POINTER(vp)]
    L.poisson_batch_plan.argtypes = [vp, i, C.POINTER(vp)]
    L.poisson_batch_set_option.argtypes = [vp, i, d]
    L.poisson_pipe_submit.argtypes = [vp, vp, vp]
    L.poisson_pipe_wait.argtypes = [vp]
    L.poisson_pipe_destroy.argtypes = [vp]
    L.poisson_cg_workspace_bytes.argtypes = [vp, C.POINTER(sz)]
    L.poisson_cg_solve.argtypes = [vp, vp, vp, vp, d, i, vp, vp, C.POINTER(PoissonCgInfo)]
    for name in EXPORTED:
        if name not in ("poisson_status_string", "poisson_last_error_detail"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status: int, where: str, allow=()):
    if status != POISSON_OK and status not in allow:
        raise PoissonError(status, where)
    return status


def _darr(values):
    vals = [float(v) for v in values]
    return (C.c_double * len(vals))(*vals)


def poisson_plan_create(nx, ny, nz, dx, dy, dz, rho0, bc, dtype):
    L = load()
    out = C.c_void_p()
    _check(L.poisson_plan_create(int(nx), int(ny), int(nz), float(dx), float(dy), _darr(dz), _darr(rho0),
                                 int(bc), int(dtype), C.byref(out)), "poisson_plan_create")
    return out.value


def poisson_plan_workspace_bytes(plan) -> int:
    n = C.c_size_t()
    _check(load().poisson_plan_workspace_bytes(plan, C.byref(n)), "poisson_plan_workspace_bytes")
    return n.value


def poisson_plan_set_option(plan, option, value):
    _check(load().poisson_plan_set_option(plan, int(option), float(value)), "poisson_plan_set_option")


def poisson_plan_set_rho0(plan, rho0_dev_ptr, stream):
    _check(load().poisson_plan_set_rho0(plan, rho0_dev_ptr, stream), "poisson_plan_set_rho0")


def poisson_solve(plan, S_ptr, p_ptr, ws_ptr, stream, want_info=False, allow_not_converged=True):
    info = PoissonInfo() if want_info else None
    st = load().poisson_solve(plan, S_ptr, p_ptr, ws_ptr, stream, C.byref(info) if info is not None else None)
    _check(st, "poisson_solve", allow=(POISSON_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return (st, info.as_dict()) if want_info else st


def poisson_solve_static_workspace(plan, S_ptr, p_ptr, stream, want_info=False):
    """Solve with the library's fixed device scratch array (allocates nothing).

    Returns the raw status (POISSON_ERR_WORKSPACE for plans above the maximum),
    or (status, info) with want_info."""
    info = PoissonInfo() if want_info else None
    st = load().poisson_solve_static_workspace(plan, S_ptr, p_ptr, stream,
                                               C.byref(info) if info is not None else None)
    return (st, info.as_dict()) if want_info else st


def poisson_solve_adjoint(plan, gp_ptr, p_ptr, gS_ptr, grho_ptr, ws_ptr, stream):
    _check(load().poisson_solve_adjoint(plan, gp_ptr, p_ptr, gS_ptr, grho_ptr, ws_ptr, stream),
           "poisson_solve_adjoint")


def poisson_plan_destroy(plan):
    if plan:
        load().poisson_plan_destroy(plan)


def poisson_plan_profile_read(plan):
    """{phase name: (total ms, launches)} since the last read."""
    k = len(PHASES)
    ms = (C.c_double * k)()
    cnt = (C.c_int * k)()
    _check(load().poisson_plan_profile_read(plan, ms, cnt, k), "poisson_plan_profile_read")
    return {PHASES[i]: (ms[i], cnt[i]) for i in range(k)}


def poisson_status_string(status) -> str:
    return load().poisson_status_string(int(status)).decode()


def poisson_last_error_detail() -> str:
    return load().poisson_last_error_detail().decode()


def poisson_batch_create(nx, ny, nz, dx, dy, dz_list, rho0_list, dtype):
    L = load()
    n = len(nx)
    I = C.c_int * n
    D = C.c_double * n
    dz_arrs = [_darr(v) for v in dz_list]
    rho_arrs = [_darr(v) for v in rho0_list]
    DP = C.POINTER(C.c_double) * n
    dzp = DP(*[C.cast(a, C.POINTER(C.c_double)) for a in dz_arrs])
    rhp = DP(*[C.cast(a, C.POINTER(C.c_double)) for a in rho_arrs])
    out = C.c_void_p()
    _check(L.poisson_batch_create(n, I(*nx), I(*ny), I(*nz), D(*dx), D(*dy), dzp, rhp, int(dtype), C.byref(out)),
           "poisson_batch_create")
    return out.value


def poisson_batch_workspace_bytes(batch) -> int:
    n = C.c_size_t()
    _check(load().poisson_batch_workspace_bytes(batch, C.byref(n)), "poisson_batch_workspace_bytes")
    return n.value


def poisson_batch_solve(batch, S_ptrs, p_ptrs, ws_ptr, stream, want_info=False):
    n = len(S_ptrs)
    P = C.c_void_p * n
    infos = (PoissonInfo * n)() if want_info else None
    st = load().poisson_batch_solve(batch, P(*S_ptrs), P(*p_ptrs), ws_ptr, stream,
                                    C.cast(infos, C.POINTER(PoissonInfo)) if want_info else None)
    _check(st, "poisson_batch_solve", allow=(POISSON_ERR_NOT_CONVERGED,))
    return (st, [x.as_dict() for x in infos]) if want_info else st


def poisson_batch_destroy(batch):
    if batch:
        load().poisson_batch_destroy(batch)


def poisson_pipe_create(plan):
    out = C.c_void_p()
    _check(load().poisson_pipe_create(plan, C.byref(out)), "poisson_pipe_create")
    return out.value


def poisson_pipe_submit(pipe, S_host_ptr, p_host_ptr):
    return _check(load().poisson_pipe_submit(pipe, S_host_ptr, p_host_ptr), "poisson_pipe_submit")


def poisson_pipe_wait(pipe):
    return _check(load().poisson_pipe_wait(pipe), "poisson_pipe_wait")


def poisson_pipe_destroy(pipe):
    if pipe:
        load().poisson_pipe_destroy(pipe)


def poisson_batch_plan(batch, i):
    out = C.c_void_p()
    _check(load().poisson_batch_plan(batch, int(i), C.byref(out)), "poisson_batch_plan")
    return out.value


def poisson_batch_set_option(batch, option, value):
    _check(load().poisson_batch_set_option(batch, int(option), float(value)), "poisson_batch_set_option")


def poisson_cg_workspace_bytes(plan):
    n = C.c_size_t(0)
    _check(load().poisson_cg_workspace_bytes(plan, C.byref(n)), "poisson_cg_workspace_bytes")
    return n.value


def poisson_cg_solve(plan, rho_ptr, S_ptr, p_ptr, tol, max_iter, ws_ptr, stream, allow_not_converged=True):
    """Returns (status, info dict)."""
    info = PoissonCgInfo()
    st = load().poisson_cg_solve(plan, rho_ptr, S_ptr, p_ptr, float(tol), int(max_iter), ws_ptr, stream,
                                 C.byref(info))
    _check(st, "poisson_cg_solve", allow=(POISSON_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return st, info.as_dict()
