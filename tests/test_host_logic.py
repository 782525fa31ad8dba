"""Host-side checks that need no GPU: the C-ABI library loads and exports every
symbol include/poisson.h declares, and argument validation returns the
documented status codes without touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2010_14132_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "poisson.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(poisson_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    assert header_functions() == sorted(N.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = N.load()
    for name in header_functions():
        assert hasattr(lib, name), name


def test_status_strings():
    assert N.poisson_status_string(0) == "ok"
    for s in range(-6, 0):
        assert N.poisson_status_string(s) not in ("", "unknown status")
    assert N.poisson_status_string(42) == "unknown status"


def _create(nx, ny, nz, dx=1.0, dy=1.0, dz=None, rho=None, bc=0, dtype=0):
    lib = N.load()
    dz = np.ones(nz) if dz is None else dz
    rho = np.ones(nz) if rho is None else rho
    out = C.c_void_p(123)
    st = lib.poisson_plan_create(nx, ny, nz, dx, dy, N._darr(dz), N._darr(rho), bc, dtype, C.byref(out))
    return st, out.value


@pytest.mark.parametrize("dims", [(5, 8, 4), (7, 8, 4), (10, 8, 4), (8, 14, 4), (2, 8, 4), (8, 2, 4), (8, 8, 1),
                                  (8, 8, 513), (8192, 8, 4), (8, 8192, 4), (8, 25, 4)])
def test_unsupported_sizes(dims):
    st, out = _create(*dims)
    assert st == N.POISSON_ERR_UNSUPPORTED
    assert out is None


@pytest.mark.parametrize("kw", [dict(dx=0.0), dict(dy=-1.0), dict(dx=float("nan")), dict(bc=3), dict(bc=2), dict(bc=-1), dict(dtype=7),
                                dict(dz=np.array([1.0, 0.0, 1.0, 1.0])), dict(rho=np.array([1.0, 1.0, -2.0, 1.0]))])
def test_invalid_arguments(kw):
    st, out = _create(8, 8, 4, **kw)
    assert st == N.POISSON_ERR_INVALID_ARG
    assert out is None


def test_null_arguments():
    lib = N.load()
    assert lib.poisson_plan_create(8, 8, 4, 1.0, 1.0, None, None, 0, 0, None) == N.POISSON_ERR_INVALID_ARG
    assert lib.poisson_solve(None, None, None, None, None, None) == N.POISSON_ERR_INVALID_ARG
    assert lib.poisson_solve_adjoint(None, None, None, None, None, None, None) == N.POISSON_ERR_INVALID_ARG
    assert lib.poisson_plan_set_option(None, 0, 1.0) == N.POISSON_ERR_INVALID_ARG
    assert lib.poisson_plan_destroy(None) == N.POISSON_OK
    assert lib.poisson_batch_destroy(None) == N.POISSON_OK
    n = C.c_size_t()
    assert lib.poisson_plan_workspace_bytes(None, C.byref(n)) == N.POISSON_ERR_INVALID_ARG
    out = C.c_void_p()
    assert lib.poisson_batch_create(0, None, None, None, None, None, None, None, 2, C.byref(out)) == \
        N.POISSON_ERR_INVALID_ARG


def test_python_wrapper_raises_on_bad_size():
    with pytest.raises(N.PoissonError) as e:
        N.poisson_plan_create(9, 8, 4, 1.0, 1.0, np.ones(4), np.ones(4), 0, 0)
    assert e.value.status == N.POISSON_ERR_UNSUPPORTED


def test_plan_rejects_unknown_boundary_condition_before_any_device_call():
    from paper_2010_14132_gb300.solver import Plan
    with pytest.raises(ValueError):
        Plan(8, 8, 4, 1.0, 1.0, np.ones(4), np.ones(4), dtype="fp64", bc="dirichlet")


def test_cg_entry_points_reject_null_arguments():
    lib = N.load()
    n = C.c_size_t(0)
    assert lib.poisson_cg_workspace_bytes(None, C.byref(n)) == N.POISSON_ERR_INVALID_ARG
    info = N.PoissonCgInfo()
    info.iterations = 7
    st = lib.poisson_cg_solve(None, None, None, None, 1e-10, 10, None, None, C.byref(info))
    assert st == N.POISSON_ERR_INVALID_ARG
    assert info.iterations == 0 and info.converged == 0   # cleared before any check


def test_header_enum_values_match_the_binding():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    values = dict((k, int(v)) for k, v in re.findall(r"\b(POISSON_[A-Z0-9_]+)\s*=\s*(-?\d+)", text))
    named = {k: v for k, v in values.items() if hasattr(N, k)}
    assert len(named) >= 20
    for k, v in named.items():
        assert getattr(N, k) == v, k
    assert N.POISSON_BATCH_OPT_BRANCHES == values["POISSON_BATCH_OPT_BRANCHES"]
