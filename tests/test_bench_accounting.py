"""Host logic of bench.py's roofline accounting (no GPU): the algorithmic bytes of a mixed
solve, per phase and in total, against the counts the method fixes."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench_acc", os.path.join(ROOT, "bench.py"))
B = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(B)


@pytest.mark.parametrize("sweeps", [0, 1, 2, 3])
def test_total_is_read_S_write_p_and_one_spectrum_round_trip_per_pass(sweeps):
    nx, ny, nz = 1024, 1024, 128
    N, Nc = nx * ny * nz, (nx // 2 + 1) * ny * nz
    per_phase, total = B.algorithmic_bytes(nx, ny, nz, sweeps)
    # first solve: S (8 B) in, p (8 B) out, spectrum (8 B/entry) written and read once
    # each sweep: S and p read, p updated (read + write), spectrum once
    assert total == 16 * N + 16 * Nc + sweeps * (32 * N + 16 * Nc)
    # the 1024^2 x 128 workload with one sweep moves 8.59 GB (64 B per point)
    if sweeps == 1:
        assert abs(total / 1e9 - 8.594) < 1e-3
    # every pass moves the spectrum once each way on the y-passes and the columns
    for name in ("yfwd", "columns", "yinv"):
        assert per_phase[name] == (1 + sweeps) * 16 * Nc
    # the correction rebuild runs before a third sweep only; a stop after sweep 1 writes p = p0 + q
    assert per_phase["residual"] == (16 * N if sweeps >= 3 else 0)
    assert per_phase["control"] == (16 * N if sweeps == 1 else 0)
    # sweep 1 stores q (4 B) when more sweeps are allowed; every later sweep stores p (8 B)
    xinv = (8 * Nc + 4 * N) + sum(8 * Nc + 4 * N + (4 * N if s > 1 else 0) + (4 * N if s == 1 else 8 * N)
                                  for s in range(1, sweeps + 1))
    assert per_phase["xinv"] == xinv


def test_one_sweep_allowed_stores_p_in_its_inverse_pass():
    nx, ny, nz = 256, 256, 64
    N, Nc = nx * ny * nz, (nx // 2 + 1) * ny * nz
    per_phase, _ = B.algorithmic_bytes(nx, ny, nz, 1, max_sweeps=1)
    assert per_phase["xinv"] == (8 * Nc + 4 * N) + (8 * Nc + 4 * N + 8 * N)
    assert per_phase["control"] == 0


def test_fp64_operation_count():
    # 1024 x 1024: real transforms 2.5 log2(1024) = 25 per point each way; complex y transforms of the
    # 513 half-spectrum columns 5 log2(1024) 513/1024 per point each way; columns 18 per complex entry
    f = B.fp64_flops_per_point(1024, 1024, 128)
    assert f == pytest.approx(2 * (25 + 50 * 513 / 1024) + 18 * 513 / 1024)


def test_forward_x_phase_bytes_are_the_roofline_unit():
    nx, ny, nz = 1024, 1024, 128
    N, Nc = nx * ny * nz, (nx // 2 + 1) * ny * nz
    per_phase, _ = B.algorithmic_bytes(nx, ny, nz, 1)
    # first solve 8N + 8Nc (S in, spectrum out); sweep 1: 12N + 8Nc (S and p0 in, spectrum out)
    assert per_phase["xfwd"] == (8 * N + 8 * Nc) + (12 * N + 8 * Nc)
    assert abs(per_phase["xfwd"] / 2 / 1e9 - 1.880) < 1e-3


def test_whole_job_rate_counts_all_ranks():
    assert B.whole_job_rate(1_000_000, 4, 2.0) == pytest.approx(4 * 1_000_000 / 2e-3 / 1e6)


def test_verified_solve_counts_one_sweep_plus_the_verification():
    nx, ny, nz = 1024, 1024, 128
    N, Nc = nx * ny * nz, (nx // 2 + 1) * ny * nz
    per_phase, total = B.algorithmic_bytes(nx, ny, nz, 1, max_sweeps=3, verified=True)
    # first solve + one applied sweep + a verification sweep (S and p read, spectrum once)
    assert total == 16 * N + 16 * Nc + (32 * N + 16 * Nc) + (16 * N + 16 * Nc)
    for name in ("yfwd", "columns"):
        assert per_phase[name] == 3 * 16 * Nc
    assert per_phase["yinv"] == 2 * 16 * Nc
    assert per_phase["control"] == 0          # the verification's residual pass stores p itself
    # its residual x-pass: S, p0, q in; spectrum and p out
    assert per_phase["xfwd"] == (8 * N + 8 * Nc) + (12 * N + 8 * Nc) + (16 * N + 8 * Nc + 8 * N)


def test_low_wavenumber_verification_moves_its_part_of_the_spectrum():
    nx, ny, nz = 1024, 1024, 128
    N, Nc = nx * ny * nz, (nx // 2 + 1) * ny * nz
    kc = B.verify_cut(nx, ny)
    assert kc == 128
    Ncx, Ncl = (kc + 1) * ny * nz, (kc + 1) * (2 * kc + 1) * nz
    per_phase, total = B.algorithmic_bytes(nx, ny, nz, 1, max_sweeps=3, verified=True, kcut=kc)
    assert total == 16 * N + 16 * Nc + (32 * N + 16 * Nc) + (16 * N + 16 * Ncx)
    assert per_phase["yfwd"] == 2 * 16 * Nc + 16 * Ncx
    assert per_phase["columns"] == 2 * 16 * Nc + 16 * Ncl
    # sweep 1 also writes its residual r0 (4 B); the first try reads r0, p0 and q (4 B each) and writes the
    # low-kx transform and p
    assert per_phase["xfwd"] == (8 * N + 8 * Nc) + (12 * N + 8 * Nc + 4 * N) + (12 * N + 8 * Ncx + 8 * N)


@pytest.mark.parametrize("nx,ny,lowk,expect", [(1024, 1024, 64, 128), (384, 256, 64, 48), (64, 512, 64, None),
                                               (256, 64, 64, None), (512, 512, 400, 64), (512, 512, 4096, None)])
def test_verify_cut_rule(nx, ny, lowk, expect):
    # kcut = nx/8 while it exceeds 8 and the low-|k| radius, stays inside the half spectrum and leaves
    # high rows in y (2 kcut + 1 < ny)
    assert B.verify_cut(nx, ny, lowk) == expect
