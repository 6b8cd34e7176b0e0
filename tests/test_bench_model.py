"""The algorithmic byte model bench.py divides by kernel time (no GPU):
the multigrid V-cycle bytes against the per-level formula written out, and
the precision forms' step bytes against their definitions."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


LEVELS = [{"rows": 1000, "nnz_a": 15000, "nnz_u": 9000, "nnz_p": 4000},
          {"rows": 40, "nnz_a": 1600, "nnz_u": 500, "nnz_p": 300},
          {"rows": 3, "nnz_a": 9, "nnz_u": None, "nnz_p": None}]


def test_vcycle_bytes(bench):
    # level 0: 8*15000 + 8*4000 (P^T) + 8*9000 (U) + 28*1000 + 16*40; level 1
    # (last smoothed): 8*1600 + 8*300 + 8*500 + 28*40 + 8*3; dense coarsest 4*9 + 8*3
    want = ((8 * 15000 + 8 * 4000 + 8 * 9000 + 28 * 1000 + 16 * 40) + (8 * 1600 + 8 * 300 + 8 * 500 + 28 * 40 + 8 * 3)
            + (4 * 9 + 8 * 3))
    assert bench.vcycle_bytes(LEVELS) == want


def test_step_bytes(bench):
    sz = {"n_phi": 1000, "n_mag": 100, "nnz_phi": 15000, "nnz_mag": 1400}
    st = {"mi": 20, "mr": 2, "evals": 3, "li": 4, "nli": 1}
    base = bench.alg_bytes(dict(st, mi=0, mr=0), sz)
    jac = bench.alg_bytes(st, sz) - base
    assert jac == 18 * (8 * 15000 + 52 * 1000) + 2 * (12 * 15000 + 60 * 1000)
    mg = bench.alg_bytes(st, sz, LEVELS) - base
    vc = bench.vcycle_bytes(LEVELS)
    assert mg == 18 * (8 * 15000 + 52 * 1000 + vc) + 2 * (12 * 15000 + 60 * 1000 + vc)


def test_step_bytes_with_the_fp32_layout(bench):
    """With the FP32 K_phi's own matrix bytes given (k32_bytes), the FP32
    products (the direction pass and the level-0 down phase) count those
    instead of 8 nnz_phi; the FP64 products keep 12 nnz_phi."""
    kb = 70000
    sz = {"n_phi": 1000, "n_mag": 100, "nnz_phi": 15000, "nnz_mag": 1400, "k32_bytes": kb}
    st = {"mi": 20, "mr": 2, "evals": 3, "li": 4, "nli": 1}
    base = bench.alg_bytes(dict(st, mi=0, mr=0), sz)
    assert bench.alg_bytes(st, sz) - base == 18 * (kb + 52 * 1000) + 2 * (12 * 15000 + 60 * 1000)
    vc = bench.vcycle_bytes(LEVELS, kb)
    assert vc == bench.vcycle_bytes(LEVELS) - 8 * 15000 + kb
    assert bench.alg_bytes(st, sz, LEVELS) - base == 18 * (kb + 52 * 1000 + vc) + 2 * (12 * 15000 + 60 * 1000 + vc)


def test_inner_step_bytes_of_the_precision_form(bench):
    """The precision form's preconditioner runs in FP32: an inner step moves
    8 nnz_mag + 228 n_mag, the per-iteration set-up and direction 244 n_mag,
    against 12 nnz_mag + 352 n_mag and 272 n_mag in FP64."""
    sz = {"n_phi": 1000, "n_mag": 100, "nnz_phi": 15000, "nnz_mag": 1400}
    st = {"mi": 0, "mr": 0, "evals": 3, "li": 4, "nli": 1}
    d64 = bench.alg_bytes(st, sz) - bench.alg_bytes(dict(st, li=0), sz)
    d32 = bench.alg_bytes(st, sz, precision=1) - bench.alg_bytes(dict(st, li=0), sz, precision=1)
    assert d64 == 4 * (12 * 1400 + 352 * 100) and d32 == 4 * (8 * 1400 + 228 * 100)
    i64 = bench.alg_bytes(st, sz) - bench.alg_bytes(dict(st, nli=0), sz)
    i32 = bench.alg_bytes(st, sz, precision=1) - bench.alg_bytes(dict(st, nli=0), sz, precision=1)
    assert i64 == 272 * 100 and i32 == 244 * 100
