"""The algorithmic byte model bench.py divides by kernel time (no GPU):
the multigrid V-cycle bytes against the per-level formula written out, and
the precision forms' step bytes against their definitions."""
import importlib.util
import json
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


def _ncu_csv(path, launches):
    """An ncu --csv --print-units base log: banner lines, then one row per
    launch and metric."""
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
           "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]
    lines = ["==PROF== Connected to process 1", ",".join(f'"{h}"' for h in hdr)]
    for i, (kern, rd, wr, ns) in enumerate(launches):
        for name, unit, v in (("dram__bytes_read.sum", "byte", rd), ("dram__bytes_write.sum", "byte", wr),
                              ("gpu__time_duration.sum", "nsecond", ns)):
            row = [str(i), "1", "python3", "host", kern, "1", "7", "(256, 1, 1)", "(608, 1, 1)", "0", "10.3",
                   "Command line profiler metrics", name, unit, f"{v:,}"]
            lines.append(",".join(f'"{x}"' for x in row))
    open(path, "w").write("\n".join(lines) + "\n")


def test_traffic_record_from_an_ncu_log(bench, tmp_path):
    """--record-traffic takes the third and fifth solver launches of the
    profiling command (the timed headline and plain FP64 field steps),
    divides their DRAM bytes by the algorithmic bytes of the run's own JSON
    line, and the bench finds the record only under the current kernel
    source digest."""
    solver = "void mm::k_solver<4>(mm::Problem)"
    _ncu_csv(tmp_path / "l.csv", [("mm::k_tet_geometry(long)", 10, 0, 5), (solver, 1, 1, 1), (solver, 2, 2, 2),
                                  (solver, 300, 60, 900), ("k_set_field(x)", 0, 0, 1), (solver, 4, 4, 4),
                                  (solver, 2000, 500, 7000)])
    line = {"timed_fields": {"per_step": [{"alg_GB": 0.3, "nli": 8, "evals": 17, "mi": 270, "mr": 21, "li": 21}]},
            "plain_fp64": {"per_step": [{"alg_GB": 2.0, "nli": 8, "evals": 17, "mi": 7000, "mr": 0, "li": 19}]}}
    (tmp_path / "j.log").write_text("noise\n" + json.dumps(line) + "\n")
    out = tmp_path / "t.json"
    bench.record_traffic(str(tmp_path / "l.csv"), str(tmp_path / "j.log"), "cmd", out_path=str(out))
    recs = {r["workload"]: r for r in json.load(open(out))["records"]}
    assert recs["polycrystal_medium"]["ratio"] == pytest.approx(360 / 0.3e9)
    assert recs["large_polycrystal"]["ratio"] == recs["polycrystal_medium"]["ratio"]
    assert recs["polycrystal_medium/plain_fp64"]["ratio"] == pytest.approx(2500 / 2.0e9)
    assert recs["polycrystal_medium"]["gpu_time_ns"] == 900
    old = bench.TRAFFIC
    try:
        bench.TRAFFIC = str(out)                      # an absolute path: os.path.join keeps it
        assert bench.traffic_record("large_polycrystal")["ratio"] == pytest.approx(360 / 0.3e9)
        assert bench.traffic_record("hard_cube") is None
        d = json.load(open(out))
        for r in d["records"]:
            r["sources"] = "0" * 16                   # as if the kernel sources had changed since
        json.dump(d, open(out, "w"))
        assert bench.traffic_record("large_polycrystal") is None
    finally:
        bench.TRAFFIC = old
