"""Benchmark: NCG iterations per second of the preconditioned NCG minimiser
over the field steps of a demagnetisation curve (Sec. 3.1, Algorithm 4),
against the plain FP64 GPU method on the same field steps.

Workload (default, large_polycrystal): a polycrystalline Nd2Fe14B cube,
250 nm edge, 149^3 voxels of 6 tetrahedra (19.8 M magnet tets, 3,375,000
magnetic nodes), 125 Voronoi grains with easy axes uniform in a 15 degree
cone about +z and a 2 nm grain-boundary phase (Ms and K1 at 40%), in an air
box of twice the edge graded by 1.06 per cell (53.2 M tets, 8,741,816
potential unknowns); m0 = +z; field along -z from 0 to -8 T in 60 values.
One step = one field step of the curve: set the field, minimise by
Algorithm 4 until t1-t3 hold.

value: NCG iterations / s of the precision form (FP32 potential solve
preconditioned by the multigrid V-cycle, FP64 refinement, FP64 everything
else) with everything resident on the device (summed over ranks, max time
over ranks).  plain_fp64: the same field steps (a prefix of them, see
--fp64-steps) in plain FP64 (Jacobi-preconditioned potential CG).  e2e: the
headline form through the public API with host buffers: each step uploads m
from pinned host memory, sets the field, minimises and reads m back.
demag_curve: full 40-field curves of the 80 nm hard cube (117,649 magnetic
nodes) in the precision and plain FP64 forms, wall time and coercive field.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the CPU oracle legs run in subprocesses with their own thread settings;
# this process pins the BLAS / OpenMP pools to one thread before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NCG iters/s & demag-curve wall time vs plain FP64 GPU at equal energy tol"
UNIT = "NCG it/s"
WORKLOADS = ["large_polycrystal", "large_polycrystal_patches", "polycrystal_medium", "polycrystal", "hard_cube",
             "medium", "soft_cube", "small"]


def workload(name, sample=False):
    """The named workload; sample=True gives the same recipe at the reduced
    resolution the CPU oracle legs time (32 voxels per magnet edge for the
    large polycrystal)."""
    import synth
    if name == "large_polycrystal":
        return synth.large_polycrystal(n_mag=32) if sample else synth.large_polycrystal()
    if name == "polycrystal_medium":
        # the large polycrystal's recipe at 100^3 voxels (same spacing and air
        # grading, 37 grains): the profiling case, a few GB on the device
        return synth.large_polycrystal(n_mag=32 if sample else 100, edge=(32 if sample else 100) * 250e-9 / 149,
                                       n_grains=37)
    if name == "large_polycrystal_patches":
        return synth.large_polycrystal(n_mag=32 if sample else 149, patches_per_grain=10)
    if name == "polycrystal":
        return synth.polycrystal_cube(n_mag=32 if sample else 114)
    if name == "hard_cube":
        return synth.hard_cube(n_mag=24 if sample else 48)
    if name == "soft_cube":
        return synth.soft_cube()
    if name == "medium":
        return synth.hard_cube(n_mag=24 if sample else 44)
    if name == "small":
        return synth.hard_cube(n_mag=12)
    raise ValueError(name)


def workload_desc(name, wl, sizes=None):
    d = {"workload": f"{wl.name}: {name}", "n_nodes": wl.mesh.n_nodes, "n_tets": wl.mesh.n_tets,
         "fields": f"{len(wl.fields)} values from {wl.fields[0].tolist()} to {wl.fields[-1].tolist()} T",
         "jmax": 4, "tau_F": 1e-10, "poisson_tol": 1e-10,
         "l2": "working set larger than L2 (no flush needed)"}
    if sizes:
        d.update(sizes)
    return d


# ------------------------------------------------------------ algorithmic bytes
def model_sizes(mag):
    """Sizes the byte model needs: the mesh's (mm_sizes) and the matrix bytes
    of one product with the FP32 K_phi in its uploaded layout."""
    sz = mag.sizes()
    k = mag.k32_layout()
    sz["k32_bytes"] = k["matrix_bytes"]
    sz["k32_table_slice_frac"] = k["table_slices"] / max(k["slices"], 1)
    return sz


def form_params(form, theta_max=0.1):
    """Parameters of the three forms of a field step: 0 plain FP64
    (Jacobi-preconditioned potential solve, the paper's method in FP64), 1
    precision form with Jacobi, 2 the headline: precision form with the
    multigrid preconditioner and the potential tolerance tied to t1."""
    from paper_1801_03690_gb300 import Params
    if form == 0:
        return Params(jmax=4, tau_F=1e-10, poisson_tol=1e-10, precision=0, theta_max=theta_max)
    if form == 1:
        return Params(jmax=4, tau_F=1e-10, poisson_tol=1e-10, precision=1, theta_max=theta_max)
    return Params(jmax=4, tau_F=1e-10, poisson_tol=1e-10, precision=1, amg=1, inner_tol=1e-3,
                  poisson_sched=1, theta_max=theta_max)


def vcycle_bytes(amg, k32_bytes=None):
    """Bytes of one multigrid V-cycle (levels l < L smoothed, L dense):
      down_l  8 nnz_A_l + 12 n_l + 8 nnz_P_l + 12 n_{l+1} (4 n_L at the last)
              (A and P^T val+col; x, b read, rpre written; b, x of l+1 written;
              at level 0, A is the FP32 K_phi: k32_bytes for the matrix when
              given, the layout's own count)
      dense   4 n_L^2 + 8 n_L
      up_l    8 nnz_U_l + 4 n_{l+1} + 16 n_l (U; y_{l+1}; b, rpre, diag^-1 -> y)"""
    L = len(amg) - 1
    tot = 4 * amg[L]["nnz_a"] + 8 * amg[L]["rows"]
    for l in range(L):
        n, nc = amg[l]["rows"], amg[l + 1]["rows"]
        a_bytes = k32_bytes if (l == 0 and k32_bytes is not None) else 8 * amg[l]["nnz_a"]
        tot += a_bytes + 12 * n + 8 * amg[l]["nnz_p"] + (4 if l + 1 == L else 12) * nc
        tot += 8 * amg[l]["nnz_u"] + 4 * nc + 16 * n
    return tot


def alg_bytes(st, sz, amg=None, precision=0):
    """Bytes one minimisation launch must move at ideal reuse (every array
    element read or written once per phase, neighbour gathers served from
    cache), from the launch's own counters:
      potential step (mi)   FP64: 12 nnz_phi + 96 n_phi (SELL val+col; z gather,
                            d, q read+write; phi, d, r, q, diag^-1 -> phi, r, z)
                            precision form: FP32 steps 8 nnz_phi + 52 n_phi,
                            FP64 refinements (mr) 12 nnz_phi + 60 n_phi;
                            with the multigrid preconditioner (amg = the
                            hierarchy's levels) an FP32 step is the
                            direction pass 8 nnz_phi + 20 n_phi, the update
                            pass 32 n_phi and a V-cycle (vcycle_bytes), a
                            refinement adds a V-cycle
      evaluation (evals)    12 nnz_phi + 64 nnz_mag + 48 n_phi + 208 n_mag
                            (potential set-up incl. D m; energy/gradient pass)
      trial point (evals-1) 112 n_mag
      inner step (li)       12 nnz_mag + 352 n_mag  (H product + update);
                            precision form: 8 nnz_mag + 228 n_mag (FP32
                            K_A and vectors; m, lambda, y in FP64)
      per iteration (nli+1) 272 n_mag               (inner set-up + direction;
                                                     precision form 244 n_mag)
    nnz_phi is the stored potential stiffness (without the rounding residues
    the upload drops).  The FP32 products' 8 nnz_phi (val+col) become
    sz["k32_bytes"] when given: the matrix bytes of the FP32 K_phi's own
    layout (slices with an offset table store values only).
    """
    nphi, nm = sz["n_phi"], sz["n_mag"]
    nzp, nzm = sz["nnz_phi"], sz["nnz_mag"]
    kb = sz.get("k32_bytes")
    k32 = 8 * nzp if kb is None else kb
    per_pcg = 12 * nzp + 96 * nphi
    per_pcg32 = k32 + 52 * nphi              # FP32 step: the matrix; 13 FP32 vector passes
    per_refine = 12 * nzp + 60 * nphi        # FP64 residual product + FP32 set-up
    per_eval = 12 * nzp + 64 * nzm + 48 * nphi + 208 * nm
    per_trial = 112 * nm
    per_inner = (8 * nzm + 228 * nm) if precision else (12 * nzm + 352 * nm)
    per_iter = (244 if precision else 272) * nm
    mr = st.get("mr", 0)
    if amg:
        vc = vcycle_bytes(amg, kb)
        per_pcg32 = k32 + 20 * nphi + 32 * nphi + vc
        per_refine += vc
    steps = (st["mi"] - mr) * per_pcg32 + mr * per_refine if mr else st["mi"] * per_pcg
    return (steps + st["evals"] * per_eval + max(st["evals"] - 1, 0) * per_trial
            + st["li"] * per_inner + (st["nli"] + 1) * per_iter)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, v in zip(names, r[2:]):
                if v.lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median([r[0] for r in rows]), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def merge_clocks(cks):
    cks = [c for c in cks if c]
    if not cks:
        return None
    return {"sm_mhz": statistics.median([c["sm_mhz"] for c in cks]), "sm_max_mhz": max(c["sm_max_mhz"] for c in cks),
            "reasons": sorted(set().union(*[set(c["reasons"]) for c in cks])),
            "samples": sum(c["samples"] for c in cks)}


# ------------------------------------------------------------------ traffic
KERNEL_SOURCES = ["paper_1801_03690_gb300/csrc/mm_solver_body.cuh",
                  "paper_1801_03690_gb300/csrc/mm_internal.cuh"]
TRAFFIC = "profiles/k_solver_traffic.json"


def kernel_source_digest():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record(workload_name):
    """The ncu DRAM-traffic record of the solver kernel on this workload
    (profiles/k_solver_traffic.json, written from one capture of
    dram__bytes_read.sum + dram__bytes_write.sum), or None when there is
    none for this workload or the kernel sources changed since."""
    try:
        recs = json.load(open(os.path.join(ROOT, TRAFFIC)))
    except (OSError, ValueError):
        return None
    for r in recs.get("records", []):
        if r.get("workload") == workload_name and r.get("sources") == kernel_source_digest():
            return r
    return None


def _ncu_launches(csv_path):
    """Per-launch metrics of an ncu --csv --print-units base log: a list of
    {"id", "kernel", metric: value} in launch order."""
    import csv
    rows = {}
    with open(csv_path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        lid = int(r["ID"])
        d = rows.setdefault(lid, {"id": lid, "kernel": r["Kernel Name"]})
        try:
            d[r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
        except ValueError:
            pass
    return [rows[k] for k in sorted(rows)]


def record_traffic(csv_path, line_path, command, out_path=None):
    """Writes profiles/k_solver_traffic.json from one ncu capture of the
    profiling command (`--workload polycrystal_medium --steps 1 --warmup 1
    --fp64-steps 1 --no-curve --no-cpu-baseline --no-e2e`) with
    dram__bytes_read.sum, dram__bytes_write.sum and gpu__time_duration.sum
    on every launch, and that run's own JSON line.  The solver launches of
    that command are, in order: warm-up (headline form, field 0), the
    untimed re-convergence of field 0 and the timed field 1 in the headline
    form, then the same two in plain FP64; the ratio DRAM bytes /
    algorithmic bytes of the timed launches is recorded for the captured
    workload and, scaled by the launch's algorithmic bytes, for the large
    polycrystal (same recipe and kernel; traffic grows with the bytes the
    counters imply)."""
    ls = [d for d in _ncu_launches(csv_path) if "k_solver" in d["kernel"]]
    if len(ls) != 5:
        raise SystemExit(f"expected 5 solver launches in {csv_path}, found {len(ls)}")
    line = None
    for ln in open(line_path):
        if ln.startswith("{"):
            line = json.loads(ln)
    if line is None:
        raise SystemExit(f"no JSON line in {line_path}")
    out = {"kernel_sources": KERNEL_SOURCES, "records": []}
    forms = (("headline", ls[2], line["timed_fields"]["per_step"][0]),
             ("plain_fp64", ls[4], line["plain_fp64"]["per_step"][0]))
    for form, d, st in forms:
        tr = d["dram__bytes_read.sum"] + d["dram__bytes_write.sum"]
        alg = st["alg_GB"] * 1e9
        ratio = tr / alg
        base = {"form": form, "sources": kernel_source_digest(), "ratio": ratio,
                "captured_on": "polycrystal_medium", "dram_bytes_read": d["dram__bytes_read.sum"],
                "dram_bytes_write": d["dram__bytes_write.sum"], "alg_bytes": alg,
                "gpu_time_ns": d.get("gpu__time_duration.sum"), "kernel": d["kernel"],
                "counters": {k: st[k] for k in ("nli", "evals", "mi", "mr", "li")},
                "command": command}
        if form == "headline":
            out["records"].append(dict(base, workload="polycrystal_medium",
                                       note="measured on this workload's timed launch"))
            out["records"].append(dict(base, workload="large_polycrystal",
                                       note="ratio from the 3.2 M-unknown medium case of the same recipe, "
                                            "scaled to the full launch by its algorithmic bytes"))
        else:
            out["records"].append(dict(base, workload="polycrystal_medium/plain_fp64",
                                       note="plain FP64 form, measured on this workload's timed launch"))
    with open(out_path or os.path.join(ROOT, TRAFFIC), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    for r in out["records"]:
        print(f"{r['workload']}: traffic {r['dram_bytes_read'] + r['dram_bytes_write']:.4g} B, "
              f"algorithmic {r['alg_bytes']:.4g} B, ratio {r['ratio']:.3f}")


# ------------------------------------------------------------------ ranks
class Ranks:
    """Replicas only: every rank solves its own copy of the workload; the
    only collectives are the timing barrier and the max/sum of the scalar
    results over ranks."""

    def __init__(self, world, device):
        self.world = world
        self.device = device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def _reduce(self, x, op):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], device=self.device, dtype=torch.float64)
        dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.MAX if self.world > 1 else None)

    def sum(self, x):
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.SUM if self.world > 1 else None)


# ------------------------------------------------------------------ oracle
def oracle_sample(name, first_field, n_iter, sample=True, warm_iter=0):
    """The CPU oracle as it stands, on the reduced-resolution sample of the
    workload's recipe (workload(name, sample=True)): assembly, then
    Algorithm 4 with the potential solved by Algorithm 1 (the same algorithm
    as the GPU's plain FP64 form) from m0 at field index first_field:
    warm_iter untimed NCG iterations, then exactly n_iter timed ones,
    continuing into the next field indices whenever a field converges (a
    field left at the warm-up's iteration cap is resumed).  Returns a dict
    with the timed seconds (assembly and warm-up excluded), the timed
    counters and the sample's sizes."""
    from oracle import fem, energy, ncg
    wl = workload(name, sample=sample)
    t0 = time.perf_counter()
    P = fem.assemble_workload(wl)
    t_asm = time.perf_counter() - t0
    state = {"m": energy.normalize(wl.m0[P.mag_nodes]), "phi": None, "k": first_field}

    def run(budget, tot, fields):
        while budget > 0 and state["k"] < len(wl.fields):
            k = state["k"]
            r = ncg.minimize(P, state["m"], P.units.field_int(wl.fields[k]),
                             ncg.Params(jmax=4, poisson="cg", max_iter=budget), phi0=state["phi"])
            state["m"], state["phi"] = r.m, r.phi
            budget -= r.stats["nli"]
            for c in tot:
                tot[c] += r.stats[c]
            if not fields or fields[-1] != k:
                fields.append(k)
            if r.status != "max_iter" or r.stats["nli"] == 0:
                state["k"] = k + 1

    t0 = time.perf_counter()
    warm = {"nli": 0, "evals": 0, "mi": 0, "li": 0, "ls_extra": 0}
    run(warm_iter, warm, [])
    t_warm = time.perf_counter() - t0
    tot = {"nli": 0, "evals": 0, "mi": 0, "li": 0, "ls_extra": 0}
    fields = []
    t0 = time.perf_counter()
    run(n_iter, tot, fields)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "assembly_s": t_asm, **tot, "fields": fields, "sample": wl.name,
            "n_phi": P.n_phi, "n_mag": P.n_mag, "warm_iter": warm["nli"], "warm_s": t_warm}


def oracle_leg(name, first_field, n_iter, threads, warm_iter=0):
    """oracle_sample in a child process whose BLAS / OpenMP pools have
    `threads` threads (numpy reads the setting at import)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg", "--workload", name,
                        "--oracle-first-field", str(first_field), "--oracle-iters", str(n_iter),
                        "--oracle-warm-iters", str(warm_iter)],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle leg failed:\n" + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["threads"] = threads
    return out


def oracle_baseline_entry(o, full=None):
    """cpu_baseline object of one oracle leg; with full = (n_phi, potential
    steps per NCG iteration of the GPU's plain FP64 form at full size), an
    estimate of the oracle at full size scaled by unknowns x potential steps
    per iteration (labelled extrapolated)."""
    v = o["nli"] / o["seconds"]
    e = {"value": v, "unit": UNIT, "cores": o["threads"], "kind": "oracle",
         "sample": (f"oracle Algorithm 4 (Jacobi-CG potential solve) on {o['sample']} (the same recipe at reduced "
                    f"resolution: {o['n_phi']} potential unknowns, {o['n_mag']} magnetic nodes) from m0"
                    + (f", after {o['warm_iter']} untimed warm-up iterations," if o.get("warm_iter") else "")
                    + f" at field indices {o['fields']}, {o['nli']} NCG iterations, {o['evals']} evaluations, "
                    f"{o['mi']} potential steps, {o['seconds']:.1f} s; assembly ({o['assembly_s']:.1f} s) excluded")}
    if full and o["nli"] and o["mi"]:
        n_phi_full, mi_per_it_full = full
        scale = (n_phi_full / o["n_phi"]) * (mi_per_it_full / (o["mi"] / o["nli"]))
        e["extrapolated_full_size"] = {"value": v / scale, "unit": UNIT,
                                       "how": "sample time per iteration x (full/sample unknowns) x (full/sample "
                                              "potential steps per iteration; full = the GPU plain FP64 form's "
                                              "counts on the same fields): extrapolated, not measured"}
    return e


# ------------------------------------------------------------------ oracle plan
def oracle_plan_leg(kind, name):
    """One leg of the CPU-baseline plan, run in this process (the caller
    sets its thread count): 'curve' = the oracle's whole demagnetisation
    curve of the workload (Sec. 3.1 field loop, Algorithm 4 per field);
    'iters' = 5 NCG iterations at full size from field index 5 (the first
    field the GPU bench times), continuing into the next fields;
    'sample' = the same on the workload's reduced-resolution sample;
    'platelets' = 5 iterations from m0 at the first field on each of the
    first 4 platelets of the seeded batch."""
    from oracle import fem, curve, ncg, energy
    prm = ncg.Params(jmax=4, poisson="cg")
    if kind == "curve":
        wl = workload(name)
        t0 = time.perf_counter()
        P = fem.assemble_workload(wl)
        t_asm = time.perf_counter() - t0
        t0 = time.perf_counter()
        r = curve.demag_curve(P, wl.fields, wl.m0, prm)
        dt = time.perf_counter() - t0
        recs = r["records"]
        return {"kind": kind, "workload": wl.name, "seconds": dt, "assembly_s": t_asm,
                "fields": len(recs), "nli": int(sum(x["nli"] for x in recs)),
                "evals": int(sum(x["evals"] for x in recs)), "mi": int(sum(x["mi"] for x in recs)),
                "Hc_T": r["Hc_T"], "n_phi": P.n_phi, "n_mag": P.n_mag}
    if kind in ("iters", "sample"):
        o = oracle_sample(name, 5, 5, sample=(kind == "sample"))
        return dict(o, kind=kind, workload=o["sample"])
    if kind == "platelets":
        import synth
        out = []
        for wl in synth.platelet_batch(64)[:4]:
            P = fem.assemble_workload(wl)
            m = energy.normalize(wl.m0[P.mag_nodes])
            t0 = time.perf_counter()
            r = ncg.minimize(P, m, P.units.field_int(wl.fields[0]), ncg.Params(jmax=4, poisson="cg", max_iter=5))
            out.append({"platelet": wl.name, "n_mag": P.n_mag, "n_phi": P.n_phi, "nli": r.stats["nli"],
                        "seconds": time.perf_counter() - t0})
        return {"kind": kind, "platelets": out}
    raise ValueError(kind)


def oracle_plan_mode(args):
    """The CPU-baseline plan: every leg once single-threaded and once with
    the BLAS / OpenMP pools at the core count, in child processes.  CPU
    only; prints one JSON object per leg and a summary line."""
    legs = [("curve", "soft_cube"), ("iters", "hard_cube"), ("sample", "polycrystal"),
            ("sample", "large_polycrystal"), ("platelets", "platelets")]
    if args.plan_legs:
        want = set(args.plan_legs.split(","))
        legs = [l for l in legs if f"{l[0]}:{l[1]}" in want]
    cores = os.cpu_count() or 1
    res = []
    for kind, name in legs:
        for threads in sorted({1, cores}):
            env = dict(os.environ)
            for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
                env[v] = str(threads)
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-plan-leg", kind, name],
                               capture_output=True, text=True, env=env, cwd=ROOT)
            if r.returncode != 0:
                raise RuntimeError("oracle plan leg failed:\n" + r.stderr[-2000:])
            o = json.loads(r.stdout.strip().splitlines()[-1])
            o["threads"] = threads
            print(json.dumps(o), flush=True)
            res.append(o)
    import platform
    print(json.dumps({"mode": "oracle_plan", "host": platform.machine(), "cores": cores, "legs": len(res)}))
    return 0


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_polycrystal", choices=WORKLOADS)
    ap.add_argument("--fp64-steps", type=int, default=8,
                    help="timed field steps of the plain FP64 comparison (a prefix of the timed steps)")
    ap.add_argument("--fp64-slice", type=int, default=200,
                    help="curve mode: iterations of the switching step timed in plain FP64 for the extrapolation")
    ap.add_argument("--jacobi", action="store_true", help="also time the Jacobi-preconditioned precision form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-curve", action="store_true", help="skip the full hard-cube curves")
    ap.add_argument("--mode", default="steps",
                    choices=["steps", "curve", "batch", "scaling", "sp3", "mlp", "oracle_plan"],
                    help="steps: the timed field steps (default line); curve: full demagnetisation "
                         "curves of the plain FP64, precision and precision + learned forms; "
                         "batch: the batched platelet workload; scaling: field steps of the hard "
                         "cube at several resolutions; oracle_plan: the CPU oracle's timing plan "
                         "(CPU only)")
    ap.add_argument("--n-platelets", type=int, default=64)
    ap.add_argument("--sp3-edges", default="8.2,8.4,8.6,8.8", help="sp3 mode: cube edges in exchange lengths")
    ap.add_argument("--sp3-n", type=int, default=24, help="sp3 mode: voxels per cube edge")
    ap.add_argument("--sp3-jmax", type=int, default=12, help="sp3 mode: j_max (Table 3's best: 12)")
    ap.add_argument("--sp3-box", type=float, default=8.0, help="sp3 mode: air box edge / cube edge")
    ap.add_argument("--mlp-rows", type=int, default=3375000, help="mlp mode: rows per forward pass")
    ap.add_argument("--forms", default="plain_fp64,precision,precision_multigrid,precision_learned")
    ap.add_argument("--theta-max", type=float, default=0.1,
                    help="curve mode: line-search cap on the largest nodal step (the paper's reading: 0.1)")
    ap.add_argument("--max-change", type=float, default=0.02,
                    help="warm start: cap on the largest predicted nodal change")
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="solver kernel instantiation / grid (0 = default)")
    ap.add_argument("--oracle-leg", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-first-field", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-iters", type=int, default=5, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-warm-iters", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-plan-leg", nargs=2, metavar=("KIND", "WORKLOAD"), help=argparse.SUPPRESS)
    ap.add_argument("--plan-legs", default="", help="oracle_plan mode: kind:workload legs to run (default all)")
    ap.add_argument("--record-traffic", nargs=3, metavar=("NCU_CSV", "JSON_LINE", "COMMAND"),
                    help="write profiles/k_solver_traffic.json from an ncu capture of the profiling command "
                         "(no GPU needed)")
    args = ap.parse_args()
    K, W = args.steps, max(args.warmup, 0)

    if args.record_traffic:
        record_traffic(*args.record_traffic)
        return 0
    if args.oracle_plan_leg:
        print(json.dumps(oracle_plan_leg(*args.oracle_plan_leg)))
        return 0
    if args.mode == "oracle_plan":
        return oracle_plan_mode(args)
    if args.oracle_leg:
        print(json.dumps(oracle_sample(args.workload, args.oracle_first_field, args.oracle_iters,
                                       warm_iter=args.oracle_warm_iters)))
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the oracle (no reference implementation exists: the reference is
        # the paper's text), timed on the host cores: W untimed NCG
        # iterations, then exactly K timed ones; one step = one NCG
        # iteration (the metric's unit)
        if rank != 0:
            return 0
        cores = os.cpu_count() or 1
        o = oracle_leg(args.workload, W, K, cores, warm_iter=W)
        v = o["nli"] / o["seconds"]
        cb = oracle_baseline_entry(o)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": o["nli"], "warmup": o["warm_iter"],
                "ms_per_step": 1000.0 * o["seconds"] / max(o["nli"], 1),
                "step": "one NCG iteration of the oracle", "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(workload_desc(args.workload, workload(args.workload, sample=True)),
                               sample_of=args.workload),
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    from paper_1801_03690_gb300 import Magnet, coercive_field

    if args.mode == "curve":
        return curve_mode(args, rank, local_rank)
    if args.mode == "batch":
        return batch_mode(args, rank, local_rank)
    if args.mode == "scaling":
        return scaling_mode(args, rank, local_rank)
    if args.mode == "sp3":
        return sp3_mode(args, rank, local_rank)
    if args.mode == "mlp":
        return mlp_mode(args, rank, local_rank)

    t0 = time.perf_counter()
    wl = workload(args.workload)
    t_gen = time.perf_counter() - t0
    fields = wl.fields
    if W < 1 or W + K > len(fields):
        raise SystemExit(f"need --warmup >= 1 and --warmup + --steps <= {len(fields)} field steps")
    mag = Magnet(device=local_rank, blocks_per_sm=args.blocks_per_sm)
    t0 = time.perf_counter()
    mag.upload_workload(wl)
    t_up = time.perf_counter() - t0
    sz = model_sizes(mag)
    stream = torch.cuda.ExternalStream(mag.stream, device=torch.device("cuda", local_rank))
    ranks = Ranks(world, torch.device("cuda", local_rank))
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum
    amg = mag.amg_info()

    # warm-up: W field steps from m0 in the headline form; every timed form
    # then starts from this state, re-converging the last warm-up field in
    # its own form (untimed) so that its potential is its own
    head = form_params(2)
    mag.set_magnetization(wl.m0)
    for k in range(W):
        mag.set_field(fields[k])
        mag.minimize(head)
    m_w = mag.get_magnetization()

    def run_form(prm, n):
        lv = amg if prm.amg else None
        mag.set_magnetization(m_w)
        mag.set_field(fields[W - 1])
        mag.minimize(prm)
        clocks = ClockSampler(local_rank)
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        nli, kern_ms, nbytes, per_step = 0, 0.0, 0, []
        for k in range(W, W + n):
            mag.set_field(fields[k])
            mag.minimize_async(prm)
            st = mag.get_stats()
            ms = mag.last_kernel_ms()
            b = alg_bytes(st, sz, lv, prm.precision)
            kern_ms += ms
            nbytes += b
            nli += st["nli"]
            per_step.append({"field_T": float(fields[k][2]), "status": st["status"], "nli": st["nli"],
                             "evals": st["evals"], "mi": st["mi"], "mr": st["mr"], "li": st["li"],
                             "ls_extra": st["ls_extra"], "F_J": st["F"], "Mz": st["M"][2], "kernel_ms": ms,
                             "alg_GB": b / 1e9})
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ck = clocks.stop()
        t_ms = max_over_ranks(ev0.elapsed_time(ev1))
        nli_all = sum_over_ranks(nli)
        return {"prm": prm, "value": nli_all / (t_ms / 1000.0), "t_ms": t_ms, "nli": nli_all, "n": n,
                "kern_ms": kern_ms, "bytes": nbytes, "per_step": per_step, "clocks": ck,
                "m": mag.get_magnetization(), "F": per_step[-1]["F_J"]}

    x1 = run_form(head, K)
    n64 = max(1, min(K, args.fp64_steps))
    fp64 = run_form(form_params(0), n64)
    jac = run_form(form_params(1), n64) if args.jacobi else None

    # ---- end to end through the public API with host buffers (headline form)
    e2e = None
    if not args.no_e2e:
        prm = head
        m_host = torch.empty((wl.mesh.n_nodes, 3), dtype=torch.float64).pin_memory()
        m_host.copy_(torch.from_numpy(m_w))
        mag.set_magnetization(m_host.numpy())
        mag.set_field(fields[W - 1])
        mag.minimize(prm)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nli_e = 0
        for k in range(W, W + K):
            mag.set_magnetization(m_host.numpy())
            mag.set_field(fields[k])
            st = mag.minimize(prm)
            m_host.copy_(torch.from_numpy(mag.get_magnetization()))
            nli_e += st["nli"]
        torch.cuda.synchronize()
        barrier()
        te = max_over_ranks(time.perf_counter() - t0)
        mbytes = wl.mesh.n_nodes * 3 * 8
        e2e = {"value": sum_over_ranks(nli_e) / te, "unit": UNIT, "h2d_bytes_per_step": mbytes + 24,
               "d2h_bytes_per_step": mbytes + 144, "form": "headline form (multigrid precision form)"}
    mag.close()

    # ---- full demagnetisation curves of the 80 nm hard cube in both forms
    curves = None
    if not args.no_curve:
        import synth
        hc_wl = synth.hard_cube()
        cm = Magnet(device=local_rank, blocks_per_sm=args.blocks_per_sm)
        cm.upload_workload(hc_wl)
        curves = {"workload": f"{hc_wl.name}: 80 nm Nd2Fe14B cube, {len(hc_wl.fields)} fields 0 to -8 T",
                  "sizes": cm.sizes()}
        for name, prm in (("precision_multigrid", form_params(2)), ("plain_fp64", form_params(0))):
            cm.set_magnetization(hc_wl.m0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sts = cm.demag_curve(hc_wl.fields, prm)
            torch.cuda.synchronize()
            wall = max_over_ranks(time.perf_counter() - t0)
            M = np.array([s["M"] for s in sts])
            curves[name] = {"wall_s": wall, "nli": int(sum(s["nli"] for s in sts)),
                            "evals": int(sum(s["evals"] for s in sts)), "mi": int(sum(s["mi"] for s in sts)),
                            "Hc_T": coercive_field(hc_wl.fields, M),
                            "statuses": sorted(set(s["status"] for s in sts)), "M": M[:, 2].tolist()}
        a, b = curves["precision_multigrid"], curves["plain_fp64"]
        curves["speedup_vs_plain_fp64"] = b["wall_s"] / a["wall_s"]
        curves["Hc_rel_diff"] = (abs(a["Hc_T"] - b["Hc_T"]) / b["Hc_T"]) if a["Hc_T"] and b["Hc_T"] else None
        curves["max_abs_dMz"] = float(np.max(np.abs(np.array(a["M"]) - np.array(b["M"]))))
        for f in ("precision_multigrid", "plain_fp64"):
            curves[f].pop("M")
        cm.close()

    if rank != 0:
        return 0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = x1["bytes"] / (x1["kern_ms"] / 1000.0) / 1e9
    ach64 = fp64["bytes"] / (fp64["kern_ms"] / 1000.0) / 1e9
    tr = traffic_record(args.workload)
    # the headline form on exactly the fields of the FP64 comparison
    x1_sub_ms = sum(p["kernel_ms"] for p in x1["per_step"][:n64])
    x1_sub_nli = sum(p["nli"] for p in x1["per_step"][:n64])
    fp64_ms = sum(p["kernel_ms"] for p in fp64["per_step"])
    line = {
        "metric": METRIC, "value": x1["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": x1["t_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32+fp64", "data": "synthetic (seeded generators in synth/)",
        "config": workload_desc(args.workload, wl, sz),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": (tr["ratio"] * x1["bytes"] / K) if tr else None,
                     "traffic_source": (f"{TRAFFIC}: DRAM bytes / algorithmic bytes = {tr['ratio']:.3f} from one "
                                        f"ncu capture ({tr['note']})") if tr else None,
                     "kernel": "k_solver", "peak_source": peak_src,
                     "alg_bytes_per_launch": x1["bytes"] / K, "kernel_ms_per_launch": x1["kern_ms"] / K},
        "plain_fp64": {"value": fp64["value"], "unit": UNIT, "ms_per_step": fp64["t_ms"] / n64,
                       "fields_timed": n64, "dtype": "f64", "roofline_frac": ach64 / hbm, "achieved_gbs": ach64,
                       "per_step": fp64["per_step"]},
        "vs_plain_fp64_same_fields": {
            "fields": [W, W + n64 - 1],
            "headline_nli_per_s": x1_sub_nli / (x1_sub_ms / 1000.0),
            "plain_fp64_nli_per_s": fp64["nli"] / (fp64_ms / 1000.0),
            "kernel_time_ratio": fp64_ms / x1_sub_ms,
            "final_energy_rel_diff": abs(x1["per_step"][n64 - 1]["F_J"] - fp64["F"]) / abs(fp64["F"]),
            "final_Mz_abs_diff": abs(x1["per_step"][n64 - 1]["Mz"] - fp64["per_step"][-1]["Mz"])},
        "multigrid": {"levels": amg, "inner_tol": x1["prm"].inner_tol},
        "timed_fields": {"fields": [W, W + K - 1], "wall_s": x1["t_ms"] / 1000.0, "per_step": x1["per_step"]},
        "setup_s": {"generate": t_gen, "upload_and_assembly": t_up},
        "gpu_launches": 2 * K,
        "gpu_launches_note": "per timed field step: k_set_field and one persistent k_solver launch",
    }
    line["config"]["precision"] = ("headline: FP32 potential solve preconditioned by the multigrid V-cycle + FP64 "
                                   "refinement, potential tolerance tied to t1 (loosened only while the last energy "
                                   "decrease exceeds 100x the t1 threshold), FP64 energy/gradient/line search/NCG; "
                                   "plain_fp64: FP64 throughout, Jacobi-preconditioned potential CG to 1e-10")
    if jac:
        achj = jac["bytes"] / (jac["kern_ms"] / 1000.0) / 1e9
        line["precision_jacobi"] = {"value": jac["value"], "unit": UNIT, "ms_per_step": jac["t_ms"] / n64,
                                    "fields_timed": n64, "roofline_frac": achj / hbm, "per_step": jac["per_step"]}
    if curves:
        line["demag_curve"] = curves
    if e2e:
        line["e2e"] = e2e
    ck = merge_clocks([x1["clocks"], fp64["clocks"], jac["clocks"] if jac else None])
    if ck:
        line["clocks"] = ck
    if world == 1 and not args.no_cpu_baseline:
        full = (sz["n_phi"], sum(p["mi"] for p in fp64["per_step"]) / max(1, fp64["nli"]))
        legs = [oracle_leg(args.workload, W, 5, 1), oracle_leg(args.workload, W, 5, os.cpu_count() or 1)]
        best = max(legs, key=lambda o: o["nli"] / o["seconds"])
        line["cpu_baseline"] = oracle_baseline_entry(best, full)
        line["cpu_baseline"]["legs"] = [oracle_baseline_entry(o, full) for o in legs]
    print(json.dumps(line))
    return 0


def curve_mode(args, rank, local_rank):
    """Full demagnetisation curves of one workload, in the forms listed by
    --forms: plain_fp64, precision (Jacobi), precision_multigrid, and
    precision_learned (the multigrid precision form with the learned warm
    start, the network trained on the method's own trajectories of the
    hard-cube and polycrystal recipes at reduced resolution, i.e. of other
    meshes).  plain_fp64_extrapolated: plain FP64 timed on a slice of the
    curve -- the warm-up-free reversible field steps after the first and the
    first --fp64-slice iterations of the switching step, from the multigrid
    form's states there -- and extrapolated to the whole curve with the
    multigrid form's per-step iteration counts (both forms take the same
    iterations; labelled extrapolated).  Reports wall time, NCG iterations,
    potential steps and coercive field (mm_coercive_field)."""
    import torch
    import synth
    from paper_1801_03690_gb300 import Magnet, Params, MLP, warmstart, coercive_field
    wl = workload(args.workload)
    fields = wl.fields
    mag = Magnet(device=local_rank, blocks_per_sm=args.blocks_per_sm)
    mag.upload_workload(wl)
    sz = mag.sizes()
    out = {}
    forms = args.forms.split(",")
    states = {}

    def run(name, prm, net=None, scales=None, keep_states=False):
        if name not in forms:
            return
        mag.set_magnetization(wl.m0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sts, kms = [], []
        for k, b in enumerate(fields):
            if keep_states:
                states[k] = mag.get_magnetization()
            if net is not None and k > 0:
                warmstart.warmstart_apply(mag, net, b, scales[0], scales[1], args.max_change)
            mag.set_field(b)
            sts.append(mag.minimize(prm))
            kms.append(mag.last_kernel_ms())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        M = np.array([s["M"] for s in sts])
        out[name] = {"wall_s": wall, "kernel_s": sum(kms) / 1e3, "nli": int(sum(s["nli"] for s in sts)),
                     "evals": int(sum(s["evals"] for s in sts)), "mi": int(sum(s["mi"] for s in sts)),
                     "Hc_T": coercive_field(fields, M),
                     "statuses": sorted(set(s["status"] for s in sts)),
                     "nli_per_step": [int(s["nli"]) for s in sts], "kernel_ms_per_step": kms,
                     "Mz": M[:, 2].tolist()}

    run("plain_fp64", Params(precision=0, theta_max=args.theta_max))
    run("precision", Params(precision=1, theta_max=args.theta_max))
    mg = form_params(2, theta_max=args.theta_max)       # the headline form (schedule included)
    run("precision_multigrid", mg, keep_states="plain_fp64_extrapolated" in forms)
    if "plain_fp64_extrapolated" in forms and "precision_multigrid" in out:
        ref = out["precision_multigrid"]
        nli = np.array(ref["nli_per_step"])
        ksw = int(np.argmax(nli))                       # the switching step
        fp = Params(precision=0, theta_max=args.theta_max)
        rev = [k for k in range(1, len(fields)) if k != ksw][:args.fp64_steps]
        t_rev, n_rev = 0.0, 0
        for k in rev:
            mag.set_magnetization(states[k])
            mag.set_field(fields[k - 1])
            mag.minimize(fp)                            # the previous minimum in this form (untimed)
            mag.set_field(fields[k])
            st = mag.minimize(fp)
            t_rev += mag.last_kernel_ms() / 1e3
            n_rev += st["nli"]
        mag.set_magnetization(states[ksw])
        mag.set_field(fields[ksw - 1])
        mag.minimize(fp)
        mag.set_field(fields[ksw])
        st = mag.minimize(Params(precision=0, theta_max=args.theta_max, max_iter=args.fp64_slice))
        t_sw, n_sw = mag.last_kernel_ms() / 1e3, st["nli"]
        per_rev, per_sw = t_rev / max(n_rev, 1), t_sw / max(n_sw, 1)
        est = float(np.sum(np.where(np.arange(len(nli)) == ksw, nli * per_sw, nli * per_rev)))
        out["plain_fp64_extrapolated"] = {
            "kernel_s": est, "measured": {"reversible_fields": rev, "reversible_nli": n_rev, "reversible_s": t_rev,
                                          "switching_field": ksw, "switching_slice_nli": n_sw,
                                          "switching_slice_s": t_sw},
            "how": "extrapolated, not measured: sum over the multigrid form's field steps of its NCG iterations x "
                   "the plain FP64 form's measured seconds per iteration (reversible steps; the switching step "
                   "from its measured slice)",
            "speedup_of_precision_multigrid": est / ref["kernel_s"]}
    if "precision_learned" in forms:
        t0 = time.perf_counter()
        net = MLP(device=local_rank, seed=11)
        Xs, Ts = [], []
        prm_t = form_params(2)
        trained_on = []
        for twl in (synth.hard_cube(n_mag=24, seed=12), synth.polycrystal_cube(n_mag=38, seed=13)):
            tm = Magnet(device=local_rank)
            tm.upload_workload(twl)
            X, T, _ = warmstart.collect(tm, net, twl.m0, twl.fields, tm.sizes()["n_mag"], prm_t)
            tm.close()
            Xs.append(X)
            Ts.append(T)
            trained_on.append(f"{twl.name} ({len(twl.fields)} fields, {X.shape[0]} node samples)")
        X, T = torch.cat(Xs), torch.cat(Ts)
        s_m, s_p, losses = warmstart.train(net, X, T, steps=1500, batch=16384, lr=2e-3, log_every=500)
        train_s = time.perf_counter() - t0
        run("precision_learned", mg, net=net, scales=(s_m, s_p))
        out["precision_learned"]["training"] = {"samples": int(X.shape[0]), "steps": 1500, "seconds": train_s,
                                                "losses": losses, "trained_on": trained_on,
                                                "max_change": args.max_change}
    ref = out.get("plain_fp64") or out.get("precision_multigrid") or out.get("precision")
    for k in ("precision", "precision_multigrid", "precision_learned"):
        if k not in out or out[k] is ref:
            continue
        o = out[k]
        o["speedup_vs_reference_form"] = ref["wall_s"] / o["wall_s"]
        if o["Hc_T"] is not None and ref["Hc_T"] is not None:
            o["Hc_rel_diff"] = abs(o["Hc_T"] - ref["Hc_T"]) / ref["Hc_T"]
        o["max_abs_dMz"] = float(np.max(np.abs(np.array(o["Mz"]) - np.array(ref["Mz"]))))
    if rank == 0:
        print(json.dumps({"mode": "curve", "workload": wl.name, "sizes": sz, "n_fields": len(fields),
                          "reference_form": [k for k in out if out[k] is ref], "forms": out}))
    mag.close()
    return 0


def mlp_mode(args, rank, local_rank):
    """The warm-start network alone: forward passes over --mlp-rows rows
    (default: the large polycrystal's 3,375,000 magnetic nodes) on the
    tcgen05 path and on the mma.sync path, and Adam training steps on
    16,384-row mini-batches; host wall time over repeated calls bracketed by
    device synchronisations (the calls synchronise the library's stream
    themselves), and the tensor work per pass
    (2 x 128 x (16 + 128 + 128 + 16) multiply-adds per row, the last layer
    padded to N = 16 on tcgen05)."""
    import torch
    from paper_1801_03690_gb300 import MLP
    n = args.mlp_rows
    net = MLP(device=local_rank, seed=1)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    X = torch.randn((n, 16), device="cuda", generator=g)
    out = {"mode": "mlp", "rows": n}
    flop_row = 2 * 128 * (16 + 128 + 128 + 16)
    for path, name in ((0, "tcgen05"), (1, "mma.sync")):
        net.set_tensor_path(path)
        for _ in range(3):
            net.forward(X)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 10
        for _ in range(reps):
            Y = net.forward(X)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        out[name] = {"ms_per_forward": dt * 1e3, "rows_per_s": n / dt, "tflops": flop_row * n / dt / 1e12,
                     "checksum": float(Y.double().abs().sum().item())}
    net.set_tensor_path(0)
    T = torch.randn((16384, 4), device="cuda", generator=g)
    xb = X[:16384].contiguous()
    for _ in range(3):
        net.train_step(xb, T, 1e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(50):
        net.train_step(xb, T, 1e-3)
    torch.cuda.synchronize()
    out["train_step_ms"] = (time.perf_counter() - t0) / 50 * 1e3
    if rank == 0:
        print(json.dumps(out))
    net.close()
    return 0


def sp3_mode(args, rank, local_rank):
    """muMAG standard problem 3 (Sec. 3.3): flower (from saturation) and
    vortex (from a sharp two-domain state) relaxed at zero field with
    tau_F = 1e-12 for cube edges L around the single-domain limit; reduced
    energies e = E / (Km L^3) and the edge where they cross, by linear
    interpolation of e_flower - e_vortex."""
    import torch
    import synth
    from paper_1801_03690_gb300 import Magnet, Params
    Ls = [float(x) for x in args.sp3_edges.split(",")]
    prm = Params(tau_F=1e-12, jmax=args.sp3_jmax, poisson_tol=1e-12, max_iter=100000)
    rows = []
    for L in Ls:
        row = {"L_lex": L}
        for start in ("flower", "vortex"):
            wl = synth.sp3_cube(L, n_mag=args.sp3_n, start=start, box_factor=args.sp3_box)
            mag = Magnet(device=local_rank)
            mag.upload_workload(wl)
            mag.set_magnetization(wl.m0)
            t0 = time.perf_counter()
            st = mag.minimize(prm)
            dt = time.perf_counter() - t0
            km, Lm = wl.meta["Km"], wl.meta["L"]
            row[start] = {"e": st["F"] / (km * Lm ** 3), "terms": [t / (km * Lm ** 3) for t in st["terms"]],
                          "M": st["M"], "status": st["status"], "nli": st["nli"], "evals": st["evals"],
                          "li": st["li"], "mi": st["mi"], "seconds": dt}
            mag.close()
        row["de"] = row["flower"]["e"] - row["vortex"]["e"]
        rows.append(row)
        if rank == 0:
            print(json.dumps(row), flush=True)
    cross = None
    for a, b in zip(rows[:-1], rows[1:]):
        if a["de"] * b["de"] < 0:
            cross = a["L_lex"] + a["de"] / (a["de"] - b["de"]) * (b["L_lex"] - a["L_lex"])
            break
    if rank == 0:
        print(json.dumps({"mode": "sp3", "n_mag": args.sp3_n, "jmax": args.sp3_jmax, "box": args.sp3_box,
                          "crossover_L_lex": cross,
                          "paper": 8.52, "rows": rows}))
    return 0


def scaling_mode(args, rank, local_rank):
    """Size sweep at fixed physics (the 80 nm hard cube at several
    resolutions, air box 2x): NCG iterations and potential CG steps per field
    step, throughput, achieved bandwidth (field steps 3-7), for the precision
    form with the Jacobi and with the multigrid potential preconditioner."""
    import torch
    import synth
    from paper_1801_03690_gb300 import Magnet
    rows = []
    for n, form in [(n, f) for n in (16, 24, 32, 40, 48, 56, 64) for f in (1, 2)]:
        prm = form_params(form)
        wl = synth.hard_cube(n_mag=n)
        mag = Magnet(device=local_rank)
        mag.upload_workload(wl)
        sz = model_sizes(mag)
        lv = mag.amg_info() if prm.amg else None
        mag.set_magnetization(wl.m0)
        for k in range(3):
            mag.set_field(wl.fields[k])
            mag.minimize(prm)
        torch.cuda.synchronize()
        nli = mi = ev = 0
        nbytes, kms = 0, 0.0
        t0 = time.perf_counter()
        for k in range(3, 8):
            mag.set_field(wl.fields[k])
            mag.minimize_async(prm)
            st = mag.get_stats()
            kms += mag.last_kernel_ms()
            nbytes += alg_bytes(st, sz, lv, prm.precision)
            nli += st["nli"]
            mi += st["mi"]
            ev += st["evals"]
        dt = time.perf_counter() - t0
        rows.append({"form": "multigrid" if prm.amg else "jacobi",
                     "levels": [lvl["rows"] for lvl in lv] if lv else None,
                     "n_mag_voxels": n, "n_mag": sz["n_mag"], "n_phi": sz["n_phi"],
                     "nli_per_step": nli / 5, "cg_steps_per_eval": mi / ev, "NCG_it_per_s": nli / dt,
                     "ms_per_step": 1000 * dt / 5, "achieved_GBs": nbytes / (kms / 1000) / 1e9})
        mag.close()
    if rank == 0:
        print(json.dumps({"mode": "scaling", "workload": "hard_cube (80 nm, box 2x)", "rows": rows}))
    return 0


def batch_mode(args, rank, local_rank):
    """The batched sensor workload: n permalloy platelets of 5k-80k magnetic
    nodes, minimised at one field in one persistent launch (after the
    autotuner picked the kernel instantiation, team split and tile shape),
    against the
    same problems minimised one after the other, in the precision form with
    the Jacobi and with the multigrid potential preconditioner."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import synth
    from paper_1801_03690_gb300 import Magnet, Batch
    wls = synth.platelet_batch(args.n_platelets)

    def make(wl):
        m = Magnet(device=local_rank)
        m.upload_workload(wl)
        return m

    with ThreadPoolExecutor(8) as ex:
        mags = list(ex.map(make, wls))
    sizes = [m.sizes() for m in mags]

    def reset(k):
        for m, wl in zip(mags, wls):
            m.set_magnetization(wl.m0)
            m.set_field(wl.fields[k])

    def run(prm):
        res = {}
        reset(0)
        batch = Batch(mags)
        bps, gamma, ms = batch.autotune(prm)
        res["autotune"] = dict(batch.get_config(), trial_ms=ms)
        for k in (0, 1, 2):                               # warm-up field steps
            reset(k) if k == 0 else [m.set_field(wl.fields[k]) for m, wl in zip(mags, wls)]
            batch.minimize(prm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nli = 0
        for k in range(3, 3 + K):
            for m, wl in zip(mags, wls):
                m.set_field(wl.fields[k])
            sts = batch.minimize(prm)
            nli += sum(s["nli"] for s in sts)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        res["batched"] = {"nli": nli, "seconds": tb, "NCG_it_per_s": nli / tb}
        batch.close()
        # the same field steps one problem after the other
        reset(0)
        for k in (0, 1, 2):
            for m, wl in zip(mags, wls):
                m.set_field(wl.fields[k])
                m.minimize(prm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nli_s = 0
        for k in range(3, 3 + K):
            for m, wl in zip(mags, wls):
                m.set_field(wl.fields[k])
                nli_s += m.minimize(prm)["nli"]
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        res["sequential"] = {"nli": nli_s, "seconds": ts, "NCG_it_per_s": nli_s / ts}
        res["speedup"] = ts / tb
        return res

    K = 5
    res = {"precision_jacobi": run(form_params(1)), "precision_multigrid": run(form_params(2)),
           "with_hierarchy": int(sum(1 for m in mags if m.amg_levels()))}
    if rank == 0:
        print(json.dumps({"mode": "batch", "n": len(wls),
                          "n_mag_total": int(sum(s["n_mag"] for s in sizes)),
                          "n_phi_total": int(sum(s["n_phi"] for s in sizes)),
                          "n_mag_range": [int(min(s["n_mag"] for s in sizes)), int(max(s["n_mag"] for s in sizes))],
                          "field_steps_timed": K, **res}))
    for m in mags:
        m.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
