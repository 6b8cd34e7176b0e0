"""Benchmark: NCG iterations per second of the preconditioned NCG minimiser
over the field steps of a demagnetisation curve (Sec. 3.1, Algorithm 4).

Workload (default): an Nd2Fe14B cube, 80 nm edge, 48^3 voxels of 6 jittered
tetrahedra (117,649 magnetic nodes), easy axis 1 degree off z, in an air box
of twice the edge (97^3 lattice, 857,375 potential unknowns, 5.3M tets);
m0 = +z; field along -z from 0 to -8 T in 40 values.  One step = one field
step of the curve: set the field, minimise by Algorithm 4 until t1-t3 hold.

value: NCG iterations / s with everything resident on the device (summed
over ranks, max time over ranks).  e2e: the same metric through the public
API with host buffers: each step uploads m from pinned host memory, sets the
field, minimises and reads m and the stats back.

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

# the CPU oracle legs run on one host core: pin the BLAS / OpenMP pools
# before numpy is imported so that the reported core count is the real one
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NCG iters/s & demag-curve wall time vs plain FP64 GPU at equal energy tol"
UNIT = "NCG it/s"


def workload(name):
    import synth
    if name == "hard_cube":
        return synth.hard_cube()
    if name == "soft_cube":
        return synth.soft_cube()
    if name == "medium":
        return synth.hard_cube(n_mag=44)
    if name == "small":
        return synth.hard_cube(n_mag=12)
    if name == "polycrystal":
        return synth.polycrystal_cube()
    raise ValueError(name)


def workload_desc(name, wl, sizes=None):
    d = {"workload": f"{wl.name}: {name}", "n_nodes": wl.mesh.n_nodes, "n_tets": wl.mesh.n_tets,
         "fields": f"{len(wl.fields)} values from {wl.fields[0].tolist()} to {wl.fields[-1].tolist()} T",
         "precision": "plain FP64", "jmax": 4, "tau_F": 1e-10, "poisson_tol": 1e-10,
         "l2": "working set larger than L2 (no flush needed)"}
    if sizes:
        d.update(sizes)
    return d


# ------------------------------------------------------------ algorithmic bytes
def form_params(form):
    """Parameters of the three forms of a field step: 0 plain FP64
    (Jacobi-preconditioned potential solve), 1 precision form with Jacobi,
    2 precision form with the multigrid preconditioner (the headline)."""
    from paper_1801_03690_gb300 import Params
    if form == 0:
        return Params(jmax=4, tau_F=1e-10, poisson_tol=1e-10, precision=0)
    if form == 1:
        return Params(jmax=4, tau_F=1e-10, poisson_tol=1e-10, precision=1)
    return Params(jmax=4, tau_F=1e-10, poisson_tol=1e-10, precision=1, amg=1, inner_tol=1e-3)


def vcycle_bytes(amg):
    """Bytes of one multigrid V-cycle (levels l < L smoothed, L dense):
      down_l  8 nnz_A_l + 12 n_l + 8 nnz_U_l + 12 n_{l+1} (4 n_L at the last)
              (A and U^T val+col; x, b read, rpre written; b, x of l+1 written)
      dense   4 n_L^2 + 8 n_L
      up_l    8 nnz_U_l + 4 n_{l+1} + 16 n_l (U; y_{l+1}; b, rpre, diag^-1 -> y)"""
    L = len(amg) - 1
    tot = 4 * amg[L]["nnz_a"] + 8 * amg[L]["rows"]
    for l in range(L):
        n, nc = amg[l]["rows"], amg[l + 1]["rows"]
        tot += 8 * amg[l]["nnz_a"] + 12 * n + 8 * amg[l]["nnz_u"] + (4 if l + 1 == L else 12) * nc
        tot += 8 * amg[l]["nnz_u"] + 4 * nc + 16 * n
    return tot


def alg_bytes(st, sz, amg=None):
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
      inner step (li)       12 nnz_mag + 352 n_mag  (H product + update)
      per iteration (nli+1) 272 n_mag               (inner set-up + direction)
    """
    nphi, nm = sz["n_phi"], sz["n_mag"]
    nzp, nzm = sz["nnz_phi"], sz["nnz_mag"]
    per_pcg = 12 * nzp + 96 * nphi
    per_pcg32 = 8 * nzp + 52 * nphi          # FP32 step: val+col 8 B/nnz; 13 FP32 vector passes
    per_refine = 12 * nzp + 60 * nphi        # FP64 residual product + FP32 set-up
    per_eval = 12 * nzp + 64 * nzm + 48 * nphi + 208 * nm
    per_trial = 112 * nm
    per_inner = 12 * nzm + 352 * nm
    per_iter = 272 * nm
    mr = st.get("mr", 0)
    if amg:
        vc = vcycle_bytes(amg)
        per_pcg32 = 8 * nzp + 20 * nphi + 32 * nphi + vc
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


# ------------------------------------------------------------------ traffic
KERNEL_SOURCES = ["paper_1801_03690_gb300/csrc/mm_solver_body.cuh",
                  "paper_1801_03690_gb300/csrc/mm_internal.cuh"]
PROFILE = "profiles/k_solver_hard_cube.md"


def kernel_source_digest():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_ratio():
    """DRAM bytes / algorithmic bytes of the solver kernel from the last ncu
    capture summarised in profiles/ (a line 'traffic_ratio: R sources: D'),
    or None when the kernel sources changed since that capture."""
    try:
        for line in open(os.path.join(ROOT, PROFILE)):
            if line.startswith("traffic_ratio:"):
                f = line.split()
                if f[3] == kernel_source_digest():
                    return float(f[1])
    except (OSError, IndexError, ValueError):
        pass
    return None


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
def oracle_sample(wl, max_iter, warm_iter=0):
    """The CPU oracle as it stands: assemble, then Algorithm 4 at the first
    field from m0 with the potential solved by Algorithm 1 (the same
    algorithm as the GPU).  Returns (nli, seconds, description)."""
    from oracle import fem, energy, ncg
    P = fem.assemble_workload(wl)
    m = energy.normalize(wl.m0[P.mag_nodes])
    h = P.units.field_int(wl.fields[0])
    phi = None
    if warm_iter:
        r = ncg.minimize(P, m, h, ncg.Params(jmax=4, poisson="cg", max_iter=warm_iter))
        m, phi = r.m, r.phi
    t0 = time.perf_counter()
    r = ncg.minimize(P, m, h, ncg.Params(jmax=4, poisson="cg", max_iter=max_iter), phi0=phi)
    dt = time.perf_counter() - t0
    desc = (f"oracle Algorithm 4 at the first field of the same workload, {r.stats['nli']} NCG "
            f"iteration(s) incl. the initial evaluation ({r.stats['evals']} evaluations, "
            f"{r.stats['mi']} potential steps), assembly excluded")
    return r.stats["nli"], dt, desc


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hard_cube", choices=["hard_cube", "medium", "soft_cube", "small", "polycrystal"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mode", default="steps", choices=["steps", "curve", "batch", "scaling"],
                    help="steps: the timed field steps (default line); curve: full demagnetisation "
                         "curves of the plain FP64, precision and precision + learned forms; "
                         "batch: the batched platelet workload; scaling: field steps of the hard "
                         "cube at several resolutions")
    ap.add_argument("--n-platelets", type=int, default=64)
    ap.add_argument("--forms", default="plain_fp64,precision,precision_multigrid,precision_learned")
    ap.add_argument("--theta-max", type=float, default=0.1,
                    help="curve mode: line-search cap on the largest nodal step (the paper's reading: 0.1)")
    ap.add_argument("--max-change", type=float, default=0.02,
                    help="warm start: cap on the largest predicted nodal change")
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="solver kernel instantiation / grid (0 = default)")
    args = ap.parse_args()
    K, W = args.steps, max(args.warmup, 0)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        wl = workload(args.workload)
        nli, dt, desc = oracle_sample(wl, max_iter=K, warm_iter=W)
        v = nli / dt
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": K, "warmup": W, "ms_per_step": 1000.0 * dt / max(nli, 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_desc(args.workload, wl),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    from paper_1801_03690_gb300 import Magnet, Params

    if args.mode == "curve":
        return curve_mode(args, rank, local_rank)
    if args.mode == "batch":
        return batch_mode(args, rank, local_rank)
    if args.mode == "scaling":
        return scaling_mode(args, rank, local_rank)

    wl = workload(args.workload)
    fields = wl.fields
    if W + K > len(fields):
        raise SystemExit(f"--warmup + --steps must be <= {len(fields)} field steps")
    mag = Magnet(device=local_rank, blocks_per_sm=args.blocks_per_sm)
    mag.upload_workload(wl)
    sz = mag.sizes()
    stream = torch.cuda.ExternalStream(mag.stream, device=torch.device("cuda", local_rank))

    ranks = Ranks(world, torch.device("cuda", local_rank))
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum

    amg = mag.amg_info()

    def run_form(prm):
        """W untimed field steps from m0, then K timed field steps."""
        lv = amg if prm.amg else None
        mag.set_magnetization(wl.m0)
        for k in range(W):
            mag.set_field(fields[k])
            mag.minimize(prm)
        clocks = ClockSampler(local_rank)
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        nli, kern_ms, nbytes, per_step = 0, 0.0, 0, []
        for k in range(W, W + K):
            mag.set_field(fields[k])
            mag.minimize_async(prm)
            st = mag.get_stats()
            ms = mag.last_kernel_ms()
            kern_ms += ms
            nbytes += alg_bytes(st, sz, lv)
            nli += st["nli"]
            per_step.append({"field_T": float(fields[k][2]), "status": st["status"], "nli": st["nli"],
                             "evals": st["evals"], "mi": st["mi"], "mr": st["mr"], "li": st["li"],
                             "F_J": st["F"], "Mz": st["M"][2], "kernel_ms": ms})
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ck = clocks.stop()
        t_ms = max_over_ranks(ev0.elapsed_time(ev1))
        nli_all = sum_over_ranks(nli)
        return {"prm": prm, "value": nli_all / (t_ms / 1000.0), "t_ms": t_ms, "nli": nli_all,
                "kern_ms": kern_ms, "bytes": nbytes, "per_step": per_step, "clocks": ck,
                "m": mag.get_magnetization(), "F": per_step[-1]["F_J"]}

    fp64 = run_form(form_params(0))
    jac = run_form(form_params(1))
    x1 = run_form(form_params(2))

    # ---- end to end through the public API with host buffers (precision form)
    e2e = None
    if not args.no_e2e:
        prm = x1["prm"]
        m_host = torch.empty((wl.mesh.n_nodes, 3), dtype=torch.float64).pin_memory()
        m_host.copy_(torch.from_numpy(wl.m0))
        mag.set_magnetization(m_host.numpy())
        for k in range(W):
            mag.set_field(fields[k])
            mag.minimize(prm)
        m_host.copy_(torch.from_numpy(mag.get_magnetization()))
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
               "d2h_bytes_per_step": mbytes + 144, "form": "precision form (FP32 potential solve + FP64 refinement)"}

    if rank != 0:
        return 0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = x1["bytes"] / (x1["kern_ms"] / 1000.0) / 1e9
    ratio = traffic_ratio()
    ach64 = fp64["bytes"] / (fp64["kern_ms"] / 1000.0) / 1e9
    achj = jac["bytes"] / (jac["kern_ms"] / 1000.0) / 1e9
    dm = float(np.abs(x1["m"] - fp64["m"]).max())
    line = {
        "metric": METRIC, "value": x1["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": x1["t_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32+fp64", "data": "synthetic",
        "config": workload_desc(args.workload, wl, sz),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": (ratio * x1["bytes"] / K) if ratio else None, "kernel": "k_solver",
                     "peak_source": peak_src, "alg_bytes_per_launch": x1["bytes"] / K,
                     "kernel_ms_per_launch": x1["kern_ms"] / K},
        "plain_fp64": {"value": fp64["value"], "unit": UNIT, "ms_per_step": fp64["t_ms"] / K,
                       "dtype": "f64", "roofline_frac": ach64 / hbm, "achieved_gbs": ach64,
                       "per_step": fp64["per_step"]},
        "precision_jacobi": {"value": jac["value"], "unit": UNIT, "ms_per_step": jac["t_ms"] / K,
                             "dtype": "fp32+fp64", "roofline_frac": achj / hbm, "achieved_gbs": achj,
                             "per_step": jac["per_step"]},
        "multigrid": {"levels": amg, "inner_tol": x1["prm"].inner_tol},
        "demag_curve": {"fields_timed": K, "wall_s_precision_form": x1["t_ms"] / 1000.0,
                        "wall_s_plain_fp64": fp64["t_ms"] / 1000.0,
                        "wall_s_precision_jacobi": jac["t_ms"] / 1000.0,
                        "speedup_vs_plain_fp64": fp64["t_ms"] / x1["t_ms"],
                        "speedup_vs_precision_jacobi": jac["t_ms"] / x1["t_ms"],
                        "final_energy_rel_diff": abs(x1["F"] - fp64["F"]) / abs(fp64["F"]),
                        "final_max_abs_dm": dm, "per_step": x1["per_step"]},
        "gpu_launches": 2 * K,
    }
    line["config"]["precision"] = ("precision form: FP32 potential solve preconditioned by the multigrid V-cycle "
                                   "+ FP64 refinement (Jacobi-preconditioned in precision_jacobi, plain FP64 "
                                   "in plain_fp64)")
    if e2e:
        line["e2e"] = e2e
    if x1["clocks"]:
        line["clocks"] = x1["clocks"]
        for o in (fp64, jac):
            if o["clocks"]:
                line["clocks"]["reasons"] = sorted(set(line["clocks"]["reasons"]) | set(o["clocks"]["reasons"]))
    if world == 1 and not args.no_cpu_baseline:
        nli_c, dt_c, desc = oracle_sample(wl, max_iter=1)
        line["cpu_baseline"] = {"value": nli_c / dt_c, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line))
    mag.close()
    return 0


def curve_mode(args, rank, local_rank):
    """Full demagnetisation curves of one workload in four forms: plain FP64,
    the precision form with the Jacobi and with the multigrid potential
    preconditioner, and the multigrid precision form with the learned warm
    start (network trained on the curve of a coarser mesh of the same
    recipe).  Reports wall time, NCG iterations and coercive field."""
    import torch
    from paper_1801_03690_gb300 import Magnet, Params, MLP, warmstart
    from paper_1801_03690_gb300.curves import coercive_field
    wl = workload(args.workload)
    fields = wl.fields
    mag = Magnet(device=local_rank, blocks_per_sm=args.blocks_per_sm)
    mag.upload_workload(wl)
    sz = mag.sizes()
    out = {}

    forms = args.forms.split(",")

    def run(name, prm, net=None, scales=None):
        if name not in forms:
            return
        mag.set_magnetization(wl.m0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sts = []
        for k, b in enumerate(fields):
            if net is not None and k > 0:
                warmstart.warmstart_apply(mag, net, b, scales[0], scales[1], args.max_change)
            mag.set_field(b)
            sts.append(mag.minimize(prm))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        M = np.array([s["M"] for s in sts])
        out[name] = {"wall_s": wall, "nli": int(sum(s["nli"] for s in sts)),
                     "evals": int(sum(s["evals"] for s in sts)), "mi": int(sum(s["mi"] for s in sts)),
                     "Hc_T": coercive_field(fields, M),
                     "statuses": sorted(set(s["status"] for s in sts)),
                     "nli_per_step": [int(s["nli"]) for s in sts], "Mz": M[:, 2].tolist()}

    run("plain_fp64", Params(precision=0, theta_max=args.theta_max))
    run("precision", Params(precision=1, theta_max=args.theta_max))
    run("precision_multigrid", Params(precision=1, amg=1, inner_tol=1e-3, theta_max=args.theta_max))
    # learned warm start: train on the curve of the same recipe at half the resolution
    if "precision_learned" not in forms:
        if rank == 0:
            print(json.dumps({"mode": "curve", "workload": wl.name, "sizes": sz, "forms": out}))
        return 0
    t0 = time.perf_counter()
    import synth
    coarse = synth.hard_cube(n_mag=max(8, wl.meta.get("n_mag", 48) // 2), seed=12,
                             n_fields=len(fields)) if args.workload == "hard_cube" else None
    if coarse is None:
        coarse = synth.hard_cube(n_mag=12, seed=12, n_fields=len(fields))
    tm = Magnet(device=local_rank)
    tm.upload_workload(coarse)
    X, T, _ = warmstart.collect(tm, coarse.m0, coarse.fields, tm.sizes()["n_mag"],
                                Params(precision=1, amg=1, inner_tol=1e-3))
    tm.close()
    net = MLP(device=local_rank, seed=11)
    s_m, s_p, losses = warmstart.train(net, X, T, steps=1500, batch=16384, lr=2e-3, log_every=500)
    train_s = time.perf_counter() - t0
    run("precision_learned", Params(precision=1, amg=1, inner_tol=1e-3, theta_max=args.theta_max), net=net,
        scales=(s_m, s_p))
    ref = out.get("plain_fp64") or out.get("precision")
    for k in ("precision", "precision_multigrid", "precision_learned"):
        if k not in out or out[k] is ref:
            continue
        o = out[k]
        o["speedup_vs_plain_fp64"] = ref["wall_s"] / o["wall_s"]
        if o["Hc_T"] is not None and ref["Hc_T"] is not None:
            o["Hc_rel_diff"] = abs(o["Hc_T"] - ref["Hc_T"]) / ref["Hc_T"]
        o["max_abs_dMz"] = float(np.max(np.abs(np.array(o["Mz"]) - np.array(ref["Mz"]))))
    out["precision_learned"]["training"] = {"samples": int(X.shape[0]), "steps": 1500, "seconds": train_s,
                                            "losses": losses, "trained_on": coarse.name,
                                            "max_change": args.max_change}
    if rank == 0:
        print(json.dumps({"mode": "curve", "workload": wl.name, "sizes": sz, "n_fields": len(fields),
                          "forms": out}))
    mag.close()
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
        sz = mag.sizes()
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
            nbytes += alg_bytes(st, sz, lv)
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
    autotuner picked the kernel instantiation and team split), against the
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
        res["autotune"] = {"blocks_per_sm": bps, "gamma": gamma, "trial_ms": ms}
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
