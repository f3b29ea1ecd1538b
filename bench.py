#!/usr/bin/env python
"""Benchmark: forward transient solves of the 100^3 inclusions workload.

One bench step is one complete forward simulation, as in the paper's inverse
problem where each sample is a full transient solve (§5.3): set the
per-element coefficients and the initial temperature, then run the 300
theta-scheme steps (Jacobi-PCG per step, Algorithm 1) on the 100^3 Q1 mesh
(1,030,301 DOF) with 200 spherical inclusions, FP32 operator with FP64 dots
and FP64 iterative refinement, rtol 1e-10.

Metric: DOF x CG-iterations per second (inner + outer iterations), whole job.
  value: inputs already resident in HBM (device-to-device coefficient/state
         upload inside the timed region).
  e2e:   the same through the public host API (pinned host coefficients and
         initial state copied in, final field copied out, every step).
Between timed steps a 256 MiB buffer is overwritten to flush L2.

--impl reference times the CPU oracle (test infrastructure, plain FP64 CSR
Jacobi-PCG) on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank runs its own independent forward solves
(replicas, weak scaling), no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF*CG-iters/s"
# What each precision computes in: "df64" is double-float arithmetic, a pair
# of FP32 values with error-free sums and products (about 48 significant bits).
DTYPE_DETAIL = {
    "fp64": "FP64 vectors, operator and dot products",
    "fp32_refined": ("inner CG in FP32 (vectors and operator; dot products summed in FP32 per warp, then FP64); "
                     "outer refinement: FP64 solution, right-hand side and residual vectors with FP64 dot "
                     "products, the residual's operator b - A x evaluated in double-float (df64, ~48 bits)"),
    "fp32_plain": "FP32 vectors and operator; dot products summed in FP32 per warp, then FP64",
}
UNIT = "DOF*iter/s"
WORKLOAD = "inclusions_cube_100: Q1 100^3 (1,030,301 DOF), 200 spherical inclusions k=10 rho_c=3, flux pulse z=1 for 50 steps, dt=1e-3, theta=0.5, 300 steps per forward solve, rtol 1e-10"
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nsteps", type=int, default=300, help="time steps per forward solve")
    ap.add_argument("--precision", default="fp32_refined", choices=["fp64", "fp32_refined", "fp32_plain"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison solve")
    ap.add_argument("--profile-reps", type=int, default=120)
    ap.add_argument("--batch-sims", type=int, default=256, help="batched workload: 40^3 samples (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=150)
    ap.add_argument("--batch-only", action="store_true", help="run only the batched workload")
    ap.add_argument("--layered-steps", type=int, default=10,
                    help="200^3 layered cube: time steps of its FP32-refined and FP64 legs (0: skip)")
    ap.add_argument("--layered-only", action="store_true", help="run only the 200^3 layered legs")
    ap.add_argument("--cheb-degrees", default="2,3",
                    help="Chebyshev-Jacobi degrees timed on the layered FP32-refined leg ('' to skip)")
    ap.add_argument("--cheb-ratio", type=float, default=10.0, help="Chebyshev interval ratio lam_hi / lam_lo")
    ap.add_argument("--p1-steps", type=int, default=30,
                    help="six-tetrahedra leg: steps of the inclusions workload on P1 and Q1 elements (0: skip)")
    ap.add_argument("--p1-only", action="store_true", help="run only the six-tetrahedra leg")
    ap.add_argument("--mh-chains", type=int, default=32,
                    help="corrosion inverse problem: Metropolis-Hastings chains solved as one batch (0: skip)")
    ap.add_argument("--mh-iters", type=int, default=8)
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="serving stream at the configured rate: requests (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-low-requests", type=int, default=100,
                    help="second serving stream at a rate one GPU sustains: requests (0: skip)")
    ap.add_argument("--serve-low-rate", type=float, default=4.0)
    ap.add_argument("--serve-budget-gb", type=float, default=16.0)
    ap.add_argument("--slab-steps", type=int, default=5,
                    help="z-slab split of the 100^3 FP64 solve: time steps per slab count (0: skip)")
    ap.add_argument("--slab-only", action="store_true", help="run only the z-slab leg")
    ap.add_argument("--serve-only", action="store_true", help="run only the two serving streams")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default kernel tuning table")
    ap.add_argument("--persistent-compare", type=int, default=1,
                    help="1: time the persistent inner iteration against the tick graph (headline and batch)")
    ap.add_argument("--tuning-json", default="",
                    help='set the kernel tuning table instead of autotuning, e.g. '
                         '\'{"variant": [-1, 1, 0], "seg_nodes": [2048, 1024, 512]}\'')
    ap.add_argument("--cpu-configs", action="store_true",
                    help="time the oracle's C solver on every configuration (host only) and exit")
    ap.add_argument("--cpu-worker", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------- oracle leg

def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return os.cpu_count() or 1, model


def c_oracle_steps(p, S, nsteps: int, threads: int, max_iter: int = 20000):
    """The oracle's C Jacobi-PCG (Algorithm 1) over the first nsteps steps:
    (seconds in the solver, CG iterations). Right-hand sides (sparse products
    in the Python oracle) are formed outside the timed solver calls."""
    import numpy as np
    from oracle import cpu, transient
    A = cpu.CSR(S.A_ff)
    u_prev, u_prev2 = p.u0.copy(), None
    u_prev[S.dir_ids] = S.dir_vals
    sec, its = 0.0, 0
    for n in range(1, nsteps + 1):
        b = transient.step_rhs(p, S, u_prev, n)
        x0 = (u_prev if u_prev2 is None else 2.0 * u_prev - u_prev2)[S.free]
        t0 = time.perf_counter()
        x, it, _, _ = cpu.pcg(A, b, x0, S.pinv_f, p.rtol, max_iter=max_iter, threads=threads)
        sec += time.perf_counter() - t0
        its += it
        u = np.empty(p.n_nodes)
        u[S.free] = x
        u[S.dir_ids] = S.dir_vals
        u_prev2, u_prev = u_prev, u
    return sec, its


def cpu_worker(nsteps_sample: int):
    """Runs in a fresh process before the GPU is touched: the oracle on the
    first time steps of the headline workload, in Python (SciPy CSR, one
    thread), in C on one thread, and in C on every host core; then the
    incomplete-Cholesky context."""
    import workloads as W
    from oracle import transient

    p = W.inclusions_cube()
    S = transient.build_system(p)  # assembly: setup, not timed
    t0 = time.perf_counter()
    res = transient.run(p, solver="pcg", nsteps=nsteps_sample, system=S)
    dt = time.perf_counter() - t0
    it = sum(res.iters)
    cores, model = host_cpu()
    out = {"python": {"seconds": dt, "iters": it, "value": p.n_nodes * it / dt, "threads": 1},
           "dof": p.n_nodes, "steps": nsteps_sample, "nproc": cores, "cpu_model": model}
    for key, th in (("c_one_core", 1), ("c_all_cores", cores)):
        sec, its = c_oracle_steps(p, S, nsteps_sample, th)
        out[key] = {"seconds": sec, "iters": its, "value": p.n_nodes * its / sec, "threads": th}
    out["incomplete_factorisation"] = ic_context()
    print(json.dumps(out))


def ic_context(n: int = 40):
    """The paper's CPU comparison solver (§5.2, Table 2): CG preconditioned by
    an incomplete Cholesky factorisation of drop tolerance 1e-3, in the
    oracle's plain C, against the oracle's C Jacobi-PCG, on the first step of
    the inclusions workload at n^3 elements (context only, one thread)."""
    from oracle import cpu, transient
    import workloads as W

    p = W.inclusions_cube(n=n)
    S = transient.build_system(p)
    b = transient.step_rhs(p, S, p.u0, 1)
    x0 = p.u0[S.free]
    A = cpu.CSR(S.A_ff)
    t0 = time.perf_counter()
    F = cpu.IC(A, 1e-3)
    t1 = time.perf_counter()
    _, it_ic, _, _ = cpu.pcg_ic(A, b, x0, S.pinv_f, F, p.rtol)
    t2 = time.perf_counter()
    _, it_jac, _, _ = cpu.pcg(A, b, x0, S.pinv_f, p.rtol, threads=1)
    t3 = time.perf_counter()
    return {"sample": f"inclusions_cube_{n} ({p.n_nodes} DOF), step 1, rtol {p.rtol:g}", "drop_tol": 1e-3,
            "factorisation": "incomplete Cholesky, drop |l_ik| < 1e-3 ||A(k:n,k)||_1 (oracle/cpcg.c)",
            "factorisation_s": t1 - t0, "factor_nnz_per_row": F.nnz / S.free.size,
            "ic_pcg": {"iterations": it_ic, "solve_s": t2 - t1},
            "jacobi_pcg": {"iterations": it_jac, "solve_s": t3 - t2}, "cores": 1}


def cpu_config_timings():
    """--cpu-configs: the oracle's C Jacobi-PCG on every configuration's
    workload, one thread and every host core, with the truncation stated:
    the 16^3 two-phase cube (all 20 steps), the 100^3 inclusions cube (first
    3 steps), one 40^3 log-normal batch member (first 20 of 150 steps), and
    the 200^3 layered cube (the first 100 CG iterations of step 1, on the
    eliminated operator padded with identity rows, assembled in stencil form).
    Prints one JSON line."""
    import numpy as np
    import scipy.sparse as sp
    import workloads as W
    from oracle import cpu, fem, transient
    cores, model = host_cpu()
    out = {"nproc": cores, "cpu_model": model, "configs": {}}
    cases = [("1 two_phase_cube 16^3", W.two_phase_cube(), None, "all 20 steps"),
             ("2 inclusions_cube 100^3", W.inclusions_cube(), 3, "first 3 of 300 steps"),
             ("3 lognormal_cube 40^3 (one member)", W.lognormal_cube(0), 20, "first 20 of 150 steps")]
    for name, p, nsteps, trunc in cases:
        S = transient.build_system(p)
        ns = nsteps or p.nsteps
        row = {"dof": p.n_nodes, "truncation": trunc}
        for key, th in (("one_core", 1), ("all_cores", cores)):
            sec, its = c_oracle_steps(p, S, ns, th)
            row[key] = {"threads": th, "seconds": sec, "cg_iterations": its, "ms_per_iteration": 1e3 * sec / its,
                        "dof_cg_iters_per_s": p.n_nodes * its / sec, "ms_per_step": 1e3 * sec / ns}
        out["configs"][name] = row
        print(json.dumps({name: row}), file=sys.stderr, flush=True)
    # 200^3 layered: step 1's system, truncated to 100 iterations
    p = W.layered_cube(nsteps=1)
    A = fem.assemble_stencil(p, 1.0 / p.dt, p.theta)
    dn, dv = fem.dirichlet_nodes(p)
    mask = np.ones(p.n_nodes)
    mask[dn] = 0.0
    D = sp.diags(mask)
    Ap = (D @ A @ D + sp.diags(1.0 - mask)).tocsr()
    g = np.zeros(p.n_nodes)
    g[dn] = dv
    b = fem.apply_all(p, p.u0, 1.0 / p.dt, p.theta - 1.0, eliminate=False) - fem.apply_all(
        p, g, 1.0 / p.dt, p.theta, eliminate=False)
    b *= mask
    pinv = 1.0 / Ap.diagonal()
    M = cpu.CSR(Ap)
    row = {"dof": p.n_nodes, "truncation": "first 100 CG iterations of step 1 (of about 1,400)"}
    for key, th in (("one_core", 1), ("all_cores", cores)):
        t0 = time.perf_counter()
        _, its, _, _ = cpu.pcg(M, b, np.zeros(p.n_nodes), pinv, 1e-30, max_iter=100, threads=th)
        sec = time.perf_counter() - t0
        row[key] = {"threads": th, "seconds": sec, "cg_iterations": its, "ms_per_iteration": 1e3 * sec / its,
                    "dof_cg_iters_per_s": p.n_nodes * its / sec}
    out["configs"]["5 layered_cube 200^3"] = row
    print(json.dumps(out), flush=True)


def run_cpu_baseline(nsteps_sample: int):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", str(nsteps_sample)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(f"cpu baseline failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers

def cheb_degrees(args):
    return tuple(int(x) for x in args.cheb_degrees.split(",") if x.strip())


# Algorithmic floating-point operations per node of the FP64 apply (the
# factorised operator of the block tile and of the warp march): forward x 2,
# forward y 4, per element (one per node) 4 x 13 for the two z-Walsh halves
# (A, B, G, Tn), inverse y 4, node sums 5 = 67; the direction update
# d = P^-1 r + beta d_old 3 and the dot product d.q 2. An FMA counts 2.
FP64_APPLY_FLOPS_PER_NODE = 72
_FP64_PEAK = None


def fp64_peak_tflops(hg):
    """The FP64 FMA rate of this GPU, measured once per run (heat_probe_fma_rate)."""
    global _FP64_PEAK
    if _FP64_PEAK is None:
        _FP64_PEAK = hg.heat_probe_fma_rate(True, 5)
    return _FP64_PEAK


def fp64_roofline(hg, nodes: int, ms_apply: float) -> dict:
    """The FP64 apply against the measured FP64 FMA peak (its bound on this GPU)."""
    peak = fp64_peak_tflops(hg)
    achieved = FP64_APPLY_FLOPS_PER_NODE * nodes / (ms_apply * 1e-3) / 1e12
    return {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flops_per_node": FP64_APPLY_FLOPS_PER_NODE, "ms_per_launch": ms_apply,
            "peak_kind": "measured FP64 FMA rate (heat_probe_fma_rate, this run)"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def current_variant(hg, precision: str):
    """(segment width, rows, warps, stages, fused) of the apply the current table runs, or None (block tiles)."""
    v = hg.heat_tuning_get()["variant"][hg.PRECISIONS[precision]]
    if v < 0:
        return None
    i = hg.heat_tuning_variant(v)
    return [i["seg_width"], i["rows"], i["warps"], i["stages"], int(i["fused"])]


def ncu_traffic(kernel_key: str, variant=None):
    """DRAM bytes per launch from a committed ncu summary, if it matches the
    current kernel source and the apply variant the table runs now."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(kernel_key)
    except Exception:
        return None
    if not d:
        return None
    h = hashlib.sha256()
    for f in d.get("sources", []):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != d.get("sha256"):
        return None  # kernel changed since the counters were taken
    if variant is not None and d.get("variant") != variant:
        return None  # the counters are another variant's
    return d.get("dram_bytes_per_launch")


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _all_reduce(world, x: float, op: str) -> float:
    """Reduce a scalar over ranks (NCCL on GPUs, gloo on CPU processes)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(world, x: float) -> float:
    return _all_reduce(world, x, "max")


def sum_over_ranks(world, x: float) -> float:
    return _all_reduce(world, x, "sum")


def aggregate(world, seconds: float, units: float):
    """Whole-job throughput of replicas: every rank's units over the slowest
    rank's time (the ranks run independent simulations; no data-path
    collective)."""
    t = max_over_ranks(world, seconds)
    u = sum_over_ranks(world, units)
    return u / t, t, u


# ---------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    """The oracle (plain FP64 CSR Jacobi-PCG in C, OpenMP on every host core),
    each bench step one time step of the headline workload."""
    if rank != 0:
        return
    import numpy as np
    import workloads as W
    from oracle import cpu, transient

    p = W.inclusions_cube()
    S = transient.build_system(p)
    A = cpu.CSR(S.A_ff)
    cores, model = host_cpu()
    u_prev, u_prev2 = p.u0.copy(), None
    times, iters = [], []
    n = 0
    for k in range(args.warmup + args.steps):
        n += 1
        t0 = time.perf_counter()
        b = transient.step_rhs(p, S, u_prev, n)
        x0 = u_prev if u_prev2 is None else 2 * u_prev - u_prev2
        x, it, _, _ = cpu.pcg(A, b, x0[S.free], S.pinv_f, p.rtol, threads=cores)
        dt = time.perf_counter() - t0
        u_new = np.empty(p.n_nodes)
        u_new[S.free] = x
        u_new[S.dir_ids] = S.dir_vals
        u_prev2, u_prev = u_prev, u_new
        if k >= args.warmup:
            times.append(dt)
            iters.append(it)
    T = sum(times)
    value = p.n_nodes * sum(iters) / T
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "none (host)",
                                            "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"steps 1..{args.warmup + args.steps} of the 300-step transient, one per bench step (right-hand side in SciPy, Jacobi-PCG in the oracle's C on {cores} threads of {model}); assembly untimed"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iters": iters}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batch / serving

def set_table(hg, t):
    """Set the kernel tuning table from a dict (keys missing from it keep their current values)."""
    hg.heat_tuning_set(t["variant"], t["seg_nodes"], t.get("pw_quads"), t.get("open_w"), t.get("loop"))


def autotune(hg, p, precision, stream, reps=40):
    """Tune the kernel table for this problem's size bucket and precision
    (untimed; CG iterations through the tick graph, as the solve runs them)."""
    with hg.Simulation.from_problem(p, precision=precision, stream=stream.cuda_stream) as s:
        s.step(1)
        table, ms = hg.heat_autotune(s.sim, reps)
    return {"table": table, "best_ms_per_cg_iteration": ms}


def run_persistent(hg, torch, stream, headline_table, batch_table, nsteps_single=30, nsims=256, nsteps_batch=10):
    """The persistent inner iteration (tuning loop = 1: one cooperative kernel
    per tick that runs the iterations with a grid barrier after each phase)
    against the replayed tick graph (an apply and an update launch per
    iteration), each under its own table, on the first steps of the headline
    workload and of the batched one. Same work items, so with equal item sizes
    the fields are bitwise equal (checked here on the headline)."""
    import numpy as np
    import workloads as W
    base = hg.heat_tuning_get()
    pid = hg.PRECISIONS["fp32_refined"]

    def table(t, loop, quads=None):
        t = {k: list(v) for k, v in t.items()}
        t["loop"][pid] = loop
        if quads is not None:
            t["pw_quads"][pid] = quads
        return t

    def timed(fn):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e), r

    out = {"single": {"workload": f"inclusions_cube_100, first {nsteps_single} steps, fp32_refined"},
           "batch": {"workload": f"{nsims} x lognormal_cube_40, first {nsteps_batch} steps, fp32_refined"},
           # one grid barrier alone, 128-thread blocks (the loop runs 3 per SM)
           "us_per_grid_barrier": {f"{bps}_blocks_per_sm": hg.heat_probe_grid_barrier(bps, 2000) for bps in (1, 3)}}
    try:
        p = W.inclusions_cube(nsteps=nsteps_single)
        fields = {}
        for name, t in (("tick", table(headline_table, 0)),
                        ("loop_same_items", table(headline_table, 1)),
                        ("loop_pw1", table(headline_table, 1, 1)), ("loop_pw2", table(headline_table, 1, 2))):
            set_table(hg, t)
            with hg.Simulation.from_problem(p, precision="fp32_refined", stream=stream.cuda_stream) as s:
                s.step(1)
                hg.heat_set_state(s.sim, p.u0, s.n_nodes)
                ms, st = timed(lambda: s.step(nsteps_single))
                fields[name] = s.state()
            out["single"][name] = {"ms_per_step": ms / nsteps_single, "cg_iterations": st["iters"],
                                   "us_per_cg_iteration_incl_step_passes": ms * 1e3 / st["iters"],
                                   "kernel_launches": st["kernel_launches"], "pw_quads": t["pw_quads"][pid]}
        out["single"]["loop_bitwise_equal_to_tick"] = bool(np.array_equal(fields["tick"],
                                                                           fields["loop_same_items"]))
        ps = [W.lognormal_cube(k, n=40, nsteps=nsteps_batch) for k in range(nsims)]
        for name, t in (("tick", table(batch_table, 0)), ("loop_pw1", table(batch_table, 1, 1)),
                        ("loop_pw2", table(batch_table, 1, 2))):
            set_table(hg, t)
            sims = [hg.Simulation.from_problem(q, precision="fp32_refined", stream=stream.cuda_stream) for q in ps]
            b = hg.heat_batch_create([x.sim for x in sims], stream.cuda_stream)
            try:
                hg.heat_batch_step(b, 1, nsims)
                for x, q in zip(sims, ps):
                    hg.heat_set_state(x.sim, q.u0, x.n_nodes)
                ms, (rc, stats) = timed(lambda: hg.heat_batch_step(b, nsteps_batch, nsims))
                its = sum(st["iters"] for st in stats)
                out["batch"][name] = {"ms_per_step": ms / nsteps_batch, "cg_iterations": its, "rc": rc,
                                      "kernel_launches": stats[0]["kernel_launches"],
                                      "dof_cg_iters_per_s": sims[0].n_nodes * its / (ms * 1e-3)}
            finally:
                hg.heat_destroy_batch(b)
                for x in sims:
                    x.close()
    finally:
        set_table(hg, base)
    return out


def run_batch(hg, torch, nsims: int, nsteps: int, stream, tune=True, fixed_tuning=False):
    """256 independent 40^3 samples with log-normal k (seeds 3000+s), FP32
    refined, one engine: every launch carries all samples."""
    import workloads as W
    ps = [W.lognormal_cube(s, n=40, nsteps=nsteps) for s in range(nsims)]
    tuning = None
    sims = [hg.Simulation.from_problem(p, precision="fp32_refined", stream=stream.cuda_stream) for p in ps]
    b = hg.heat_batch_create([s.sim for s in sims], stream.cuda_stream)
    try:
        rc, _ = hg.heat_batch_step(b, 2, nsims)  # warm-up steps (graph capture, caches)
        if tune and not fixed_tuning:  # the whole batch's CG iterations through its tick graph (untimed)
            table, ms = hg.heat_batch_autotune(b, 40)
            tuning = {"table": table, "best_ms_per_cg_iteration": ms}
            rc, _ = hg.heat_batch_step(b, 1, nsims)
        for s, p in zip(sims, ps):
            hg.heat_set_state(s.sim, p.u0, s.n_nodes)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc, stats = hg.heat_batch_step(b, nsteps, nsims)
        e.record(stream)
        e.synchronize()
        sec = a.elapsed_time(e) / 1e3
        if rc != 0:
            raise RuntimeError(hg.heat_last_error())
        its = sum(st["iters"] for st in stats)
        dof = sims[0].n_nodes
        # the batch's CG-iteration kernels timed alone (L2 flushed before each launch)
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        torch.cuda.nvtx.range_push("roofline_batch")  # ncu captures filter on this range
        prof = hg.heat_batch_profile_iteration(b, 20, flush)
        torch.cuda.nvtx.range_pop()
        peak, _ = measured_peaks()
        achieved = prof["bytes_apply"] / (prof["ms_apply"] * 1e-3) / 1e9
        return {"workload": f"{nsims} x lognormal_cube_40 (68,921 DOF each), {nsteps} steps, dt=2e-3, theta=0.5, rtol 1e-10, fp32_refined",
                "seconds": sec, "sims_per_s": nsims / sec, "dof_cg_iters_per_s": dof * its / sec,
                "cg_iterations_per_sim_step": its / (nsims * nsteps),
                "kernel_launches": stats[0]["kernel_launches"], "tuning": tuning,
                "roofline": {"bound": "hbm", "kernel": "k_apply_dot<float>", "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak,
                             "traffic": ncu_traffic("k_apply_dot<float>@lognormal_batch_256x40",
                                                   current_variant(hg, "fp32_refined")),
                             "ms_per_launch": prof["ms_apply"],
                             "algorithmic_bytes_per_launch": prof["bytes_apply"],
                             "update_kernel": {"ms_per_launch": prof["ms_update"],
                                               "achieved": prof["bytes_update"] / (prof["ms_update"] * 1e-3) / 1e9}}}
    finally:
        hg.heat_destroy_batch(b)
        for s in sims:
            s.close()


def run_layered(hg, torch, nsteps: int, stream, tune=True, cheb_degrees=(), cheb_ratio=10.0):
    """The 200^3 layered cube (8,120,601 DOF, k 1:1000 layers and 0.01 pockets,
    Dirichlet 1 on z=0, dt=5e-4, theta=0.5, rtol 1e-10): its first `nsteps`
    steps in FP32-refined and in FP64, timed with CUDA events, plus the
    dominant kernel of each timed alone after an L2 flush; then the same
    FP32-refined steps with the Chebyshev-Jacobi preconditioner of each
    degree in cheb_degrees."""
    import numpy as np
    import workloads as W
    p = W.layered_cube(nsteps=nsteps)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    peak, _ = measured_peaks()
    out = {"workload": f"layered_cube_200 (8,120,601 DOF), first {nsteps} of its 100 steps, dt=5e-4, theta=0.5, rtol 1e-10"}
    fields = {}
    tuned32 = None
    for precision in ("fp32_refined", "fp64"):
        tuning = autotune(hg, p, precision, stream) if tune else None
        if precision == "fp32_refined":
            tuned32 = tuning
        with hg.Simulation.from_problem(p, precision=precision, stream=stream.cuda_stream) as s:
            s.step(1)  # warm-up (graph capture)
            hg.heat_set_state(s.sim, p.u0, s.n_nodes)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = s.step(nsteps)
            e.record(stream)
            e.synchronize()
            sec = a.elapsed_time(e) / 1e3
            fields[precision] = s.state()
            torch.cuda.nvtx.range_push(f"roofline_layered_{precision}")  # ncu captures filter on this range
            prof = hg.heat_profile_iteration(s.sim, 20, flush)
            torch.cuda.nvtx.range_pop()
        achieved = prof["bytes_apply"] / (prof["ms_apply"] * 1e-3) / 1e9
        if precision == "fp64":
            out["fp64_roofline"] = fp64_roofline(hg, p.n_nodes, prof["ms_apply"])
        out[precision] = {"seconds": sec, "ms_per_step": sec * 1e3 / nsteps, "cg_iterations": st["iters"],
                          "dof_cg_iters_per_s": p.n_nodes * st["iters"] / sec, "kernel_tuning": tuning,
                          "apply": {"ms_per_launch": prof["ms_apply"], "achieved_gbs": achieved, "peak_gbs": peak,
                                    "frac": achieved / peak, "algorithmic_bytes_per_launch": prof["bytes_apply"],
                                    "traffic": ncu_traffic("k_apply_dot<float>@layered_cube_200",
                                                                           current_variant(hg, "fp32_refined"))
                                    if precision == "fp32_refined" else None},
                          "update": {"ms_per_launch": prof["ms_update"],
                                     "achieved_gbs": prof["bytes_update"] / (prof["ms_update"] * 1e-3) / 1e9
                                     if prof["ms_update"] > 0 else None}}
    u32, u64 = fields["fp32_refined"], fields["fp64"]
    out["final_field_rel_err_fp32_refined_vs_fp64"] = float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64))
    if cheb_degrees:
        # Chebyshev-Jacobi against the FP32-refined Jacobi leg, same steps and
        # kernel table (a fused variant gives way to its register-prefetch form)
        if tuned32 is not None:
            set_table(hg, tuned32["table"])
        jac = out["fp32_refined"]
        legs = {}
        for m in cheb_degrees:
            with hg.Simulation.from_problem(p, precision="fp32_refined", stream=stream.cuda_stream,
                                            cheb_degree=m, cheb_ratio=cheb_ratio) as s:
                s.step(1)
                hg.heat_set_state(s.sim, p.u0, s.n_nodes)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st = s.step(nsteps)
                e.record(stream)
                e.synchronize()
                sec = a.elapsed_time(e) / 1e3
                lo, hi = hg.heat_cheb_interval(s.sim)
                uc = s.state()
            legs[f"degree_{m}"] = {"ms_per_step": sec * 1e3 / nsteps, "cg_iterations": st["iters"],
                                   "iterations_vs_jacobi": st["iters"] / jac["cg_iterations"],
                                   "operator_passes_vs_jacobi": st["iters"] * m / jac["cg_iterations"],
                                   "time_vs_jacobi": sec * 1e3 / nsteps / jac["ms_per_step"],
                                   "interval": [lo, hi], "status": st["status"],
                                   "final_field_rel_diff_vs_jacobi": float(np.linalg.norm(uc - u32) / np.linalg.norm(u32))}
        out["chebyshev_fp32_refined"] = {"ratio": cheb_ratio, **legs}
    # the laminate on §4.1's own element (six tetrahedra per box), same steps and table
    pp = W.layered_cube(nsteps=nsteps)
    pp.element = "p1"
    if tuned32 is not None:
        set_table(hg, tuned32["table"])
    with hg.Simulation.from_problem(pp, precision="fp32_refined", stream=stream.cuda_stream) as s:
        s.step(1)
        hg.heat_set_state(s.sim, pp.u0, s.n_nodes)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = s.step(nsteps)
        e.record(stream)
        e.synchronize()
        sec = a.elapsed_time(e) / 1e3
        up = s.state()
    out["six_tetrahedra_fp32_refined"] = {
        "ms_per_step": sec * 1e3 / nsteps, "cg_iterations": st["iters"], "status": st["status"],
        "dof_cg_iters_per_s": pp.n_nodes * st["iters"] / sec,
        "final_field_rel_diff_vs_trilinear": float(np.linalg.norm(up - u32) / np.linalg.norm(u32))}
    return out


def run_p1(hg, torch, nsteps: int, stream, table=None):
    """The inclusions workload on six-tetrahedra boxes (§4.1's element: 6
    million linear tetrahedra on the 100^3 grid, 1,030,301 DOF), FP32-refined,
    first `nsteps` of its 300 steps; plus the P1 apply kernel timed alone after
    an L2 flush. The trilinear leg's numbers for the same steps are the
    comparison."""
    import workloads as W
    out = {"workload": f"inclusions_cube_100 on six-tetrahedra boxes (6,000,000 tetrahedra, 1,030,301 DOF), "
                       f"first {nsteps} of its 300 steps, FP32-refined, rtol 1e-10"}
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    peak, _ = measured_peaks()
    if table is not None:  # the headline's kernel table (later legs retune for their own sizes)
        set_table(hg, table)
    out["kernel_table"] = hg.heat_tuning_get()
    for element in ("p1", "q1"):
        p = W.inclusions_cube(nsteps=nsteps)
        p.element = element
        with hg.Simulation.from_problem(p, precision="fp32_refined", stream=stream.cuda_stream) as s:
            s.step(1)  # warm-up (graph capture)
            hg.heat_set_state(s.sim, p.u0, s.n_nodes)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = s.step(nsteps)
            e.record(stream)
            e.synchronize()
            sec = a.elapsed_time(e) / 1e3
            torch.cuda.nvtx.range_push(f"roofline_{element}")
            prof = hg.heat_profile_iteration(s.sim, 40, flush)
            torch.cuda.nvtx.range_pop()
        achieved = prof["bytes_apply"] / (prof["ms_apply"] * 1e-3) / 1e9
        out[element] = {"ms_per_step": sec * 1e3 / nsteps, "cg_iterations": st["iters"], "status": st["status"],
                        "dof_cg_iters_per_s": p.n_nodes * st["iters"] / sec,
                        "apply": {"ms_per_launch": prof["ms_apply"], "achieved_gbs": achieved, "peak_gbs": peak,
                                  "frac": achieved / peak, "algorithmic_bytes_per_launch": prof["bytes_apply"]},
                        "update_ms_per_launch": prof["ms_update"]}
    return out


def run_mh(hg, torch, nchains: int, niter: int, stream):
    """The §5.3 inverse problem on a synthetic plate (corrosion_plate: 64 x 20 x 64
    elements, 88,725 DOF, 100 steps of 0.1 s): camera data from the GPU forward
    model at the true depth plus seeded noise, then nchains Metropolis-Hastings
    chains whose proposals are solved as one batch per iteration (FP32-refined,
    rtol 1e-10). Wall time of the chain steps (host accept/reject included)."""
    import numpy as np
    import workloads as W
    pl = W.corrosion_plate()
    geom = hg.make_corrosion(*(pl.geom[k] for k in ("z0", "half_width", "rho_c_sound", "k_sound", "rho_c_corr",
                                                    "k_corr")))
    p = pl.problem()
    with hg.Simulation.from_problem(p, precision="fp64", stream=stream.cuda_stream) as s:
        hg.heat_set_face_flux(s.sim, pl.flux_face, pl.flux_q)
        hg.heat_set_coeffs_corrosion(s.sim, geom, pl.depth_true)
        s.step(pl.nsteps)
        u = s.state()
    i = np.arange(pl.nx + 1)
    k = np.arange(pl.nz + 1)
    face = (i[None, :] + (pl.nx + 1) * (pl.ny + 1) * k[:, None]).ravel()  # y = 0, i fastest
    data = pl.camera(u[face])
    normals, uniforms = pl.draws(niter, nchains)
    start = np.linspace(1.0, 11.0, nchains)
    with hg.MHDriver(pl.nx, pl.ny, pl.nz, pl.extent, geom, data, pl.sigma, nchains, pl.nsteps, pl.depth_max,
                     flux_face=pl.flux_face, flux_q=pl.flux_q, obs_face=pl.obs_face, u0=pl.u0, theta=pl.theta,
                     dt=pl.dt, rtol=pl.rtol, precision="fp32_refined", stream=stream.cuda_stream) as mh:
        ll0 = mh.loglik(start)  # also captures the batch's tick graph
        solves0, iters0 = mh.stats()
        t0 = time.perf_counter()
        st, ll, dtr, ltr, acc = mh.run(niter, 0.5, normals, uniforms, start, ll0)
        sec = time.perf_counter() - t0
        solves, iters = mh.stats()
    solves -= solves0
    iters -= iters0
    return {"workload": f"corrosion_plate 64x20x64 (88,725 DOF), {pl.nsteps} steps of {pl.dt} s, {nchains} chains x "
                        f"{niter} Metropolis-Hastings steps, fp32_refined rtol {pl.rtol}, true depth {pl.depth_true} mm",
            "seconds": sec, "mh_steps_per_s": niter * nchains / sec, "forward_solves_per_s": solves / sec,
            "dof_cg_iters_per_s": p.n_nodes * iters / sec, "acceptance": float(acc.mean()),
            "chain_mean_depth_last": float(st.mean())}


def run_serving(hg, nreq: int, rate: float, budget_gb: float):
    """Poisson arrivals of serving_request(r) (edge U{20..120}, two-phase k,
    50..300 steps, rtol 1e-8, fp32_refined) at `rate` per second."""
    import numpy as np
    import workloads as W
    arrivals = W.poisson_arrivals(nreq, rate=rate)
    reqs, nodes = [], []
    for r in range(nreq):  # inputs prepared before the clock starts; only the request arrays are kept
        p = W.serving_request(r)
        reqs.append(hg.make_request(p))
        nodes.append(p.n_nodes)
        del p
    srv = hg.heat_server_create(int(budget_gb * (1 << 30)), 64)
    try:
        t0 = time.perf_counter()
        tickets = []
        for (req, keep), ta in zip(reqs, arrivals):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            tickets.append(hg.heat_submit(srv, req))
        lat, its_dof = [], 0.0
        for t, nn in zip(tickets, nodes):
            u, st, l = hg.heat_wait(srv, t, nn, timeout_s=3600.0)
            lat.append(l)
            its_dof += nn * st["iters"]
        wall = time.perf_counter() - t0
        sst = hg.heat_server_get_stats(srv)
    finally:
        hg.heat_destroy_server(srv)
    lat = np.array(lat)
    return {"workload": f"{nreq} requests, Poisson {rate}/s, cubic Q1 20^3..120^3, two-phase k 10:1 at phi U[0.1,0.5], 50..300 steps, dt=1e-3, rtol 1e-8, fp32_refined, HBM budget {budget_gb} GB",
            "requests": nreq, "arrival_rate_per_s": rate, "arrival_span_s": float(arrivals[-1]),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "sims_per_s": nreq / wall, "dof_cg_iters_per_s": its_dof / wall, "wall_s": wall,
            "offered_dof": float(sum(nodes)), "kernel_launches": sst["kernel_launches"],
            "failed": sst["failed"]}


def run_slab(hg, torch, nsteps: int, stream):
    """The z-slab split of one simulation (§4.4): the 100^3 inclusions
    workload's first `nsteps` steps in FP64, unsplit (the tick engine) and
    split into 1, 2, 4 and 8 slabs on this GPU, in the merged one-reduction
    iteration and (4 slabs) in Algorithm 1's two-reduction form. Times are
    CUDA events on the stream; every split field is compared with the
    unsplit one."""
    import numpy as np
    import workloads as W
    p = W.inclusions_cube(nsteps=nsteps)
    out = {"workload": f"inclusions_cube_100 (1,030,301 DOF), first {nsteps} steps, FP64, rtol 1e-10"}

    def timed(run):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = run()
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e) / 1e3, st

    with hg.Simulation.from_problem(p, precision="fp64", stream=stream.cuda_stream) as s:
        s.step(1)
        hg.heat_set_state(s.sim, p.u0, p.n_nodes)
        sec, st = timed(lambda: s.step(nsteps))
        whole = s.state()
    out["unsplit"] = {"ms_per_step": sec * 1e3 / nsteps, "cg_iterations": st["iters"],
                      "dof_cg_iters_per_s": p.n_nodes * st["iters"] / sec}
    for ns, merged in ((1, True), (2, True), (4, True), (8, True), (4, False)):
        with hg.SlabSimulation.from_problem(p, ns, merged=merged, stream=stream.cuda_stream) as s:
            s.step(1)
            s.set_state(p.u0)
            sec, st = timed(lambda: s.step(nsteps))
            u = s.state()
        key = f"slabs_{ns}_{'merged' if merged else 'algorithm1'}"
        out[key] = {"ms_per_step": sec * 1e3 / nsteps, "cg_iterations": st["iters"],
                    "dof_cg_iters_per_s": p.n_nodes * st["iters"] / sec,
                    "kernel_launches": st["kernel_launches"],
                    "field_rel_diff_vs_unsplit": float(np.linalg.norm(u - whole) / np.linalg.norm(whole))}
    return out


# ---------------------------------------------------------------- our arm

def main():
    args = parse()
    if args.cpu_configs:
        cpu_config_timings()
        return
    if args.cpu_worker:
        cpu_worker(args.cpu_worker)
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, world, rank)
        return

    # the CPU baseline runs in a fresh process before this one touches the GPU
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(2)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1905_07622_gb300 as hg
    import workloads as W

    stream = torch.cuda.current_stream()
    if args.layered_only:  # the 200^3 layered legs alone (used for profiling captures)
        if args.tuning_json:
            t = json.loads(args.tuning_json)
            set_table(hg, t)
        print(json.dumps({"layered": run_layered(hg, torch, args.layered_steps, stream,
                                                 not (args.no_autotune or args.tuning_json),
                                                 cheb_degrees(args), args.cheb_ratio)}), flush=True)
        return
    if args.slab_only:  # the z-slab leg alone
        print(json.dumps({"z_slabs": run_slab(hg, torch, args.slab_steps, stream)}), flush=True)
        return
    if args.serve_only:  # the two serving streams alone
        out = {"serving": run_serving(hg, args.serve_requests, args.serve_rate, args.serve_budget_gb)
               if args.serve_requests > 0 else None,
               "serving_sustainable_rate": run_serving(hg, args.serve_low_requests, args.serve_low_rate,
                                                       args.serve_budget_gb) if args.serve_low_requests > 0 else None}
        print(json.dumps(out), flush=True)
        return
    if args.p1_only:  # the six-tetrahedra leg alone (used for profiling captures)
        print(json.dumps({"tetrahedra": run_p1(hg, torch, args.p1_steps, stream)}), flush=True)
        return
    if args.batch_only:  # the batched workload alone (used for profiling captures)
        fixed = bool(args.tuning_json)
        if fixed:
            t = json.loads(args.tuning_json)
            set_table(hg, t)
        print(json.dumps({"batched": run_batch(hg, torch, args.batch_sims, args.batch_steps, stream,
                                               not args.no_autotune, fixed)}), flush=True)
        return
    p = W.inclusions_cube(nsteps=args.nsteps)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    fixed = bool(args.tuning_json)
    if fixed:
        t = json.loads(args.tuning_json)
        set_table(hg, t)
        tuning = {"table": hg.heat_tuning_get(), "set_by": "--tuning-json"}
    else:
        tuning = None if args.no_autotune else autotune(hg, p, args.precision, stream)
    sim = hg.Simulation.from_problem(p, precision=args.precision, stream=stream.cuda_stream)
    nn, ne = sim.n_nodes, sim.n_elems
    rc_d = torch.tensor(p.rho_c, device="cuda")
    k_d = torch.tensor(p.k, device="cuda")
    u0_d = torch.tensor(p.u0, device="cuda")

    def forward_device():
        hg.heat_set_coeffs(sim.sim, rc_d, k_d, ne)
        hg.heat_set_state(sim.sim, u0_d, nn)
        return hg.heat_step(sim.sim, args.nsteps)

    # pinned host inputs/outputs for the end-to-end leg
    rc_h = torch.tensor(p.rho_c).pin_memory().numpy()
    k_h = torch.tensor(p.k).pin_memory().numpy()
    u0_h = torch.tensor(p.u0).pin_memory().numpy()
    u_out = torch.empty(nn, dtype=torch.float64).pin_memory().numpy()

    def forward_host():
        hg.heat_set_coeffs(sim.sim, rc_h, k_h, ne)
        hg.heat_set_state(sim.sim, u0_h, nn)
        return hg.heat_solve_transient_into(sim.sim, args.nsteps, u_out)

    def timed(fn, K, W_):
        for _ in range(W_):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        ms, its, launches = [], 0, 0
        for _ in range(K):
            flush.random_(0, 255)  # evict L2 between timed steps (not timed)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            its += st["iters"]
            launches += st["kernel_launches"]
        torch.cuda.synchronize()
        barrier(world)
        return ms, its, launches

    with ClockSampler(torch.cuda.current_device()) as clk:
        ms, its, launches = timed(forward_device, args.steps, args.warmup)
    clocks = clk.summary()
    ms_e2e, its_e2e, _ = timed(forward_host, args.steps, 1)

    value, T, units = aggregate(world, sum(ms) / 1e3, float(nn) * its)
    value_e2e, _, _ = aggregate(world, sum(ms_e2e) / 1e3, float(nn) * its_e2e)

    # accuracy of this configuration's final field vs the FP64 path (same GPU)
    u_ref = None
    fp64 = None
    if not args.no_fp64 and rank == 0:
        sim64 = hg.Simulation.from_problem(p, precision="fp64", stream=stream.cuda_stream)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st64 = sim64.step(args.nsteps)
        b.record(stream)
        b.synchronize()
        t64 = a.elapsed_time(b) / 1e3
        u_ref = sim64.state()
        prof64 = hg.heat_profile_iteration(sim64.sim, args.profile_reps, flush)
        fp64 = {"value": nn * st64["iters"] / t64, "unit": UNIT, "iters": st64["iters"],
                "ms_per_forward_solve": t64 * 1e3, "roofline": fp64_roofline(hg, nn, prof64["ms_apply"])}
        sim64.close()
    final_err = None
    if u_ref is not None:
        u = sim.state()
        final_err = float(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref))

    # dominant kernel (apply + direction + d.q of the inner solve), timed alone
    # with CUDA events on this stream, L2 flushed before each launch
    torch.cuda.nvtx.range_push("roofline")  # ncu captures filter on this range
    prof = hg.heat_profile_iteration(sim.sim, args.profile_reps, flush)
    torch.cuda.nvtx.range_pop()
    peak, peak_kind = measured_peaks()
    achieved = prof["bytes_apply"] / (prof["ms_apply"] * 1e-3) / 1e9
    kernel_key = f"k_apply_dot<{'double' if args.precision == 'fp64' else 'float'}>@inclusions_cube_100"
    traffic = ncu_traffic(kernel_key, current_variant(hg, args.precision))

    batched = serving = layered = mh = p1 = None
    if rank == 0 and args.batch_sims > 0:
        batched = run_batch(hg, torch, args.batch_sims, args.batch_steps, stream, not args.no_autotune, fixed)
    persistent = None
    if rank == 0 and args.persistent_compare:
        bt = (batched or {}).get("tuning") or {}
        persistent = run_persistent(hg, torch, stream, tuning["table"] if tuning else hg.heat_tuning_get(),
                                    bt.get("table") or hg.heat_tuning_get())
    if rank == 0 and args.layered_steps > 0:
        layered = run_layered(hg, torch, args.layered_steps, stream, not (args.no_autotune or fixed),
                              cheb_degrees(args), args.cheb_ratio)
    if rank == 0 and args.mh_chains > 0:
        mh = run_mh(hg, torch, args.mh_chains, args.mh_iters, stream)
    if rank == 0 and args.p1_steps > 0:
        p1 = run_p1(hg, torch, args.p1_steps, stream, tuning["table"] if tuning else None)
    if rank == 0 and args.serve_requests > 0:
        serving = run_serving(hg, args.serve_requests, args.serve_rate, args.serve_budget_gb)
    serving_low = slab = None
    if rank == 0 and args.serve_low_requests > 0:
        serving_low = run_serving(hg, args.serve_low_requests, args.serve_low_rate, args.serve_budget_gb)
    if rank == 0 and args.slab_steps > 0:
        slab = run_slab(hg, torch, args.slab_steps, stream)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32_refined": "f32+df64+f64", "fp32_plain": "f32"}[args.precision],
            "dtype_detail": DTYPE_DETAIL[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision, "dof": nn,
                       "time_steps_per_forward_solve": args.nsteps, "cg_iterations_per_step_avg": its / (args.steps * args.nsteps),
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "flushed between timed steps (256 MiB overwrite)",
                       "kernel_tuning": tuning},
            "e2e": {"value": value_e2e, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * (2 * ne + nn), "d2h_bytes_per_step": 8 * nn},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "frac_of_nominal_7900_gbs": achieved / 7900.0,
                         "kernel": kernel_key.split("@")[0], "peak_kind": f"{peak_kind} HBM copy (burst)",
                         "ms_per_launch": prof["ms_apply"], "algorithmic_bytes_per_launch": prof["bytes_apply"],
                         "update_kernel": {"ms_per_launch": prof["ms_update"], "algorithmic_bytes_per_launch": prof["bytes_update"],
                                           "achieved": prof["bytes_update"] / (prof["ms_update"] * 1e-3) / 1e9}},
            "clocks": clocks,
            "fp64_path": fp64,
            "final_field_rel_err_vs_fp64_path": final_err,
            "batched": batched,
            "persistent_iteration": persistent,
            "layered": layered,
            "inverse_problem": mh,
            "tetrahedra": p1,
            "serving": serving,
            "serving_sustainable_rate": serving_low,
            "z_slabs": slab,
        }
        if cpu is not None:
            c = cpu["c_all_cores"]
            line["cpu_baseline"] = {
                "value": c["value"], "unit": UNIT, "cores": c["threads"], "kind": "oracle",
                "sample": (f"the oracle's C Jacobi-PCG (Algorithm 1, CSR, OpenMP on {c['threads']} threads of "
                           f"{cpu['cpu_model']}), first {cpu['steps']} time steps of the same workload "
                           f"({c['iters']} CG iterations, {c['seconds']:.2f} s in the solver; assembly and "
                           "right-hand sides untimed)"),
                "nproc": cpu["nproc"], "cpu_model": cpu["cpu_model"],
                "one_core": {"value": cpu["c_one_core"]["value"], "seconds": cpu["c_one_core"]["seconds"],
                             "kind": "oracle, C, 1 thread (the paper's one-core baseline)"},
                "python_one_core": {"value": cpu["python"]["value"], "seconds": cpu["python"]["seconds"],
                                    "kind": "oracle, NumPy/SciPy CSR, 1 thread"},
                "incomplete_cholesky_context": cpu.get("incomplete_factorisation")}
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
