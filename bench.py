#!/usr/bin/env python3
"""Throughput of the ARK4(3)6L[2]SA + HPS time step on one GB300: DOF x implicit stages / s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): u_t = 0.01 Lap u + u - u^3 on [0,1]^2, 64 x 64 leaves, p = 16
(N = 919,296 unknowns), dt = 1e-3, u0 ~ U[-0.1, 0.1].  A step is one full ARK step: the
explicit first stage, 5 implicit HPS stage solves, the ARK combination and the identity-
operator projection.  Two forms are timed: FP64 with one right-hand side (seed 0), and the
batched mixed-precision form (--rhs states, seeds 0..R-1; FP32 sweeps + --refine FP64
refinement sweeps per solve), whose columns 0 and R-1 are checked against the FP64 path
after the run.  The headline value is the mixed form when that error is <= 1e-10, else FP64:
value = R * N * 5 * K / (sum of the K step times), device-timed with CUDA events on the
launch stream; L2 (129 MB) is flushed by writing a 512 MB buffer before every timed step.  N > 1 (torchrun): independent replicas, one per GPU (the method
needs no exchange between them); value = all ranks' units / the max over ranks of the time.

--impl reference times the CPU oracle (oracle/, NumPy FP64) on the host cores on the same
workload: each step is one full-size stage solve (a bounded sample of an ARK step).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STAGES = 5  # implicit HPS solves per ARK4(3)6L[2]SA step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="allen_cahn_64x64_p16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eager", action="store_true", help="launch every kernel from the host (no CUDA graph)")
    ap.add_argument("--rhs", type=int, default=32, help="right-hand sides of the mixed-precision batch")
    ap.add_argument("--only", choices=["fp64", "mixed", "serving", "per-node-fp32", "many-instances"], default=None,
                    help="time one form only (profiling); serving: only the serving run; per-node-fp32: "
                         "--steps FP32 single-right-hand-side sweeps on the --per-node-workload handle")
    ap.add_argument("--serving-jobs", type=int, default=48, help="jobs of the serving run (0: skip)")
    ap.add_argument("--refine", type=int, default=1, help="FP64 refinement sweeps per implicit solve (mixed)")
    ap.add_argument("--groups", type=int, default=1, help="column groups of the mixed batch (own streams each)")
    ap.add_argument("--per-node-workload", default="varcoef_128x128_p16",
                    help="workload of the per-node-operator section (single-RHS HBM-bound solve, mixed vs FP64); "
                         "'none' skips it")
    ap.add_argument("--per-node-refine", type=int, default=2, help="refinement sweeps of its mixed ARK step")
    ap.add_argument("--instances", type=int, default=64, help="instances of the many-instance run (0: skip)")
    ap.add_argument("--per-node-umma", type=int, default=2, choices=[0, 1, 2],
                    help="its leaf applies on the tcgen05 tensor cores: 0 none, 1 first sweeps, 2 every sweep")
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-budget", type=float, default=12.0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-steps", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
SAMPLE_LEAVES = 64 * 64  # larger workloads are timed on a 32 x 32-leaf piece with the same p and coefficients


def oracle_setup(wname):
    import numpy as np
    from oracle.grid import Grid
    from oracle.hps import HPS
    from paper_2306_02526_gb300 import workloads
    wl = workloads.WORKLOADS[wname]
    n1, n2 = (wl.n1, wl.n2) if wl.n1 * wl.n2 <= SAMPLE_LEAVES else (32, 32)
    g = Grid(n1, n2, wl.p)
    X, Y = g.coords()
    I = np.arange(g.N_int)
    coef = wl.coef(X[I], Y[I])
    t0 = time.perf_counter()
    H = HPS(g, coef, 0.25 * wl.dt)
    build_s = time.perf_counter() - t0
    rhs = np.random.default_rng(1).uniform(-0.1, 0.1, g.N_int)
    return g, H, rhs, build_s


def cpu_sample(wname, budget, steps=0, warmup=0):
    """Time full-size oracle stage solves: `warmup` untimed, then `steps` timed (steps = 0: until
    `budget` seconds have passed, at least one)."""
    g, H, rhs, build_s = oracle_setup(wname)
    for _ in range(warmup):
        H.solve(rhs)
    n, t0 = 0, time.perf_counter()
    while True:
        H.solve(rhs)
        n += 1
        el = time.perf_counter() - t0
        if (steps and n >= steps) or (not steps and el >= budget):
            break
    return {"solves": n, "seconds": el, "N": g.N, "build_s": build_s, "leaves": "%dx%d" % (g.n1, g.n2)}


def run_cpu_sample_subprocess(wname, budget, threads=1, steps=0, warmup=0):
    """The oracle in a child process whose BLAS / OpenMP pools have `threads` threads."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", wname, "--cpu-budget", str(budget),
           "--cpu-steps", str(steps), "--warmup", str(warmup)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1200)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["threads"] = threads
    return out


def best_oracle_threads(wname, budget):
    """Short oracle samples with 1, 4 and all host threads in the BLAS pool; the fastest setting
    and every sample's rate (DOF x stage solves / s)."""
    cores = os.cpu_count() or 1
    rates = {}
    for th in sorted({1, min(4, cores), cores}):
        smp = run_cpu_sample_subprocess(wname, budget, th)
        rates[th] = smp["N"] * smp["solves"] / smp["seconds"]
    best = max(rates, key=rates.get)
    return best, rates


# ---------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi SM clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def fp64_dgemm_tflops(torch):
    """cuBLAS FP64 GEMM throughput (context for the FP64 ALU roofline)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def leaf_up_flops(N_int, q, b, m, nterms):
    """Algorithmic FP64 flops of one k_leaf_up launch: per leaf the q x q apply (2 q^2), the
    right-hand-side combination (2 q nterms) and the edge fluxes (2 b m)."""
    nleaf = N_int // q
    return nleaf * (2 * q * q + 2 * q * nterms + 2 * b * m)


def tree_levels(n1, n2, m):
    """(nodes, n3, nb) of every merge level, root first: boxes split across the longer side
    (ties: a vertical cut), interface n3 = short side x m, box boundary nb = 2 (a + c) m."""
    out, a, c, nodes = [], n1, n2, 1
    while a * c > 1:
        if a >= c:
            out.append((nodes, c * m, 2 * (a + c) * m))
            a //= 2
        else:
            out.append((nodes, a * m, 2 * (a + c) * m))
            c //= 2
        nodes *= 2
    return out


def solve_operator_elems(n1, n2, p):
    """Operator elements one single-RHS HPS solve with per-node operators reads (each once): per leaf
    A_ii^{-1} (q x q) and S (q x b); per merge node X (n3 x n3), S^t (n3 x nb) and [T^a_13; T^b_23]
    (nb x n3), the root without the last."""
    m = p - 2
    q, b = m * m, 4 * m
    lv = tree_levels(n1, n2, m)
    leaves = n1 * n2 * (q * q + q * b)
    merges = sum(nodes * (n3 * n3 + 2 * n3 * nb) for nodes, n3, nb in lv) - lv[0][1] * lv[0][2]
    return leaves, merges


def merge_flops_per_launch(slot, n1, n2, m, cols):
    """Average flops of one launch of a merge apply (one launch per level): w3 = X d (2 n3^2),
    h = hcat + Tcat w3 (2 nb n3, not at the root), u3 = S u_b + w3 (2 n3 nb), per node and column."""
    lv = tree_levels(n1, n2, m)
    if slot == "merge_up_w3":
        per = [nodes * 2 * n3 * n3 for nodes, n3, nb in lv]
    elif slot == "merge_up_h":
        per = [nodes * 2 * nb * n3 for nodes, n3, nb in lv[1:]]
    else:
        per = [nodes * 2 * n3 * nb for nodes, n3, nb in lv]
    return cols * sum(per) / max(1, len(per))


def fd_leaf_flops(N_int, q, b, m, nterms):
    """FP64 flops of one fast-diagonalization leaf apply: the right-hand-side combination
    (2 q nterms), four m-point line passes (8 m^3), the eigenvalue scaling (q) and the edge
    fluxes (2 b m), per leaf."""
    return N_int // q * (2 * q * nterms + 8 * m ** 3 + q + 2 * b * m)


def residual_flops(p, first, flux=True):
    """FP64 flops of the collocation residual R - (u - gamma dt L u) on one leaf and column, as the
    even-odd kernel evaluates it (p even, constant coefficients folded into the half matrices):
    the symmetric / antisymmetric line sums (2 m p), per orbit of four mirror points 2 lines x 2
    directions x (p/2 + p/2) multiply-adds plus 8 recombinations per derivative order, per point
    the sum of the scaled terms and the residual (3 flops, 2 more with first derivatives), and the
    flux sums of the four sides (per boundary line 2 x p/2 multiply-adds and 2 recombinations)."""
    m, h = p - 2, p // 2
    orders = 2 if first else 1
    return (2 * m * p + (h - 1) ** 2 * orders * (16 * h + 8) + m * m * (3 + (2 if first else 0)) +
            (2 * m * (4 * h + 2) if flux else 0))


def step_flops(n1, n2, p, R, refine, first, nstages=5):
    """Algorithmic flops of one batched mixed-precision ARK step (constant coefficients, edge-
    projection close), split by pipe.  FP64: the collocation residual of every refinement sweep
    (residual_flops), the explicit first-stage evaluation of L u^n and g (the residual's line sums
    without flux terms, plus 6 flops per point), the stage right-hand sides (2 flops per term after
    the leading u^n: 2 (i - 1) terms for stage i), the stage epilogue (6 flops per point: dt L U_i
    from the stage equation, dt g), the corrections u += du (1 per point and sweep) and the close
    (u + 6 explicit terms: 12 flops per point).  FP32: per sweep the fast-diagonalization leaf
    apply (8 m^3 per leaf), the leaf solve (2 q b per leaf) and the merge applies (2 n3^2 +
    2 nb n3 + 2 n3 nb per node, the root without h), all times R."""
    m = p - 2
    q, b = m * m, 4 * m
    leaves = n1 * n2
    n_int = leaves * q
    cols = leaves * R
    res = residual_flops(p, first, True)
    fp64 = (nstages * refine * cols * res
            + cols * (residual_flops(p, first, False) + 6 * q)
            + sum(2 * 2 * (i - 1) for i in range(2, nstages + 2)) * n_int * R
            + 6 * nstages * n_int * R
            + nstages * refine * n_int * R
            + 12 * n_int * R)
    lv = tree_levels(n1, n2, m)
    merge = sum(nodes * (2 * n3 * n3 + 2 * n3 * nb) for nodes, n3, nb in lv) + \
        sum(nodes * 2 * nb * n3 for nodes, n3, nb in lv[1:])
    sweeps = nstages * (1 + refine)
    fp32 = sweeps * R * (leaves * (8 * m ** 3 + 2 * q * b) + merge)
    return fp64, fp32


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------------------------
def max_over_ranks(x, world, device):
    """The largest value of x over all ranks (the job is as slow as its slowest replica)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, units_per_rank, max_ms):
    """Whole-job throughput of `world` independent replicas: all ranks' units over the max time."""
    return world * units_per_rank / (max_ms * 1e-3)


def timed_run(S, step, args, world, local_rank, flush, torch, events_in_region=True):
    """W warm-up steps, a traced pass for per-kernel shares, then K timed steps (L2 flushed
    before each, CUDA events on the launch stream, barrier + synchronize on both sides).  The
    dominant kernel is event-timed inside the timed region; with events_in_region False (a short,
    latency-bound step whose dominant kernel launches dozens of times per step: the events in the
    recorded graph lengthen the chain) the timed region runs without per-kernel events and the
    kernel is timed in a separate pass of the same steps right after it."""
    from paper_2306_02526_gb300 import _lib
    stream = torch.cuda.current_stream()
    n = 0
    for _ in range(args.warmup):
        step()
        n += 1
    S.trace_enable(_lib.KERNELS)
    for _ in range(2):  # eager + recording: the graph now carries timing events of every kernel
        step()
        n += 1
    S.trace_enable(_lib.KERNELS)  # same mask: counters reset, recorded graph kept
    for _ in range(4):
        step()
        n += 1
    shares = S.trace_read()
    dom = max(shares, key=lambda k: shares[k][2])
    # only the dominant kernel is event-timed in the timed region (all launches are counted);
    # two untimed steps record the graph that carries the new timing events
    S.trace_enable((dom,) if events_in_region else ())
    for _ in range(2):
        step()
        n += 1
    S.trace_enable((dom,) if events_in_region else ())
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
            n += 1
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tr = S.trace_read()
    launches = sum(v[0] for v in tr.values())
    if not events_in_region:
        S.trace_enable((dom,))
        for _ in range(2):
            step()
            n += 1
        S.trace_enable((dom,))
        for k in range(min(args.steps, 5)):
            flush.fill_(float(k))
            step()
            n += 1
        tr = S.trace_read()
    total_ms = max_over_ranks(sum(step_ms), world, "cuda")
    tot = sum(v[2] for v in shares.values()) or 1.0
    return {"total_ms": total_ms, "step_ms": step_ms, "wall": wall, "clocks": clk.summary(), "dom": dom,
            "dom_avg_ms": tr[dom][2] / max(1, tr[dom][1]), "launches": launches,
            "dom_timing": "in the timed region" if events_in_region else "separate pass of %d steps" % min(args.steps, 5),
            "shares": {k: round(v[2] / tot, 4) for k, v in shares.items() if v[2] > 0}, "steps_done": n}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernels,
# from the ncu captures summarised under profiles/; an entry is removed when its kernel changes.
NCU_TRAFFIC = {
    ("allen_cahn_64x64_p16", "fp64", "leaf_up"): 45.56e6,
    ("allen_cahn_64x64_p16", "mixed", "residual"): 694.1e6,
}


def p99(xs):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(math.ceil(0.99 * len(xs))) - 1)]


def bench_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2306_02526_gb300 import build as _b
    from paper_2306_02526_gb300 import hps, workloads

    torch.cuda.set_device(local_rank)
    if rank == 0:
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    wl = workloads.WORKLOADS[args.workload]
    tree = hps.Tree(wl.n1, wl.n2)
    N, N_int, N_bd = hps.hps_sizes(tree, wl.p)
    x, y = hps.hps_coords(tree, wl.p)
    bidx = hps.hps_boundary_index(tree, wl.p)
    I = np.arange(N_int)
    coef = wl.coef(x[I], y[I])
    cdev = {k: (torch.tensor(v, dtype=torch.float64, device="cuda") if np.ndim(v) else float(v))
            for k, v in coef.items()}
    t0 = time.perf_counter()
    S = hps.HPSSolver(tree, wl.p, cdev, 0.25 * wl.dt)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    c = hps.hps_ark_abscissae()
    R = args.rhs

    def stage_terms(cols):
        # synthetic workload: the stage data of the first step, held fixed (the bench workload has none)
        q = f = None
        if wl.q(x[:1], y[:1], 0.0) is not None:
            qs = np.stack([wl.q(x[I], y[I], cj * wl.dt) for cj in c])
            q = torch.tensor(np.repeat(qs[:, :, None], cols, axis=2) if cols > 1 else qs, dtype=torch.float64,
                             device="cuda").reshape(-1)
        if wl.f(x[:1], y[:1], 0.0) is not None:
            fs = np.stack([wl.f(x[bidx], y[bidx], cj * wl.dt) for cj in c])
            f = torch.tensor(np.repeat(fs[:, :, None], cols, axis=2) if cols > 1 else fs, dtype=torch.float64,
                             device="cuda").reshape(-1)
        return q, f

    q1, f1 = stage_terms(1)
    qR, fR = stage_terms(R)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    if not args.eager:
        S.set_graph(True)  # each ARK step is replayed from a recorded CUDA graph
    u0 = wl.u0(x, y, bidx)

    def fp64_steps(uu, nsteps):
        for _ in range(nsteps):
            S.ark_step(uu, 0.0, wl.dt, q=q1, f=f1, g=wl.g, g_param=wl.g_param)

    # ---- FP64, one right-hand side -----------------------------------------------------------
    if args.only == "mixed":
        args_short = argparse.Namespace(**vars(args))
        args_short.steps, args_short.warmup = 2, 1
        u = torch.tensor(u0, dtype=torch.float64, device="cuda")
        r64 = timed_run(S, lambda: fp64_steps(u, 1), args_short, world, local_rank, flush, torch, False)
        value64 = replica_value(world, N * STAGES * 2, r64["total_ms"])
    else:
        u = torch.tensor(u0, dtype=torch.float64, device="cuda")
        r64 = timed_run(S, lambda: fp64_steps(u, 1), args, world, local_rank, flush, torch, False)
        assert torch.isfinite(u).all(), "FP64 solution went non-finite"
        value64 = replica_value(world, N * STAGES * args.steps, r64["total_ms"])
    if args.only == "fp64":
        args.rhs = R = 4
        args.steps, args.warmup = 2, 1
        qR, fR = stage_terms(R)

    # ---- slope form, FP64: the workload itself (eq. slope with its g when its boundary data are
    # time-independent), else its linear part ------------------------------------------------------
    slope = None
    slope_g = wl.g if f1 is None and fR is None else None
    slope_kw = {"g": slope_g, "g_param": wl.g_param} if slope_g else {}
    if args.only is None:
        us = torch.tensor(u0, dtype=torch.float64, device="cuda")
        for _ in range(3):
            S.ark_slope_step(us, 0.0, wl.dt, **slope_kw)
        torch.cuda.synchronize()
        se = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
        for k in range(10):
            flush.fill_(float(k))
            se[k][0].record(stream)
            S.ark_slope_step(us, 0.0, wl.dt, **slope_kw)
            se[k][1].record(stream)
        torch.cuda.synchronize()
        sms = [a.elapsed_time(b) for a, b in se]
        assert torch.isfinite(us).all(), "slope-form state went non-finite"
        slope = {"value": N * STAGES * len(sms) / (sum(sms) * 1e-3), "unit": "DOF*stages/s",
                 "ms_per_step": sum(sms) / len(sms), "steps": len(sms), "launch": "eager",
                 "g": slope_g,
                 "note": "slope form with penalized interface rows (eq. slope: explicit slopes for g, zero "
                         "slope boundary data), same grid and operators, FP64, L2 flushed before every step"}

    # ---- mixed precision, R right-hand sides (FP32 sweeps + FP64 refinement) ----------------------
    S.batch_reserve(R, groups=args.groups)
    U0 = np.stack([u0] + [workloads.uniform_state(j, N, bidx) for j in range(1, R)], axis=1)
    U = torch.tensor(U0, dtype=torch.float64, device="cuda")

    def mixed_step(uu):
        S.ark_step_batch(uu, 0.0, wl.dt, q=qR, f=fR, g=wl.g, g_param=wl.g_param, refine=args.refine)

    rmx = timed_run(S, lambda: mixed_step(U), args, world, local_rank, flush, torch)
    assert torch.isfinite(U).all(), "mixed solution went non-finite"

    # ---- slope form, R states, mixed precision (g = 0: the workload's linear part) ----------------
    slope_mixed = None
    if args.only is None and args.groups == 1:
        Us = torch.tensor(U0, dtype=torch.float64, device="cuda")
        for _ in range(3):
            S.ark_slope_step_batch(Us, 0.0, wl.dt, refine=2, **slope_kw)
        torch.cuda.synchronize()
        se = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
        for k in range(10):
            flush.fill_(float(k))
            se[k][0].record(stream)
            S.ark_slope_step_batch(Us, 0.0, wl.dt, refine=2, **slope_kw)
            se[k][1].record(stream)
        torch.cuda.synchronize()
        sms = [a.elapsed_time(b) for a, b in se]
        assert torch.isfinite(Us).all(), "batched slope-form state went non-finite"
        # one step from the same states against the FP64 slope step, first and last column
        Us = torch.tensor(U0, dtype=torch.float64, device="cuda")
        S.ark_slope_step_batch(Us, 0.0, wl.dt, refine=2, **slope_kw)
        serr = 0.0
        for j in (0, R - 1):
            v = torch.tensor(np.ascontiguousarray(U0[:, j]), dtype=torch.float64, device="cuda")
            S.ark_slope_step(v, 0.0, wl.dt, **slope_kw)
            serr = max(serr, float((Us[:, j] - v).abs().max() / v.abs().max()))
        slope_mixed = {"value": N * STAGES * R * len(sms) / (sum(sms) * 1e-3), "unit": "DOF*stages/s",
                       "ms_per_step": sum(sms) / len(sms), "steps": len(sms), "rhs": R, "refine": 2,
                       "err_vs_fp64_slope": serr, "err_columns": [0, R - 1],
                       "over_fp64_slope": None if not slope else
                       N * STAGES * R * len(sms) / (sum(sms) * 1e-3) / slope["value"],
                       "g": slope_g,
                       "note": "ark_slope_step_batch: FP32 sweeps + 2 FP64 refinement sweeps per slope system "
                               "(interface rows carry the penalization), CUDA graph replay, L2 flushed before "
                               "every step"}
    value_mixed = replica_value(world, R * N * STAGES * args.steps, rmx["total_ms"])
    # accuracy: columns 0 and R-1 against the FP64 path run for the same number of steps
    errs = []
    for j in sorted({0, R - 1}):
        ref = torch.tensor(U0[:, j].copy(), dtype=torch.float64, device="cuda")
        fp64_steps(ref, rmx["steps_done"])
        errs.append(float((U[:, j] - ref).abs().max() / ref.abs().max()))
    err_mixed = max(errs)

    # ---- end to end through the C ABI with HOST buffers (ark_step_host / ark_step_batch_host:
    # host -> device copy of the states, the step, device -> host copy, all inside the call) ----
    def e2e(step_host, host_u):
        ms = []
        for k in range(max(5, min(args.steps, 20)) + 2):
            flush.fill_(float(k))  # L2 flushed before every step, as in the device-timed runs
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step_host(host_u)
            b.record(stream)
            b.synchronize()
            if k >= 2:
                ms.append(a.elapsed_time(b))
        return statistics.mean(ms), len(ms)

    e64_ms, e_n = e2e(lambda hu: S.ark_step_host(hu, 0.0, wl.dt, q=q1, f=f1, g=wl.g, g_param=wl.g_param),
                      torch.tensor(u0, dtype=torch.float64).pin_memory())
    emx_ms, _ = e2e(lambda hu: S.ark_step_batch_host(hu, 0.0, wl.dt, q=qR, f=fR, g=wl.g, g_param=wl.g_param,
                                                     refine=args.refine),
                    torch.tensor(U0, dtype=torch.float64).pin_memory())

    out = None
    if rank == 0:
        q, b, m = (wl.p - 2) ** 2, 4 * (wl.p - 2), wl.p - 2
        nleaf = N_int // q
        sm_mhz = rmx["clocks"]["sm_mhz"] or 2070.0
        peak_fp64 = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12   # 2 DFMA / SM / cycle (ncu peak_sustained)
        peak_fp32 = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # 128 FP32 lanes / SM
        dgemm = fp64_dgemm_tflops(torch)

        def roofline(run, mixed):
            dom = run["dom"]
            roof = {"kernel": dom, "bound": "alu", "unit": "TFLOP/s",
                    "traffic": NCU_TRAFFIC.get((wl.name, "mixed" if mixed else "fp64", dom)),
                    "avg_launch_ms": run["dom_avg_ms"], "timing": run["dom_timing"]}
            fl, pk, src = None, None, None
            if dom == "leaf_up" and not mixed:
                fl = (fd_leaf_flops(N_int, q, b, m, 11) if S.batch_option("fast_diag") and not S.nodal
                      else leaf_up_flops(N_int, q, b, m, 11))
                pk, src = peak_fp64, "FP64"
            elif dom in ("merge_up_w3", "merge_up_h", "merge_down"):  # latency-bound applies, average launch
                fl = merge_flops_per_launch(dom, wl.n1, wl.n2, m, R if mixed else 1)
                pk, src = (peak_fp32, "FP32") if mixed else (peak_fp64, "FP64")
            elif dom == "leaf_up" and mixed:
                fl, pk, src = nleaf * 2 * q * q * R, peak_fp32, "FP32"
            elif dom == "residual" and mixed:  # FP64 residual by the even-odd evaluation of L u
                first = S.nodal or any(float(coef.get(k_, 0.0)) != 0.0 for k_ in ("a1", "a2") if np.ndim(coef.get(k_, 0.0)) == 0)
                fl, pk, src = nleaf * R * residual_flops(wl.p, first, bool(S.batch_option("fuse_jump"))), peak_fp64, "FP64"
            if fl is not None:
                roof.update({"flops_per_launch": fl, "achieved": fl / (run["dom_avg_ms"] * 1e-3) / 1e12, "peak": pk,
                             "peak_source": "%s units x clocks: 152 SMs x %s x %.0f MHz (cuBLAS DGEMM measured "
                                            "%.3f TFLOP/s)" % (src, "2 DFMA" if src == "FP64" else "128 FMA lanes",
                                                              sm_mhz, dgemm)})
                roof["frac"] = roof["achieved"] / pk
            return roof

        fp64 = {"value": value64, "ms_per_step": r64["total_ms"] / args.steps,
                "p50_step_ms": statistics.median(r64["step_ms"]), "p99_step_ms": p99(r64["step_ms"]),
                "roofline": roofline(r64, False), "kernel_shares": r64["shares"], "gpu_launches": r64["launches"],
                "e2e": {"value": N * STAGES / (e64_ms * 1e-3), "unit": "DOF*stages/s", "h2d_bytes_per_step": N * 8,
                        "d2h_bytes_per_step": N * 8, "steps": e_n},
                "clocks": r64["clocks"]}
        mixed_ok = err_mixed <= 1e-10
        head = rmx if mixed_ok else r64
        step_roofline = None
        if mixed_ok and not S.nodal:  # the whole step against the pipe that bounds it
            first = any(float(coef.get(k_, 0.0)) != 0.0 for k_ in ("a1", "a2"))
            f64, f32 = step_flops(wl.n1, wl.n2, wl.p, R, args.refine, first)
            ms = head["total_ms"] / args.steps
            t64, t32 = f64 / (peak_fp64 * 1e12) * 1e3, f32 / (peak_fp32 * 1e12) * 1e3
            step_roofline = {"bound": "alu", "pipe": "FP64" if t64 >= t32 else "FP32",
                             "fp64_gflop": f64 / 1e9, "fp32_gflop": f32 / 1e9, "ideal_ms": max(t64, t32),
                             "ms_per_step": ms, "frac": max(t64, t32) / ms,
                             "note": "algorithmic flops of the step (bench.step_flops) at the unit-count peaks "
                                     "(FP64 %.3f, FP32 %.1f TFLOP/s); ideal = the slower pipe's time, the FP32 "
                                     "sweeps assumed to overlap it" % (peak_fp64, peak_fp32)}
        out = {
            "metric": "DOF*stages/s (N x implicit HPS stage solves per second, ARK4(3)6L[2]SA step)",
            "value": value_mixed if mixed_ok else value64, "unit": "DOF*stages/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["total_ms"] / args.steps, "p50_step_ms": statistics.median(head["step_ms"]),
            "p99_step_ms": p99(head["step_ms"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 sweeps + f64 refinement" if mixed_ok else "f64",
            "data": "synthetic (seeded u0 ~ U[-0.1,0.1], one seed per right-hand side)",
            "config": {"workload": wl.name, "n1": wl.n1, "n2": wl.n2, "p": wl.p, "N": N,
                       "p2n1n2": wl.p ** 2 * wl.n1 * wl.n2, "dt": wl.dt, "stages_per_step": STAGES,
                       "rhs": R if mixed_ok else 1, "refine": args.refine if mixed_ok else 0,
                       "column_groups": args.groups if mixed_ok else 1,
                       "operators": "one per tree node (nodal coefficients)" if S.nodal else
                                    "one per tree level (constant coefficients)",
                       "l2": "flushed (512 MB write) before every timed step",
                       "launch": "eager" if args.eager else "CUDA graph replay (hps_set_graph)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "err_vs_fp64": err_mixed,
            "roofline": roofline(head, mixed_ok),
            "step_roofline": step_roofline,
            "kernel_shares": head["shares"],
            "gpu_launches": head["launches"],
            "e2e": ({"value": R * N * STAGES / (emx_ms * 1e-3), "unit": "DOF*stages/s",
                     "h2d_bytes_per_step": N * R * 8, "d2h_bytes_per_step": N * R * 8, "steps": e_n}
                    if mixed_ok else fp64["e2e"]),
            "clocks": head["clocks"],
            "fp64_single_rhs": fp64,
            "fp64_slope_form": slope,
            "mixed_slope_form": slope_mixed,
            "fp32_single_rhs_solve": None,
            "mixed_over_fp64": value_mixed / value64,
            "build_s": build_s, "wall_s": head["wall"],
        }
    S.close()
    if rank == 0 and out is not None and args.only is None and args.per_node_workload != "none":
        out["per_node"] = bench_per_node(args, flush)
    if rank == 0 and out is not None and args.only is None and args.instances > 0:
        out["many_instances"] = bench_multi(args, flush)
        pn = out["per_node"]
        out["fp32_single_rhs_solve"] = pn["fp32_sweep_solve"]
    if rank == 0 and out is not None and args.serving_jobs > 0 and args.only is None:
        out["serving"] = bench_serving(args)
        out["serving"]["batched_over_plain_fp64_sweep"] = (out["serving"]["batched_mixed"]["dof_stages_per_s"] /
                                                           out["fp64_single_rhs"]["value"])
    return out


def per_node_fp32_sweeps(args):
    """Profiling form: --warmup + --steps FP32 sweeps with one right-hand side (hps_solve_batch,
    R = 1, no refinement) on the per-node-operator handle of --per-node-workload, eager launches."""
    import numpy as np
    import torch
    from paper_2306_02526_gb300 import build as _b
    from paper_2306_02526_gb300 import hps, workloads
    _b.build()
    wl = workloads.WORKLOADS[args.per_node_workload]
    tree = hps.Tree(wl.n1, wl.n2)
    N, N_int, N_bd = hps.hps_sizes(tree, wl.p)
    x, y = hps.hps_coords(tree, wl.p)
    I = np.arange(N_int)
    coef = {k: torch.tensor(np.broadcast_to(v, (N_int,)).copy(), dtype=torch.float64, device="cuda")
            for k, v in wl.coef(x[I], y[I]).items()}
    S = hps.HPSSolver(tree, wl.p, coef, 0.25 * wl.dt)
    S.batch_reserve(1)
    rhs = torch.tensor(np.random.default_rng(3).uniform(-0.1, 0.1, (N_int, 1)), dtype=torch.float64, device="cuda")
    u = torch.empty((N, 1), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        S.solve_batch(rhs, u=u, refine=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.solve_batch(rhs, u=u, refine=0)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / max(1, args.steps)
    S.close()
    return {"workload": wl.name, "N": N, "sweeps": args.steps, "ms_per_sweep_wall": ms}


def bench_per_node(args, flush):
    """Per-node operators (variable coefficients, 128 x 128 leaves, p = 16 by default), one GPU:
      * single-RHS solves, each with the L2 flushed before it: the FP64 HPS solve; one FP32 sweep
        (hps_solve_batch, R = 1, no refinement); the refined FP32 solve (1 FP64 refinement sweep);
        whole-solve rooflines from the algorithmic bytes (operators read once + 6 N vector words),
        the FP64 one against min(HBM, FP64 pipe) time;
      * the ARK step: FP64 with one state against the batched mixed-precision step with --rhs states
        and --per-node-refine refinement sweeps, error of columns 0 and R-1 against the FP64 path."""
    import numpy as np
    import torch
    from paper_2306_02526_gb300 import hps, workloads
    wl = workloads.WORKLOADS[args.per_node_workload]
    tree = hps.Tree(wl.n1, wl.n2)
    N, N_int, N_bd = hps.hps_sizes(tree, wl.p)
    x, y = hps.hps_coords(tree, wl.p)
    bidx = hps.hps_boundary_index(tree, wl.p)
    I = np.arange(N_int)
    coef = wl.coef(x[I], y[I])
    cdev = {k: torch.tensor(np.broadcast_to(v, (N_int,)).copy(), dtype=torch.float64, device="cuda")
            for k, v in coef.items()}
    t0 = time.perf_counter()
    S = hps.HPSSolver(tree, wl.p, cdev, 0.25 * wl.dt)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    S.set_graph(True)
    stream = torch.cuda.current_stream()
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    peak_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in measured_peaks() else "fallback 6800 GB/s"
    leaves, merges = solve_operator_elems(wl.n1, wl.n2, wl.p)

    def timed(fn, n, trace=()):
        for _ in range(3):
            fn()
        S.trace_enable(trace)
        for _ in range(2):  # eager + recording (the graph then carries the trace events)
            fn()
        S.trace_enable(trace)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], S.trace_read()

    def shares(fn, n=3):
        from paper_2306_02526_gb300 import _lib
        _, tr = timed(fn, n, _lib.KERNELS)
        tot = sum(v[2] for v in tr.values()) or 1.0
        return {k: {"launches": v[0] // n, "ms": round(v[2] / n, 4), "share": round(v[2] / tot, 4)}
                for k, v in tr.items() if v[0]}

    out = {"workload": wl.name, "n1": wl.n1, "n2": wl.n2, "p": wl.p, "N": N, "build_s": build_s,
           "operators": "one per tree node (nodal coefficients)",
           "operator_elements": {"leaves": leaves, "merges": merges, "leaf_share": leaves / (leaves + merges)}}
    rhs = torch.tensor(np.random.default_rng(3).uniform(-0.1, 0.1, N_int), dtype=torch.float64, device="cuda")
    u64 = torch.empty(N, dtype=torch.float64, device="cuda")
    # ---- FP64 single-RHS solve ----
    ms64, _ = timed(lambda: S.solve(rhs, u=u64), 10)
    t64 = statistics.mean(ms64)
    flops = 2.0 * (leaves + merges)
    sm_mhz = 2070.0
    peak_fp64 = 152 * 2 * 2 * sm_mhz * 1e6
    bytes64 = (leaves + merges + 6 * N) * 8
    t_ideal = max(bytes64 / (hbm * 1e9), flops / peak_fp64)
    out["fp64_solve"] = {
        "ms": t64, "value": N / (t64 * 1e-3), "unit": "DOF*solves/s",
        "roofline": {"bound": "alu" if flops / peak_fp64 > bytes64 / (hbm * 1e9) else "hbm",
                     "bytes": bytes64, "flops": flops, "ideal_ms": t_ideal * 1e3, "frac": t_ideal * 1e3 / t64,
                     "achieved_gbs": bytes64 / (t64 * 1e-3) / 1e9, "achieved_tflops": flops / (t64 * 1e-3) / 1e12,
                     "peak_gbs": hbm, "peak_tflops": peak_fp64 / 1e12,
                     "peak_source": "%s; FP64 152 SMs x 2 DFMA x 2 flop x %.0f MHz" % (peak_src, sm_mhz),
                     "note": "ideal time = max(bytes / HBM, flops / FP64 pipe); frac = ideal / measured"},
        "kernel_shares": shares(lambda: S.solve(rhs, u=u64))}
    # ---- FP32 sweeps, one right-hand side (the HBM-bound form) ----
    S.batch_reserve(1)
    r1 = rhs.reshape(N_int, 1).contiguous()
    ub = torch.empty((N, 1), dtype=torch.float64, device="cuda")
    bytes32 = (leaves + merges) * 4 + 6 * N * 4
    for refine in (0, 1):
        ms32, tr = timed(lambda: S.solve_batch(r1, u=ub, refine=refine), 10, ("leaf_up",))
        t32 = statistics.mean(ms32)
        err = float((ub[:, 0] - u64).abs().max() / u64.abs().max())
        alg = bytes32 * (refine + 1) + refine * (N_int * 5 + 3 * N) * 8  # + the FP64 residual's vectors
        up_ms = tr["leaf_up"][2] / max(1, tr["leaf_up"][1])
        q_, b_ = (wl.p - 2) ** 2, 4 * (wl.p - 2)
        up_bytes = wl.n1 * wl.n2 * (q_ * ((q_ + 3) // 4 * 4) * 4 + q_ * 8 + q_ * 4 + b_ * 4)
        out["fp32_sweep_solve" if refine == 0 else "fp32_refined_solve"] = {
            "ms": t32, "refine": refine, "err_vs_fp64": err, "value": N / (t32 * 1e-3), "unit": "DOF*solves/s",
            "roofline": {"bound": "hbm", "unit": "GB/s", "bytes": alg, "achieved": alg / (t32 * 1e-3) / 1e9,
                         "peak": hbm, "peak_source": peak_src, "frac": alg / (t32 * 1e-3) / 1e9 / hbm,
                         "note": "bytes = %d sweep(s) x (FP32 operators read once + 6 N FP32 vector words)%s"
                                 % (refine + 1, " + the FP64 residual's vectors" if refine else "")},
            "leaf_up": {"avg_launch_ms": up_ms, "bytes_per_launch": up_bytes,
                        "achieved": up_bytes / (up_ms * 1e-3) / 1e9, "frac": up_bytes / (up_ms * 1e-3) / 1e9 / hbm},
            "kernel_shares": shares(lambda: S.solve_batch(r1, u=ub, refine=refine))}
    # ---- ARK step: FP64 (1 state) vs batched mixed precision (R states) ----
    c = hps.hps_ark_abscissae()
    qs = None
    if wl.q(x[:1], y[:1], 0.0) is not None:
        qs = np.stack([wl.q(x[I], y[I], cj * wl.dt) for cj in c])
    q1 = None if qs is None else torch.tensor(qs.reshape(-1), dtype=torch.float64, device="cuda")
    u0 = wl.u0(x, y, bidx)
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    step64 = lambda uu: S.ark_step(uu, 0.0, wl.dt, q=q1, g=wl.g, g_param=wl.g_param)
    ms_s64, _ = timed(lambda: step64(u), 5)
    R = args.rhs
    S.batch_reserve(R)
    S.batch_option("umma_leaf", args.per_node_umma)  # tensor-core leaf applies (per-node operators)
    qR = None if qs is None else torch.tensor(np.repeat(qs[:, :, None], R, axis=2), dtype=torch.float64,
                                              device="cuda")
    U0 = np.stack([u0] + [workloads.uniform_state(j, N, bidx) for j in range(1, R)], axis=1)
    U = torch.tensor(U0, dtype=torch.float64, device="cuda")
    stepmx = lambda: S.ark_step_batch(U, 0.0, wl.dt, q=qR, g=wl.g, g_param=wl.g_param, refine=args.per_node_refine)
    ms_mx, _ = timed(stepmx, 5)
    nsteps = 3 + 2 + 5
    errs = []
    ref = torch.empty(N, dtype=torch.float64, device="cuda")
    for j in sorted({0, R - 1}):
        ref.copy_(torch.from_numpy(U0[:, j].copy()))
        for _ in range(nsteps):
            step64(ref)
        errs.append(float((U[:, j] - ref).abs().max() / ref.abs().max()))
    v64 = N * STAGES / (statistics.mean(ms_s64) * 1e-3)
    vmx = R * N * STAGES / (statistics.mean(ms_mx) * 1e-3)
    out["ark_step"] = {"fp64": {"value": v64, "unit": "DOF*stages/s", "ms_per_step": statistics.mean(ms_s64),
                                "p50_step_ms": statistics.median(ms_s64), "steps": len(ms_s64)},
                       "mixed": {"value": vmx, "unit": "DOF*stages/s", "ms_per_step": statistics.mean(ms_mx),
                                 "p50_step_ms": statistics.median(ms_mx), "steps": len(ms_mx), "rhs": R,
                                 "refine": args.per_node_refine, "err_vs_fp64": max(errs),
                                 "umma_leaf": args.per_node_umma,
                                 "err_columns": sorted({0, R - 1}), "steps_compared": nsteps},
                       "mixed_over_fp64": vmx / v64,
                       "mixed_kernel_shares": shares(stepmx, 2)}
    out["l2"] = "flushed (512 MB write) before every timed solve / step"
    out["launch"] = "CUDA graph replay (hps_set_graph)"
    S.close()
    return out


def bench_multi(args, flush):
    """Many independent instances of uneven sizes (workloads.instances: 64 seeded reaction-diffusion
    instances, leaf grids 16^2..64^2, p in {8, 12, 16}, per-node operators), --rhs states each,
    advanced together by hps_multi_ark_step (every instance's batched mixed-precision step on its
    own stream, the whole step one CUDA graph), tensor-core leaf applies in every sweep and
    --per-node-refine refinement sweeps; the same steps with the instances one after another on
    one stream for comparison; columns 0 and R-1 of four instances against the FP64 path."""
    import numpy as np
    import torch
    from paper_2306_02526_gb300 import hps, workloads
    ins = workloads.instances(count=args.instances)
    R = args.rhs
    t0 = time.perf_counter()
    solvers, states, U0s, Ns = [], [], [], []
    op_bytes = 0
    for w in ins:
        tree = hps.Tree(w.n1, w.n2)
        N, N_int, _ = hps.hps_sizes(tree, w.p)
        x, y = hps.hps_coords(tree, w.p)
        bd = hps.hps_boundary_index(tree, w.p)
        coef = {k: torch.tensor(v, dtype=torch.float64, device="cuda") for k, v in w.coef(x[:N_int], y[:N_int]).items()}
        S = hps.HPSSolver(tree, w.p, coef, 0.25 * w.dt)
        S.batch_reserve(R)
        S.batch_option("umma_leaf", args.per_node_umma)
        op_bytes += hps.hps_bytes(tree, w.p, nodal=True)
        U0 = np.stack([workloads.uniform_state(1000 * len(solvers) + j, N, bd) for j in range(R)], axis=1)
        solvers.append(S)
        U0s.append(U0)
        states.append(torch.tensor(U0, dtype=torch.float64, device="cuda"))
        Ns.append(N)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    M = hps.MultiStep(solvers)
    M.set_graph(True)
    stream = torch.cuda.current_stream()
    dt, gk = ins[0].dt, dict(g="allen_cahn", g_param=(1.0, 0.0))
    step = lambda: M.ark_step(states, dt, refine=args.per_node_refine, **gk)
    nwarm, ntimed = 3, max(3, min(args.steps, 5))
    for _ in range(nwarm):
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ntimed)]
    for k in range(ntimed):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    # the same step in lockstep: one grouped merge launch per tree level for all instances
    M.set_lockstep(True)
    for _ in range(nwarm):
        step()
    lev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ntimed)]
    for k in range(ntimed):
        flush.fill_(float(k))
        lev[k][0].record(stream)
        step()
        lev[k][1].record(stream)
    torch.cuda.synchronize()
    lock_ms = [a.elapsed_time(b) for a, b in lev]
    M.set_lockstep(False)
    # the same step with the instances one after another on the caller's stream (no graph)
    M.set_graph(False)
    seq = []
    for k in range(2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(float(k))
        a.record(stream)
        for S, u in zip(solvers, states):
            S.ark_step_batch(u, 0.0, dt, refine=args.per_node_refine, **gk)
        b.record(stream)
        b.synchronize()
        seq.append(a.elapsed_time(b))
    nsteps = 2 * (nwarm + ntimed) + 2
    errs = []
    for i in range(0, len(solvers), max(1, len(solvers) // 4)):
        S = solvers[i]
        ref = torch.empty(Ns[i], dtype=torch.float64, device="cuda")
        for j in sorted({0, R - 1}):
            ref.copy_(torch.from_numpy(U0s[i][:, j].copy()))
            for n in range(nsteps):
                S.ark_step(ref, n * dt, dt, **gk)
            errs.append(float((states[i][:, j] - ref).abs().max() / ref.abs().max()))
    M.close()
    for S in solvers:
        S.close()
    units = sum(Ns) * R * STAGES
    return {"instances": len(ins), "rhs_each": R, "sum_N": sum(Ns), "leaf_grids": sorted({w.n1 for w in ins}),
            "orders": sorted({w.p for w in ins}), "operators": "one per tree node (seeded coefficients)",
            "operator_bytes_fp64": op_bytes, "build_s": build_s,
            "value": units / (statistics.mean(ms) * 1e-3), "unit": "DOF*stages/s",
            "ms_per_step": statistics.mean(ms), "steps": ntimed,
            "launch": "one CUDA graph per step for all instances (hps_multi_set_graph)",
            "lockstep_ms_per_step": statistics.mean(lock_ms),
            "lockstep": "hps_multi_set_lockstep: grouped merge launches per tree level, one graph per step",
            "sequential_ms_per_step": statistics.mean(seq),
            "concurrent_over_sequential": statistics.mean(seq) / statistics.mean(ms),
            "refine": args.per_node_refine, "umma_leaf": args.per_node_umma,
            "err_vs_fp64": max(errs), "err_sample": "columns 0 and R-1 of every %d-th instance after %d steps"
                                                    % (max(1, len(solvers) // 4), nsteps),
            "l2": "flushed before every timed step"}


# operations the serving stream draws from (leaf grid, p, kind): heat u_t = Lap u (dt = 0.01) or
# Allen-Cahn u_t = 0.01 Lap u + u - u^3 (dt = 1e-3), spanning leaf grids 8x8 .. 128x128 and p 8 .. 16
SERVING_CATALOG = ((8, 8, "heat"), (16, 12, "ac"), (32, 16, "heat"), (64, 16, "ac"), (128, 8, "heat"),
                   (64, 12, "ac"), (32, 12, "varcoef_src"))


class _SeparableSource:
    """q(x, t) = Q(x) cos(t) (Q resident on the device), f = 0: the per-step fill of a served job
    with variable coefficients, six scaled copies on the job's stream."""

    def __init__(self, Q, c):
        self.Q, self.c = Q, c

    def __call__(self, t, dt, q, f):
        import math
        import torch
        w = torch.tensor([math.cos(t + cj * dt) for cj in self.c], dtype=torch.float64).to(q.device, non_blocking=True)
        torch.mul(w[:, None], self.Q[None, :], out=q)
        f.zero_()


def serving_jobs(n_jobs, seed=2026):
    """A seeded Poisson-arrival stream (200 jobs/s) of jobs drawn uniformly from SERVING_CATALOG,
    10..500 steps each, initial states U[-0.1, 0.1] (zero on the boundary); 'varcoef_src' jobs have
    nodal coefficients and a source q = sin(pi x) sin(pi y) cos(t) filled on the device per step."""
    import numpy as np
    from paper_2306_02526_gb300 import hps
    r = np.random.default_rng(seed)
    t, jobs = 0.0, []
    for _ in range(n_jobs):
        t += r.exponential(1.0 / 200.0)
        n, p, kind = SERVING_CATALOG[int(r.integers(len(SERVING_CATALOG)))]
        tree = hps.Tree(n, n)
        N, _, _ = hps.hps_sizes(tree, p)
        bd = hps.hps_boundary_index(tree, p)
        u0 = r.uniform(-0.1, 0.1, N)
        u0[bd] = 0.0
        steps = int(r.integers(10, 501))
        if kind == "heat":
            jobs.append(dict(tree=tree, p=p, coef={"a11": 1.0, "a22": 1.0}, dt=0.01, steps=steps, u0=u0,
                             arrival_s=t))
        elif kind == "varcoef_src":  # nodal coefficients (one seeded field for all such jobs) and a source
            import torch
            x, y = hps.hps_coords(tree, p)
            N_int = hps.hps_sizes(tree, p)[1]
            xi, yi = x[:N_int], y[:N_int]
            coef = {"a11": 0.02 * (1.0 + 0.5 * np.sin(3 * xi) * np.cos(2 * yi)), "a22": 0.02 * (1.0 + 0.3 * xi * yi),
                    "a1": 0.05 * np.cos(yi), "a0": -0.1 + 0.0 * xi}
            Q = torch.tensor(np.sin(np.pi * xi) * np.sin(np.pi * yi), dtype=torch.float64, device="cuda")
            jobs.append(dict(tree=tree, p=p, coef=coef, dt=1e-3, steps=steps, u0=u0, g="fisher", g_param=(0.5, 0.0),
                             arrival_s=t, terms=_SeparableSource(Q, hps.hps_ark_abscissae())))
        else:
            jobs.append(dict(tree=tree, p=p, coef={"a11": 0.01, "a22": 0.01}, dt=1e-3, steps=steps, u0=u0,
                             g="allen_cahn", g_param=(1.0, 0.0), arrival_s=t))
    return jobs


def bench_serving(args):
    """The serving stream through the native loop twice: every job stepping alone in FP64, and
    jobs of the same operation coalesced into batched mixed-precision steps (up to 32 columns,
    refinement sweeps chosen per operation by the server from its stiffness).  The batched results are compared with the FP64 ones job by job."""
    import numpy as np
    from paper_2306_02526_gb300.serve import Server
    jobs = serving_jobs(args.serving_jobs)
    out = {"arrival_rate_per_s": 200.0, "jobs": len(jobs), "catalog": [list(c) for c in SERVING_CATALOG],
           "steps_range": [10, 500],
           "note": "factorization builds happen inside the run (cache misses) and count in the makespan; "
                   "DOF*stages/s = sum over jobs of N x 5 x steps / makespan"}
    results = {}
    for name, cols in (("fp64", 0), ("batched_mixed", 32)):
        S = Server(64 << 30, max_active=64 if cols else 16, batch_cols=cols, refine=-1)
        ids = [S.submit(**j) for j in jobs]
        S.run()
        results[name] = [S.result(i).copy() for i in ids]
        summ = S.summary()
        summ["form"] = ("every job alone, FP64 ark_step, one stream per job" if not cols else
                        "jobs of one operation as columns of ark_step_batch (FP32 sweeps + FP64 refinement, sweeps "
                        "chosen per operation by its stiffness), "
                        "at most 32 per batch, joining at step boundaries")
        out[name] = summ
        S.close()
    err = 0.0
    for j, a, b in zip(jobs, results["fp64"], results["batched_mixed"]):
        # relative to the larger of the initial and the final state (heat jobs decay by many orders)
        scale = max(np.abs(a).max(), np.abs(j["u0"]).max())
        err = max(err, float(np.abs(a - b).max() / scale))
    out["batched_err_vs_fp64"] = err
    out["batched_err_note"] = "max over jobs of |u_batched - u_fp64|_inf / max(|u_fp64|_inf, |u0|_inf)"
    out["batched_over_fp64_served"] = out["batched_mixed"]["dof_stages_per_s"] / out["fp64"]["dof_stages_per_s"]
    return out


def bench_reference(args, rank, world):
    """The oracle (the reference arm of this measurement) on the host cores: the BLAS thread count
    is chosen by short probes (1, 4, all threads), then W untimed and K timed full-size stage
    solves run in a child process with that many threads."""
    if rank != 0:
        return None
    th, rates = best_oracle_threads(args.workload, 4.0)
    smp = run_cpu_sample_subprocess(args.workload, 0.0, th, steps=args.steps, warmup=min(args.warmup, 1))
    value = smp["N"] * smp["solves"] / smp["seconds"]
    return {
        "impl": "reference", "metric": "DOF*stages/s (N x implicit HPS stage solves per second, ARK4(3)6L[2]SA step)",
        "value": value, "unit": "DOF*stages/s", "n_gpus": 1, "steps": smp["solves"], "warmup": args.warmup,
        "ms_per_step": smp["seconds"] / smp["solves"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": args.workload, "N": smp["N"]},
        "cpu_baseline": {"value": value, "unit": "DOF*stages/s", "cores": th, "kind": "oracle",
                         "sample": "%d full-size oracle stage solves (one step = one stage solve) with %d BLAS/OpenMP "
                                   "threads, the fastest of %s (probe rates %s; host has %d cores); oracle build "
                                   "%.1f s not timed" % (smp["solves"], th, sorted(rates),
                                                         {k: "%.3g" % v for k, v in rates.items()}, os.cpu_count(),
                                                         smp["build_s"])},
        "e2e": {"value": value, "unit": "DOF*stages/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.cpu_sample, args.cpu_budget, args.cpu_steps, args.warmup)))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = bench_reference(args, rank, world)
        if out:
            print(json.dumps(out))
        return
    import torch
    if args.only == "serving":
        from paper_2306_02526_gb300 import build as _b
        _b.build()
        print(json.dumps(bench_serving(args)))
        return
    if args.only == "per-node-fp32":
        print(json.dumps(per_node_fp32_sweeps(args)))
        return
    if args.only == "many-instances":
        from paper_2306_02526_gb300 import build as _b
        _b.build()
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps(bench_multi(args, flush)))
        return
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:  # before any GPU work in this process
        th, rates = best_oracle_threads(args.workload, 4.0)
        cpu = run_cpu_sample_subprocess(args.workload, args.cpu_budget, th)
        cpu["probe_rates"] = rates
    out = bench_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        if cpu is not None:
            out["cpu_baseline"] = {"value": cpu["N"] * cpu["solves"] / cpu["seconds"], "unit": "DOF*stages/s",
                                   "cores": cpu["threads"], "kind": "oracle",
                                   "sample": "%d oracle stage solves on %s leaves (p as the workload) in %.1f s with "
                                             "%d BLAS/OpenMP threads, the fastest of %s threads (probe rates %s); "
                                             "oracle build %.1f s not timed"
                                             % (cpu["solves"], cpu["leaves"], cpu["seconds"], cpu["threads"],
                                                sorted(cpu["probe_rates"]),
                                                {k: "%.3g" % v for k, v in cpu["probe_rates"].items()},
                                                cpu["build_s"])}
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
