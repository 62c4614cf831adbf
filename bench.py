#!/usr/bin/env python3
"""Throughput of the ARK4(3)6L[2]SA + HPS time step on one GB300: DOF x implicit stages / s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): u_t = 0.01 Lap u + u - u^3 on [0,1]^2, 64 x 64 leaves, p = 16
(N = 919,296 unknowns), dt = 1e-3, u0 ~ U[-0.1, 0.1] seed 0, FP64.  A step is one full ARK
step: the explicit first stage, 5 implicit HPS stage solves, the ARK combination and the
identity-operator projection.  value = N * 5 * K / (sum of the K step times), device-timed
with CUDA events on the launch stream; L2 (129 MB) is flushed by writing a 512 MB buffer
before every timed step.  N > 1 (torchrun): independent replicas, one per GPU (the method
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
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-budget", type=float, default=12.0, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
def oracle_setup(wname):
    import numpy as np
    from oracle.grid import Grid
    from oracle.hps import HPS
    from paper_2306_02526_gb300 import workloads
    wl = workloads.WORKLOADS[wname]
    g = Grid(wl.n1, wl.n2, wl.p)
    X, Y = g.coords()
    I = np.arange(g.N_int)
    coef = wl.coef(X[I], Y[I])
    t0 = time.perf_counter()
    H = HPS(g, coef, 0.25 * wl.dt)
    build_s = time.perf_counter() - t0
    rhs = np.random.default_rng(1).uniform(-0.1, 0.1, g.N_int)
    return g, H, rhs, build_s


def cpu_sample(wname, budget):
    """Time full-size oracle stage solves until `budget` seconds have passed (at least one)."""
    g, H, rhs, build_s = oracle_setup(wname)
    n, t0 = 0, time.perf_counter()
    while True:
        H.solve(rhs)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget:
            break
    return {"solves": n, "seconds": el, "N": g.N, "build_s": build_s}


def run_cpu_sample_subprocess(wname, budget):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", wname, "--cpu-budget", str(budget)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


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


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------------------------
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
    u0 = wl.u0(x, y, bidx)
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")

    def stage_terms(t):
        q = f = None
        if wl.q(x[:1], y[:1], 0.0) is not None:
            q = torch.tensor(np.stack([wl.q(x[I], y[I], t + cj * wl.dt) for cj in c]).reshape(-1),
                             dtype=torch.float64, device="cuda")
        if wl.f(x[:1], y[:1], 0.0) is not None:
            f = torch.tensor(np.stack([wl.f(x[bidx], y[bidx], t + cj * wl.dt) for cj in c]).reshape(-1),
                             dtype=torch.float64, device="cuda")
        return q, f

    static_q, static_f = stage_terms(0.0)  # synthetic workload: time-dependent data held fixed per step

    def step(uu, t):
        S.ark_step(uu, t, wl.dt, q=static_q, f=static_f, g=wl.g, g_param=wl.g_param)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    if not args.eager:
        S.set_graph(True)  # each ARK step is replayed from a recorded CUDA graph
    t = 0.0
    for _ in range(args.warmup):
        step(u, t)
        t += wl.dt
    # per-kernel shares from a traced pass (all kernels event-timed), untimed
    from paper_2306_02526_gb300 import _lib
    S.trace_enable(_lib.KERNELS)
    for _ in range(4):
        step(u, t)
        t += wl.dt
    shares = S.trace_read()
    dom = max(shares, key=lambda k: shares[k][2])
    # timed region: only the dominant kernel is event-timed (launches of all kernels are counted);
    # two untimed steps first so that the graph with the new timing events is recorded
    S.trace_enable((dom,))
    for _ in range(2):
        step(u, t)
        t += wl.dt
    S.trace_enable((dom,))
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
            step(u, t)
            evs[k][1].record(stream)
            t += wl.dt
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tr = S.trace_read()
    total_ms = sum(step_ms)
    if world > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    assert torch.isfinite(u).all(), "solution went non-finite"
    value = world * N * STAGES * args.steps / (total_ms * 1e-3)
    launches = sum(v[0] for v in tr.values())

    # end to end through the C ABI from pinned host buffers: H2D of u, one step, D2H of u
    host_u = torch.tensor(u0, dtype=torch.float64).pin_memory()
    host_out = torch.empty(N, dtype=torch.float64).pin_memory()
    ue = torch.empty(N, dtype=torch.float64, device="cuda")
    e2e_steps = max(5, min(args.steps, 20))
    e_ms = []
    for k in range(e2e_steps + 2):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ue.copy_(host_u, non_blocking=True)
        step(ue, 0.0)
        host_out.copy_(ue, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if k >= 2:
            e_ms.append(a.elapsed_time(b))
    e2e_value = N * STAGES / (statistics.mean(e_ms) * 1e-3)

    out = None
    if rank == 0:
        q, b, m = (wl.p - 2) ** 2, 4 * (wl.p - 2), wl.p - 2
        n_dom, n_timed, dom_ms = tr[dom]
        avg_ms = dom_ms / max(1, n_timed)
        dgemm = fp64_dgemm_tflops(torch)
        peak_fp64 = 1.25  # nominal GB300 FP64 (TFLOP/s)
        roof = {"kernel": dom, "bound": "alu", "unit": "TFLOP/s", "peak": peak_fp64,
                "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table); cuBLAS DGEMM measured %.3f" % dgemm,
                "traffic": None}
        if dom == "leaf_up":
            fl = leaf_up_flops(N_int, q, b, m, 11)
            roof["achieved"] = fl / (avg_ms * 1e-3) / 1e12
            roof["frac"] = roof["achieved"] / peak_fp64
            roof["flops_per_launch"] = fl
        tot_share = sum(v[2] for v in shares.values())
        out = {
            "metric": "DOF*stages/s (N x implicit HPS stage solves per second, ARK4(3)6L[2]SA step)",
            "value": value, "unit": "DOF*stages/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "p50_step_ms": statistics.median(step_ms),
            "p99_step_ms": sorted(step_ms)[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded u0 ~ U[-0.1,0.1])",
            "config": {"workload": wl.name, "n1": wl.n1, "n2": wl.n2, "p": wl.p, "N": N, "p2n1n2": wl.p ** 2 * wl.n1 * wl.n2,
                       "dt": wl.dt, "stages_per_step": STAGES, "operators": "one per tree level (constant coefficients)",
                       "l2": "flushed (512 MB write) before every timed step",
                       "launch": "eager" if args.eager else "CUDA graph replay (hps_set_graph)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof,
            "kernel_shares": {k: round(v[2] / tot_share, 4) for k, v in shares.items()},
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "DOF*stages/s", "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8,
                    "steps": e2e_steps},
            "clocks": clk.summary(),
            "build_s": build_s, "wall_s": wall,
        }
    S.close()
    return out


def bench_reference(args, rank, world):
    if rank != 0:
        return None
    import numpy as np  # noqa: F401
    g, H, rhs, build_s = oracle_setup(args.workload)
    t0 = time.perf_counter()
    H.solve(rhs)
    est = time.perf_counter() - t0
    steps = max(1, min(args.steps, int(150.0 / max(est, 1e-3))))
    for _ in range(min(args.warmup, 1)):
        H.solve(rhs)
    t0 = time.perf_counter()
    for _ in range(steps):
        H.solve(rhs)
    el = time.perf_counter() - t0
    value = g.N * steps / el
    cores = os.cpu_count()
    return {
        "impl": "reference", "metric": "DOF*stages/s (N x implicit HPS stage solves per second, ARK4(3)6L[2]SA step)",
        "value": value, "unit": "DOF*stages/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": el / steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": args.workload, "N": g.N},
        "cpu_baseline": {"value": value, "unit": "DOF*stages/s", "cores": cores, "kind": "oracle",
                         "sample": "%d full-size oracle stage solves (one step = one stage solve); oracle build %.1f s "
                                   "not timed" % (steps, build_s)},
        "e2e": {"value": value, "unit": "DOF*stages/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.cpu_sample, args.cpu_budget)))
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
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = run_cpu_sample_subprocess(args.workload, args.cpu_budget)  # before any GPU work in this process
    out = bench_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        if cpu is not None:
            out["cpu_baseline"] = {"value": cpu["N"] * cpu["solves"] / cpu["seconds"], "unit": "DOF*stages/s",
                                   "cores": 1, "kind": "oracle",
                                   "sample": "%d full-size oracle stage solves in %.1f s on one host thread "
                                             "(BLAS threads = 1); oracle build %.1f s not timed"
                                             % (cpu["solves"], cpu["seconds"], cpu["build_s"])}
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
