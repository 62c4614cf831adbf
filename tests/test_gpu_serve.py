"""Serving loop (hps_server_*): continuous batching of time-stepping jobs with different trees
and orders.  Each job's result is the same alone and in the mix (bit for bit: the same kernels
on the same data), equals the direct ark_step path, and admission respects the memory budget."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle import ark as oark
from oracle import nonlinear
from oracle.grid import Grid
from oracle.hps import HPS

pytestmark = pytest.mark.gpu

HEAT = {"a11": 1.0, "a22": 1.0}
AC = {"a11": 0.01, "a22": 0.01}


def _jobs():
    from paper_2306_02526_gb300 import hps
    out = []
    t = hps.Tree(8, 8)
    x, y = hps.hps_coords(t, 10)
    u = np.sin(np.pi * x) * np.sin(np.pi * y)
    u[hps.hps_boundary_index(t, 10)] = 0.0
    out.append(dict(tree=t, p=10, coef=HEAT, dt=0.01, steps=12, u0=u, g=None, arrival_s=0.0))
    t = hps.Tree(16, 16)
    N, _, _ = hps.hps_sizes(t, 12)
    bd = hps.hps_boundary_index(t, 12)
    for seed, arr in ((1, 0.0), (2, 0.03)):
        u = np.random.default_rng(seed).uniform(-0.1, 0.1, N)
        u[bd] = 0.0
        out.append(dict(tree=t, p=12, coef=AC, dt=1e-3, steps=20, u0=u, g="allen_cahn", g_param=(1.0, 0.0),
                        arrival_s=arr))
    t = hps.Tree(4, 8)
    x, y = hps.hps_coords(t, 8)
    u = 0.2 * np.sin(np.pi * x) * np.sin(np.pi * y) + 0.1
    u[hps.hps_boundary_index(t, 8)] = 0.0
    out.append(dict(tree=t, p=8, coef=AC, dt=0.02, steps=8, u0=u, g="fisher", g_param=(0.5, 0.0), arrival_s=0.01))
    return out


def _serve(jobs, budget=8 << 30, max_active=8):
    from paper_2306_02526_gb300.serve import Server
    S = Server(budget, max_active)
    ids = [S.submit(**j) for j in jobs]
    S.run()
    res = [S.result(i).copy() for i in ids]
    stats = [S.job_stats(i) for i in ids]
    summ = S.summary()
    S.close()
    return res, stats, summ


def test_alone_equals_in_mix_and_direct_path():
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    jobs = _jobs()
    alone = [_serve([dict(j, arrival_s=0.0)])[0][0] for j in jobs]
    mixed, stats, summ = _serve(jobs)
    for a, m, s in zip(alone, mixed, stats):
        assert s["state"] == 2 and s["status"] == 0
        assert np.array_equal(a, m)
    assert summ["jobs_done"] == len(jobs) and summ["max_concurrent"] >= 2
    assert summ["factorizations_shared"] >= 1 and stats[2]["shared_operators"] == 1
    assert summ["step_ms_p99"] >= summ["step_ms_p50"] > 0.0
    # the served result equals the direct C-ABI path step by step
    j = jobs[1]
    S = hps.HPSSolver(j["tree"], j["p"], j["coef"], 0.25 * j["dt"])
    u = to_dev(torch, j["u0"])
    for n in range(j["steps"]):
        S.ark_step(u, n * j["dt"], j["dt"], g=j["g"], g_param=j["g_param"])
    assert np.array_equal(u.cpu().numpy(), mixed[1])
    S.close()


def test_served_job_matches_oracle():
    need_gpu()
    j = _jobs()[3]
    res, stats, _ = _serve([j])
    g = Grid(4, 8, 8)
    coef = j["coef"]
    prob = oark.Problem(g, coef, g=nonlinear.fisher(0.5))
    Hi, Hid = HPS(g, coef, 0.25 * j["dt"]), HPS(g, coef, 0.0)
    u = j["u0"].copy()
    for n in range(j["steps"]):
        u, _ = oark.ark_step(prob, Hi, Hid, u, n * j["dt"], j["dt"])
    assert rel_max(res[0], u) <= 1e-12


def test_memory_budget_admission():
    need_gpu()
    from paper_2306_02526_gb300 import hps
    jobs = _jobs()
    need = max(hps.hps_bytes(j["tree"], j["p"]) + 8 * hps.hps_sizes(j["tree"], j["p"])[0] for j in jobs)
    res_ref, _, _ = _serve(jobs)
    res, stats, summ = _serve(jobs, budget=int(need * 1.02))
    assert summ["jobs_done"] == len(jobs) and summ["max_concurrent"] == 1 and summ["peak_bytes"] <= need * 1.02
    for a, b in zip(res_ref, res):
        assert np.array_equal(a, b)
    # a job that can never fit is rejected, the others still run
    small = min(hps.hps_bytes(j["tree"], j["p"]) for j in jobs)
    res, stats, summ = _serve([jobs[0], jobs[3]], budget=int(small * 1.5))
    assert [s["state"] for s in stats].count(3) >= 1 and summ["jobs_done"] >= 1


def test_evicted_job_resumes_bit_identical():
    """Eviction with checkpoint / resume (hps_server_evict_after): a job checkpointed to host memory
    after 5 steps, released and re-admitted behind the other jobs ends bit-identical to an
    uninterrupted run."""
    need_gpu()
    from paper_2306_02526_gb300.serve import Server
    jobs = _jobs()
    ref, _, _ = _serve([dict(jobs[1], arrival_s=0.0)])
    S = Server(8 << 30, 2)  # two slots: the evicted job waits for one
    ids = [S.submit(**j) for j in jobs]
    S.evict_after(ids[1], 5)
    S.run()
    st = S.job_stats(ids[1])
    got = S.result(ids[1]).copy()
    S.close()
    assert st["state"] == 2 and st["status"] == 0 and st["evictions"] == 1 and st["steps_done"] == jobs[1]["steps"]
    assert np.array_equal(got, ref[0])
