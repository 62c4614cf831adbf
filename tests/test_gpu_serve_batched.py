"""Serving with continuous batching at the kernel level (hps_server_set_batching): jobs of the same
operation (operator and g) advance as columns of one batched mixed-precision step; jobs join
running batches at step boundaries.  Tolerance of the mixed path: 1e-10 relative max-norm, against
the FP64 ark_step of the same job and between a job alone and in the mix."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle import ark as oark
from oracle import nonlinear
from oracle.grid import Grid
from oracle.hps import HPS

pytestmark = pytest.mark.gpu

TOL = 1e-10
HEAT = {"a11": 1.0, "a22": 1.0}
AC = {"a11": 0.01, "a22": 0.01}


def _jobs():
    """Two operations with several jobs each (staggered arrivals, different step counts) and one
    single job of a third operation."""
    from paper_2306_02526_gb300 import hps
    out = []
    t = hps.Tree(16, 16)
    N, _, _ = hps.hps_sizes(t, 12)
    bd = hps.hps_boundary_index(t, 12)
    for seed in range(6):
        u = np.random.default_rng(seed).uniform(-0.1, 0.1, N)
        u[bd] = 0.0
        out.append(dict(tree=t, p=12, coef=AC, dt=1e-3, steps=10 + 3 * seed, u0=u, g="allen_cahn",
                        g_param=(1.0, 0.0), arrival_s=0.004 * seed))
    t = hps.Tree(8, 8)
    x, y = hps.hps_coords(t, 10)
    bd = hps.hps_boundary_index(t, 10)
    for j in range(3):  # (a mode that decays by less than 1e-2 over the run: relative errors stay meaningful)
        u = (1.0 + 0.5 * j) * np.sin(np.pi * x) * np.sin(np.pi * y) + 0.05 * np.sin(2 * np.pi * x) * np.sin(np.pi * y)
        u[bd] = 0.0
        out.append(dict(tree=t, p=10, coef=HEAT, dt=0.01, steps=8 + 4 * j, u0=u, g=None, arrival_s=0.002 + 0.01 * j))
    t = hps.Tree(4, 8)
    x, y = hps.hps_coords(t, 8)
    u = 0.2 * np.sin(np.pi * x) * np.sin(np.pi * y) + 0.1
    u[hps.hps_boundary_index(t, 8)] = 0.0
    out.append(dict(tree=t, p=8, coef=AC, dt=0.02, steps=8, u0=u, g="fisher", g_param=(0.5, 0.0), arrival_s=0.01))
    return out


def _serve(jobs, budget=16 << 30, max_active=16, cols=8, refine=-1):
    from paper_2306_02526_gb300.serve import Server
    S = Server(budget, max_active, batch_cols=cols, refine=refine)
    ids = [S.submit(**j) for j in jobs]
    S.run()
    res = [S.result(i).copy() for i in ids]
    stats = [S.job_stats(i) for i in ids]
    summ = S.summary()
    S.close()
    return res, stats, summ


def _fp64(torch, j):
    from paper_2306_02526_gb300 import hps
    S = hps.HPSSolver(j["tree"], j["p"], j["coef"], 0.25 * j["dt"])
    u = to_dev(torch, j["u0"])
    for n in range(j["steps"]):
        S.ark_step(u, n * j["dt"], j["dt"], g=j["g"], g_param=j.get("g_param", (1.0, 1.0)))
    out = u.cpu().numpy()
    S.close()
    return out


def test_batched_serving_matches_fp64_and_alone():
    torch = need_gpu()
    jobs = _jobs()
    mixed, stats, summ = _serve(jobs)
    assert summ["jobs_done"] == len(jobs) and summ["jobs_rejected"] == 0
    assert summ["batches_formed"] <= 4 and summ["mean_batch_cols"] > 1.5   # jobs shared batches
    assert summ["max_concurrent"] >= 4 and summ["step_ms_p99"] >= summ["step_ms_p50"] > 0.0
    assert sum(s["shared_operators"] for s in stats) >= len(jobs) - 3
    for j, m, s in zip(jobs, mixed, stats):
        assert s["state"] == 2 and s["status"] == 0 and s["steps_done"] == j["steps"]
        assert rel_max(m, _fp64(torch, j)) <= TOL
    for k in (0, 5, 7, 9):  # alone (a batch of one) equals its result in the mix
        alone, st, _ = _serve([dict(jobs[k], arrival_s=0.0)])
        assert st[0]["state"] == 2
        assert rel_max(alone[0], mixed[k]) <= TOL


def test_batched_serving_job_matches_oracle():
    need_gpu()
    j = _jobs()[9]
    res, stats, _ = _serve([j], refine=2)
    g = Grid(4, 8, 8)
    prob = oark.Problem(g, j["coef"], g=nonlinear.fisher(0.5))
    Hi, Hid = HPS(g, j["coef"], 0.25 * j["dt"]), HPS(g, j["coef"], 0.0)
    u = j["u0"].copy()
    for n in range(j["steps"]):
        u, _ = oark.ark_step(prob, Hi, Hid, u, n * j["dt"], j["dt"])
    assert rel_max(res[0], u) <= TOL


def test_batched_serving_memory_budget():
    need_gpu()
    jobs = _jobs()[:6]  # one operation
    ref, _, _ = _serve(jobs)
    # a budget for one batch of 4 columns (its size measured by a first run): the jobs queue for
    # columns, all complete
    from paper_2306_02526_gb300 import hps
    _, _, one = _serve(jobs[:4], cols=4)
    budget = int(one["peak_bytes"] * 1.05)
    res, stats, summ = _serve(jobs, budget=budget, cols=4)
    assert summ["jobs_done"] == len(jobs) and summ["peak_bytes"] <= budget
    assert summ["batches_formed"] == 1
    for a, b in zip(ref, res):
        assert rel_max(b, a) <= TOL
    # a job that can never fit is rejected
    res, stats, summ = _serve(jobs[:1], budget=hps.hps_bytes(jobs[0]["tree"], jobs[0]["p"]) // 2)
    assert stats[0]["state"] == 3


def test_batched_evicted_job_resumes():
    """A batch member checkpointed after 4 steps leaves its batch, queues again, rejoins a batch and
    ends within the mixed-precision tolerance of its uninterrupted result and of the FP64 path."""
    torch = need_gpu()
    from paper_2306_02526_gb300.serve import Server
    jobs = _jobs()[:6]
    ref, _, _ = _serve(jobs)
    S = Server(16 << 30, 16, batch_cols=8, refine=-1)
    ids = [S.submit(**j) for j in jobs]
    S.evict_after(ids[2], 4)
    S.run()
    st = S.job_stats(ids[2])
    got = S.result(ids[2]).copy()
    S.close()
    assert st["state"] == 2 and st["evictions"] == 1 and st["steps_done"] == jobs[2]["steps"]
    assert rel_max(got, ref[2]) <= TOL
    assert rel_max(got, _fp64(torch, jobs[2])) <= TOL
