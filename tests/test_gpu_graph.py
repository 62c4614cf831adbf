"""Graph replay (hps_set_graph) gives the same bits as eager launches, re-records when the
arguments change, and keeps the launch counters and event timing of the tracing facility."""
import numpy as np
import pytest

from gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def _solver(torch, n1=8, n2=8, p=10, dt=0.01):
    from paper_2306_02526_gb300 import hps, workloads
    tree = hps.Tree(n1, n2)
    N, N_int, N_bd = hps.hps_sizes(tree, p)
    coef = {k: to_dev(torch, v) for k, v in workloads.random_coefficients(3, N_int).items()}
    return hps.HPSSolver(tree, p, coef, 0.25 * dt), N, N_int


def test_graph_steps_equal_eager_steps():
    torch = need_gpu()
    S, N, N_int = _solver(torch)
    r = np.random.default_rng(0)
    u0 = r.uniform(-0.1, 0.1, N)
    ue = to_dev(torch, u0)
    for n in range(6):
        S.ark_step(ue, n * 0.01, 0.01, g="fisher", g_param=(0.5, 0.0))
    S.set_graph(True)
    ug = to_dev(torch, u0)
    for n in range(6):
        S.ark_step(ug, n * 0.01, 0.01, g="fisher", g_param=(0.5, 0.0))
    assert torch.equal(ue, ug)
    # a different buffer re-records; results still identical
    ug2 = to_dev(torch, u0)
    for n in range(6):
        S.ark_step(ug2, n * 0.01, 0.01, g="fisher", g_param=(0.5, 0.0))
    assert torch.equal(ue, ug2)
    # hps_solve in graph mode
    rhs = to_dev(torch, r.standard_normal(N_int))
    a = S.solve(rhs).clone()
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    for _ in range(3):
        S.solve(rhs, u=out)
    assert torch.equal(a, out)
    S.close()


def test_graph_replay_counts_launches_and_times_kernels():
    torch = need_gpu()
    S, N, N_int = _solver(torch, 4, 4, 8)
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    S.trace_enable(("leaf_up",))
    S.ark_step(u, 0.0, 0.01)          # eager
    eager = S.trace_read()
    S.set_graph(True)
    S.trace_enable(("leaf_up",))
    for n in range(2):                 # eager + record
        S.ark_step(u, 0.0, 0.01)
    S.trace_enable(("leaf_up",))      # same mask: graph kept, counters reset
    for n in range(3):                 # replays
        S.ark_step(u, 0.0, 0.01)
    rep = S.trace_read()
    for k in eager:
        assert rep[k][0] == 3 * eager[k][0], k
    # one leaf solve per implicit stage (5 per step; the step close is the edge projection)
    assert rep["leaf_up"][1] == 3 * 5 and rep["leaf_up"][2] > 0.0
    S.close()
