"""Many independent instances of uneven sizes advanced together (hps_multi_*): every instance's
batched mixed-precision ARK step on its own internal stream, the whole multi-instance step
recorded into one CUDA graph and replayed.  Each instance must equal the same instance stepped
alone with ark_step_batch bit for bit (the same kernels on the same data), and its FP64 ark_step
result to the mixed-precision tolerance (1e-10)."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from paper_2306_02526_gb300 import workloads

pytestmark = pytest.mark.gpu


def _instances(torch):
    from paper_2306_02526_gb300 import hps
    ins = workloads.instances(count=5, seed=3, grids=(2, 4, 8), orders=(6, 8, 12))
    out = []
    for k, w in enumerate(ins):
        tree = hps.Tree(w.n1, w.n2)
        N, N_int, _ = hps.hps_sizes(tree, w.p)
        x, y = hps.hps_coords(tree, w.p)
        bd = hps.hps_boundary_index(tree, w.p)
        coef = {c: to_dev(torch, v) for c, v in w.coef(x[:N_int], y[:N_int]).items()}
        R = (4, 8, 16, 5, 13)[k]
        U0 = np.stack([workloads.uniform_state(100 * k + j, N, bd) for j in range(R)], axis=1)
        out.append((w, tree, coef, R, U0))
    return out


def test_multi_step_equals_instances_alone_and_fp64():
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    cases = _instances(torch)
    solvers, states = [], []
    for w, tree, coef, R, U0 in cases:
        S = hps.HPSSolver(tree, w.p, coef, 0.25 * w.dt)
        S.batch_reserve(R)
        solvers.append(S)
        states.append(to_dev(torch, U0))
    M = hps.MultiStep(solvers)
    M.set_graph(True)
    steps = 4  # eager, recorded, replayed, replayed
    for _ in range(steps):
        M.ark_step(states, cases[0][0].dt, g="allen_cahn", g_param=(1.0, 0.0), refine=2)
    torch.cuda.synchronize()
    got = [u.cpu().numpy() for u in states]
    M.close()
    for (w, tree, coef, R, U0), S, G in zip(cases, solvers, got):
        S.status()
        alone = to_dev(torch, U0)
        for _ in range(steps):
            S.ark_step_batch(alone, 0.0, w.dt, g="allen_cahn", g_param=(1.0, 0.0), refine=2)
        assert np.array_equal(alone.cpu().numpy(), G), w.name
        for j in (0, R - 1):
            ref = to_dev(torch, U0[:, j].copy())
            for n in range(steps):
                S.ark_step(ref, n * w.dt, w.dt, g="allen_cahn", g_param=(1.0, 0.0))
            assert rel_max(G[:, j], ref.cpu().numpy()) <= 1e-10, (w.name, j)
        S.close()


def test_multi_rejects_bad_arguments():
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib, hps
    S = hps.HPSSolver(hps.Tree(2, 2), 6, {"a11": 1.0, "a22": 1.0}, 2.5e-4)
    S.batch_reserve(4)
    M = hps.MultiStep([S])
    u = torch.zeros((S.N, 8), dtype=torch.float64, device="cuda")  # more columns than reserved
    with pytest.raises(_lib.HPSError):
        M.ark_step([u], 1e-3)
    M.close()
    S.close()


def _lockstep_run(torch, cases, lockstep, graph, steps, g="allen_cahn"):
    from paper_2306_02526_gb300 import hps
    solvers, states = [], []
    for w, tree, coef, R, U0 in cases:
        S = hps.HPSSolver(tree, w.p, coef, 0.25 * w.dt)
        S.batch_reserve(R)
        solvers.append(S)
        states.append(to_dev(torch, U0))
    M = hps.MultiStep(solvers)
    M.set_lockstep(lockstep)
    M.set_graph(graph)
    for _ in range(steps):
        M.ark_step(states, cases[0][0].dt, g=g, g_param=(1.0, 0.0), refine=2)
    torch.cuda.synchronize()
    got = [u.cpu().numpy() for u in states]
    M.close()
    return solvers, got


def test_lockstep_merges_match_concurrent_and_fp64():
    """Lockstep (one grouped merge launch per tree level for all instances, trees of 2 to 6
    levels) against the concurrent per-instance step to the mixed-precision tolerance, eager and
    replayed from one graph bit for bit, and column 0 of each instance against FP64 ark_step."""
    torch = need_gpu()
    cases = _instances(torch)
    steps = 4
    _, conc = _lockstep_run(torch, cases, False, False, steps)
    _, eager = _lockstep_run(torch, cases, True, False, steps)
    solvers, graphed = _lockstep_run(torch, cases, True, True, steps)
    for (w, tree, coef, R, U0), S, A, B, C in zip(cases, solvers, conc, eager, graphed):
        assert np.array_equal(B, C), w.name
        assert rel_max(B, A) <= 1e-10, (w.name, rel_max(B, A))
        ref = to_dev(torch, U0[:, 0].copy())
        for n in range(steps):
            S.ark_step(ref, n * w.dt, w.dt, g="allen_cahn", g_param=(1.0, 0.0))
        assert rel_max(B[:, 0], ref.cpu().numpy()) <= 1e-10, w.name
        S.status()
        S.close()


def test_lockstep_more_instances_than_one_grouped_launch():
    """70 instances (more than the 64 a grouped launch takes): one to four columns each, so that
    register-tile widths differ within a level, trees of 1 to 4 levels."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    ins = workloads.instances(count=70, seed=9, grids=(1, 2, 4), orders=(6, 8))
    cases = []
    for k, w in enumerate(ins):
        tree = hps.Tree(w.n1, w.n2)
        N, N_int, _ = hps.hps_sizes(tree, w.p)
        x, y = hps.hps_coords(tree, w.p)
        bd = hps.hps_boundary_index(tree, w.p)
        coef = {c: to_dev(torch, v) for c, v in w.coef(x[:N_int], y[:N_int]).items()}
        R = 1 + k % 4
        U0 = np.stack([workloads.uniform_state(1000 + 10 * k + j, N, bd) for j in range(R)], axis=1)
        cases.append((w, tree, coef, R, U0))
    _, conc = _lockstep_run(torch, cases, False, False, 2, g=None)
    solvers, lock = _lockstep_run(torch, cases, True, True, 2, g=None)
    for (w, *_), S, A, B in zip(cases, solvers, conc, lock):
        assert rel_max(B, A) <= 1e-10, (w.name, rel_max(B, A))
        S.close()


def test_lockstep_rejects_column_groups():
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib, hps
    S = hps.HPSSolver(hps.Tree(2, 2), 6, {"a11": 1.0, "a22": 1.0}, 2.5e-4)
    S.batch_reserve(8, groups=2)
    M = hps.MultiStep([S])
    with pytest.raises(_lib.HPSError):
        M.set_lockstep(True)
    M.close()
    S.close()
