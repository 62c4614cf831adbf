"""Edge cases at the limits of the C ABI: the largest order p = 32 (FP64 solve and ARK step against
the oracle), the largest column count R = 64 of the batched path (and R = 65 rejected), a
served job of zero steps (its state comes back unchanged), a single-leaf tree in the batched
step."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle import ark as oark
from oracle import nonlinear
from oracle.grid import Grid
from oracle.hps import HPS
from paper_2306_02526_gb300 import workloads

pytestmark = pytest.mark.gpu


def _solver(torch, g, coef, gdt):
    from paper_2306_02526_gb300 import hps
    tree = hps.Tree(g.n1, g.n2, g.x0, g.x1, g.y0, g.y1)
    cg = {k: (to_dev(torch, v) if np.ndim(v) else float(v)) for k, v in coef.items()}
    return hps.HPSSolver(tree, g.p, cg, gdt)


@pytest.mark.parametrize("nodal", [False, True])
def test_largest_p_solve_and_step_match_oracle(nodal):
    torch = need_gpu()
    g = Grid(2, 1, 32)
    coef = workloads.random_coefficients(5, g.N_int) if nodal else {"a11": 1.0, "a22": 0.5, "a1": 0.2, "a0": -0.3}
    S = _solver(torch, g, coef, 0.004)
    r = np.random.default_rng(32)
    rhs = r.standard_normal(g.N_int)
    f = r.standard_normal(g.boundary_indices().size)
    got = S.solve(to_dev(torch, rhs), to_dev(torch, f)).cpu().numpy()
    assert rel_max(got, HPS(g, coef, 0.004).solve(rhs, f)) <= 1e-12
    # one ARK step (Fisher) against the oracle
    X, Y = g.coords()
    u = 0.3 * np.sin(np.pi * X) * np.sin(np.pi * Y)
    u[g.boundary_indices()] = 0.0
    dt = 0.016
    ud = to_dev(torch, u)
    S.ark_step(ud, 0.0, dt, g="fisher", g_param=(0.5, 0.0))
    prob = oark.Problem(g, coef, g=nonlinear.fisher(0.5))
    v, _ = oark.ark_step(prob, HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0), u, 0.0, dt)
    assert rel_max(ud.cpu().numpy(), v) <= 1e-12
    S.close()


def test_largest_column_count():
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib
    g = Grid(4, 4, 8)
    coef = workloads.random_coefficients(7, g.N_int)
    S = _solver(torch, g, coef, 0.01)
    with pytest.raises(_lib.HPSError):
        S.batch_reserve(65)
    R = 64
    S.batch_reserve(R)
    r = np.random.default_rng(64)
    rhs = r.standard_normal((g.N_int, R))
    got = S.solve_batch(to_dev(torch, rhs), refine=2).cpu().numpy()
    for j in (0, 31, 63):
        want = S.solve(to_dev(torch, rhs[:, j].copy())).cpu().numpy()
        assert rel_max(got[:, j], want) <= 1e-10
    assert rel_max(got[:, 0], HPS(g, coef, 0.01).solve(rhs[:, 0])) <= 1e-10
    S.close()


def test_single_leaf_batched_step_matches_oracle():
    torch = need_gpu()
    g = Grid(1, 1, 12)
    coef = {"a11": 0.3, "a22": 0.3}
    dt = 0.01
    S = _solver(torch, g, coef, 0.25 * dt)
    S.batch_reserve(3)
    X, Y = g.coords()
    U0 = np.stack([(0.2 + 0.1 * j) * np.sin(np.pi * X) * np.sin(np.pi * Y) for j in range(3)], axis=1)
    U0[g.boundary_indices(), :] = 0.0
    ub = to_dev(torch, U0)
    for n in range(2):
        S.ark_step_batch(ub, n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0), refine=2)
    prob = oark.Problem(g, coef, g=nonlinear.allen_cahn(1.0))
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    got = ub.cpu().numpy()
    for j in range(3):
        v = U0[:, j].copy()
        for n in range(2):
            v, _ = oark.ark_step(prob, Hi, Hid, v, n * dt, dt)
        assert rel_max(got[:, j], v) <= 1e-10
    S.close()


@pytest.mark.parametrize("batch_cols", [0, 8])
def test_zero_step_job_returns_its_state(batch_cols):
    need_gpu()
    from paper_2306_02526_gb300 import hps
    from paper_2306_02526_gb300.serve import Server
    t = hps.Tree(4, 4)
    N, _, _ = hps.hps_sizes(t, 8)
    u0 = np.random.default_rng(0).uniform(-0.1, 0.1, N)
    u0[hps.hps_boundary_index(t, 8)] = 0.0
    S = Server(4 << 30, 4, batch_cols=batch_cols)
    a = S.submit(tree=t, p=8, coef={"a11": 1.0, "a22": 1.0}, dt=0.01, steps=0, u0=u0)
    b = S.submit(tree=t, p=8, coef={"a11": 1.0, "a22": 1.0}, dt=0.01, steps=3, u0=u0)
    S.run()
    sa, sb = S.job_stats(a), S.job_stats(b)
    ra = S.result(a).copy()
    S.close()
    assert sa["state"] == 2 and sa["steps_done"] == 0 and np.array_equal(ra, u0)
    assert sb["state"] == 2 and sb["steps_done"] == 3
