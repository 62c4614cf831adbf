"""ark_slope_step_batch (slope form, g = 0, penalized interface rows, R states, FP32 sweeps with
FP64 refinement against the residual of every slope system, interface rows included) against
the FP64 ark_slope_step column by column (mixed-precision tolerance 1e-10) and against the
oracle's slope-form step."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle import ark_slope
from oracle.grid import Grid
from oracle.hps import HPS
from paper_2306_02526_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _solver(torch, g, coef, gdt):
    from paper_2306_02526_gb300 import hps
    tree = hps.Tree(g.n1, g.n2, g.x0, g.x1, g.y0, g.y1)
    cg = {k: (to_dev(torch, v) if np.ndim(v) else float(v)) for k, v in coef.items()}
    return hps.HPSSolver(tree, g.p, cg, gdt)


@pytest.mark.parametrize("n1,n2,p,R,nodal,refine", [(4, 2, 9, 5, False, 2), (8, 8, 12, 8, True, 2),
                                                    (16, 8, 10, 4, False, 2), (2, 1, 8, 1, True, 3)])
def test_slope_batch_with_flux_jumps_matches_fp64(n1, n2, p, R, nodal, refine):
    """States with flux jumps on every shared edge (the penalization acts) and a source per column;
    constant (fast-diagonalization leaves) or nodal coefficients; 3 steps.  (The random states decay
    by orders of magnitude: one refinement sweep leaves about 1e-10 relative to the final state,
    two sweeps are taken.)"""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    g = Grid(n1, n2, p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = workloads.VarCoef128().coef(X[I], Y[I]) if nodal else {"a11": 0.8, "a22": 0.5, "a1": 0.2}
    dt = 0.01
    c = hps.hps_ark_abscissae()
    rng = np.random.default_rng(R + p)
    U0 = rng.standard_normal((g.N, R))
    U0[bd, :] = 0.0
    S = _solver(torch, g, coef, 0.25 * dt)
    S.batch_reserve(R)
    qf = lambda t, j: (1.0 + 0.3 * j) * np.cos(X[I] + t) * np.sin(2 * Y[I] + j)
    ub = to_dev(torch, U0)
    us = [to_dev(torch, U0[:, j].copy()) for j in range(R)]
    t = 0.0
    for n in range(3):
        qb = np.stack([np.stack([qf(t + cj * dt, j) for j in range(R)], axis=1) for cj in c])  # (6, N_int, R)
        S.ark_slope_step_batch(ub, t, dt, q=to_dev(torch, qb.reshape(-1)), refine=refine)
        for j in range(R):
            S.ark_slope_step(us[j], t, dt, q=to_dev(torch, np.ascontiguousarray(qb[:, :, j]).reshape(-1)))
        t += dt
    got = ub.cpu().numpy()
    for j in range(R):
        assert rel_max(got[:, j], us[j].cpu().numpy()) <= TOL, (j, rel_max(got[:, j], us[j].cpu().numpy()))
    if g.N <= 3000:  # column 0 against the oracle
        Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
        u = U0[:, 0].copy()
        t = 0.0
        for n in range(3):
            u, _ = ark_slope.ark_slope_step(g, coef, Hi, Hid, u, t, dt, q=lambda s: qf(s, 0))
            t += dt
        assert rel_max(got[:, 0], u) <= TOL
    S.status()
    S.close()


def test_slope_batch_with_u_t_boundary_data_and_graph():
    """Time-dependent Dirichlet data through the slopes' boundary data u_t, 4 columns of different
    amplitude; replayed from a CUDA graph the steps equal the eager ones."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    g = Grid(4, 4, 10)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = {"a11": 1.0, "a22": 1.0}
    s2 = (Y - 0.5) ** 2
    ue = lambda t: np.sin(np.pi * X) * np.exp(-t * s2)

    def qf(t):
        u = ue(t)
        lap = -np.pi ** 2 * u + np.sin(np.pi * X) * np.exp(-t * s2) * ((2 * t * (Y - 0.5)) ** 2 - 2 * t)
        return (-s2 * u - lap)[I]

    kbc = lambda t: (-s2 * ue(t))[bd]
    amp = np.array([1.0, 0.5, 2.0, -1.0])
    R = amp.size
    dt = 0.05
    c = hps.hps_ark_abscissae()
    S = _solver(torch, g, coef, 0.25 * dt)
    S.batch_reserve(R)

    def run(graph, steps=5):
        S.set_graph(graph)
        ub = to_dev(torch, np.outer(ue(0.0), amp))
        q = torch.empty(6 * g.N_int * R, dtype=torch.float64, device="cuda")
        k = torch.empty(6 * bd.size * R, dtype=torch.float64, device="cuda")
        t = 0.0
        for n in range(steps):  # the same q, k buffers every step (graph replay reads them)
            q.copy_(torch.from_numpy(np.stack([np.outer(qf(t + cj * dt), amp) for cj in c]).reshape(-1)))
            k.copy_(torch.from_numpy(np.stack([np.outer(kbc(t + cj * dt), amp) for cj in c]).reshape(-1)))
            S.ark_slope_step_batch(ub, t, dt, q=q, kbc=k, refine=2)
            t += dt
        torch.cuda.synchronize()
        return ub.cpu().numpy(), t

    eager, T = run(False)
    graphed, _ = run(True)
    assert np.array_equal(eager, graphed)
    for j in range(R):  # near the exact solution (time-dependent data, no order reduction)
        assert rel_max(eager[:, j], amp[j] * ue(T)) < 1e-6
    # and the FP64 slope step on column 1
    S.set_graph(False)
    u = to_dev(torch, amp[1] * ue(0.0))
    t = 0.0
    for n in range(5):
        S.ark_slope_step(u, t, dt, q=to_dev(torch, amp[1] * np.stack([qf(t + cj * dt) for cj in c]).reshape(-1)),
                         kbc=to_dev(torch, amp[1] * np.stack([kbc(t + cj * dt) for cj in c]).reshape(-1)))
        t += dt
    assert rel_max(eager[:, 1], u.cpu().numpy()) <= TOL
    S.close()


@pytest.mark.parametrize("gname,gp,nodal", [("allen_cahn", (1.5, 0.0), False), ("burgers", (0.7, -0.4), True)])
def test_slope_batch_with_g_matches_fp64(gname, gp, nodal):
    """The slope form with a nonlinear term on 4 states (explicit slopes by the batched leaf
    evaluation and edge projection) against the FP64 slope step column by column, and column 0
    against the oracle; states with flux jumps, a source, zero boundary data, 3 steps."""
    torch = need_gpu()
    from oracle import nonlinear
    from paper_2306_02526_gb300 import hps
    g = Grid(8, 4, 10)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = workloads.VarCoef128().coef(X[I], Y[I]) if nodal else {"a11": 0.8, "a22": 0.5, "a1": 0.2}
    R, dt = 4, 0.01
    c = hps.hps_ark_abscissae()
    U0 = 0.2 * np.random.default_rng(21).standard_normal((g.N, R))
    U0[bd, :] = 0.0
    qf = lambda t, j: (0.5 + 0.2 * j) * np.cos(X[I] + t) * np.sin(2 * Y[I] + j)
    S = _solver(torch, g, coef, 0.25 * dt)
    S.batch_reserve(R)
    ub = to_dev(torch, U0)
    us = [to_dev(torch, U0[:, j].copy()) for j in range(R)]
    t = 0.0
    for n in range(3):
        qb = np.stack([np.stack([qf(t + cj * dt, j) for j in range(R)], axis=1) for cj in c])
        S.ark_slope_step_batch(ub, t, dt, q=to_dev(torch, qb.reshape(-1)), g=gname, g_param=gp, refine=2)
        for j in range(R):
            S.ark_slope_step(us[j], t, dt, q=to_dev(torch, np.ascontiguousarray(qb[:, :, j]).reshape(-1)),
                             g=gname, g_param=gp)
        t += dt
    got = ub.cpu().numpy()
    for j in range(R):
        assert rel_max(got[:, j], us[j].cpu().numpy()) <= TOL, (j, rel_max(got[:, j], us[j].cpu().numpy()))
    gf = nonlinear.allen_cahn(gp[0]) if gname == "allen_cahn" else nonlinear.burgers(gp[0], gp[1])
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    u = U0[:, 0].copy()
    t = 0.0
    for n in range(3):
        u, _, _ = ark_slope.ark_slope_step_g(g, coef, Hi, Hid, u, t, dt, gf, q=lambda s: qf(s, 0))
        t += dt
    assert rel_max(got[:, 0], u) <= TOL
    S.status()
    S.close()
