"""GPU (libhps.so through its C ABI) vs the CPU oracle, element by element.

Tolerance: the FP64 GPU path must match the FP64 oracle to 1e-12 relative max-norm
(both solve the same collocation system; only rounding order differs)."""
import math

import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle import ark as oark
from oracle import dense, nonlinear, residual
from oracle.grid import Grid
from oracle.hps import HPS
from paper_2306_02526_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12

SOLVE_CASES = [  # (n1, n2, p): one leaf, rectangles, several tiles, ragged row lengths
    (1, 1, 4), (2, 1, 5), (1, 2, 6), (2, 2, 8), (4, 2, 7), (2, 8, 9), (8, 8, 10), (4, 4, 16), (16, 8, 12), (8, 16, 13),
]


def _gpu_solver(torch, n1, n2, p, coef, gdt, dom=(0.0, 1.0, 0.0, 1.0), per_node=False):
    from paper_2306_02526_gb300 import hps
    tree = hps.Tree(n1, n2, *dom)
    cg = {k: (to_dev(torch, v) if np.ndim(v) else float(v)) for k, v in coef.items()}
    return hps.HPSSolver(tree, p, cg, gdt, per_node=per_node)


@pytest.mark.parametrize("n1,n2,p", SOLVE_CASES)
@pytest.mark.parametrize("kind", ["const", "nodal"])
def test_hps_solve_matches_oracle(n1, n2, p, kind):
    torch = need_gpu()
    dom = (-0.3, 1.1, 0.2, 1.0)
    g = Grid(n1, n2, p, *dom)
    r = np.random.default_rng(n1 * 1000 + n2 * 10 + p)
    if kind == "const":
        coef = {"a11": 1.3, "a22": 0.7, "a1": 0.4, "a2": -0.2, "a0": -1.0}
    else:
        coef = workloads.random_coefficients(p, g.N_int)
    gdt = 0.0123
    rhs = r.standard_normal(g.N_int)
    f = r.standard_normal(g.boundary_indices().size)
    want = HPS(g, coef, gdt).solve(rhs, f)
    S = _gpu_solver(torch, n1, n2, p, coef, gdt, dom)
    got = S.solve(to_dev(torch, rhs), to_dev(torch, f)).cpu().numpy()
    assert rel_max(got, want) <= TOL
    if g.N <= 1500:
        assert rel_max(got, dense.solve(g, coef, gdt, rhs, f)) <= 10 * TOL


def test_per_node_layout_equals_shared():
    """A constant-coefficient problem gives the same answer with one operator per node."""
    torch = need_gpu()
    coef = {"a11": 1.0, "a22": 2.0, "a1": 0.1, "a2": 0.0, "a0": 0.5}
    g = Grid(8, 4, 9)
    r = np.random.default_rng(1)
    rhs, f = r.standard_normal(g.N_int), r.standard_normal(g.boundary_indices().size)
    a = _gpu_solver(torch, 8, 4, 9, coef, 0.01).solve(to_dev(torch, rhs), to_dev(torch, f)).cpu().numpy()
    b = _gpu_solver(torch, 8, 4, 9, coef, 0.01, per_node=True).solve(to_dev(torch, rhs), to_dev(torch, f)).cpu().numpy()
    assert rel_max(a, b) <= TOL


def test_zero_rhs_zero_solution_and_repeatability():
    torch = need_gpu()
    S = _gpu_solver(torch, 4, 4, 8, {"a11": 1.0, "a22": 1.0}, 0.01)
    z = torch.zeros(S.N_int, dtype=torch.float64, device="cuda")
    assert float(S.solve(z).abs().max()) == 0.0
    r = to_dev(torch, np.random.default_rng(2).standard_normal(S.N_int))
    u1 = S.solve(r).cpu().numpy()
    u2 = S.solve(r).cpu().numpy()
    assert np.array_equal(u1, u2)  # deterministic: no atomics in the sweep


def _stage_inputs(torch, wl, g, t, dt, c):
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    q = f = None
    if wl.q(X, Y, 0.0) is not None:
        q = np.stack([wl.q(X, Y, t + cj * dt)[I] for cj in c])
    if wl.f(X, Y, 0.0) is not None:
        f = np.stack([wl.f(X, Y, t + cj * dt)[bd] for cj in c])
    return (None if q is None else to_dev(torch, q.reshape(-1)), None if f is None else to_dev(torch, f.reshape(-1)))


def test_ark_heat_trajectory_matches_oracle():
    """Heat 4x4 leaves, p = 8, dt = 0.01, 100 ARK4 steps: every step within 1e-12 of the oracle."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    wl = workloads.Heat4x4()
    g = Grid(wl.n1, wl.n2, wl.p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = wl.coef(X[I], Y[I])
    prob = oark.Problem(g, coef, q=lambda t: wl.q(X, Y, t)[I])
    Hi, Hid = HPS(g, coef, 0.25 * wl.dt), HPS(g, coef, 0.0)
    S = _gpu_solver(torch, wl.n1, wl.n2, wl.p, coef, 0.25 * wl.dt)
    c = hps.hps_ark_abscissae()
    u_or = wl.u0(X, Y, bd)
    u_gpu = to_dev(torch, u_or)
    t = 0.0
    worst = 0.0
    for n in range(wl.steps):
        q, f = _stage_inputs(torch, wl, g, t, wl.dt, c)
        S.ark_step(u_gpu, t, wl.dt, q=q, f=f)
        u_or, _ = oark.ark_step(prob, Hi, Hid, u_or, t, wl.dt)
        t += wl.dt
        worst = max(worst, rel_max(u_gpu.cpu().numpy(), u_or))
    assert worst <= TOL
    # and the discrete solution is close to the exact one (spatial + temporal error)
    assert np.abs(u_gpu.cpu().numpy() - wl.exact(X, Y, t)).max() < 1e-5


@pytest.mark.parametrize("gname,close", [("allen_cahn", "projection"), ("fisher", "projection"),
                                         ("burgers", "projection"), ("allen_cahn", "sweep")])
def test_ark_nonlinear_and_inhomogeneous_match_oracle(gname, close):
    """Variable coefficients, time-dependent boundary data, a source and each g preset; the step
    close by the edge projection (default) and by the identity-operator sweep."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    n1, n2, p, dt = 4, 8, 9, 0.02
    g = Grid(n1, n2, p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = workloads.VarCoef128().coef(X[I], Y[I])
    qf = lambda t: np.cos(X[I] + t) * np.sin(2 * Y[I])
    ff = lambda t: (np.sin(X + 2 * Y) * (1 + t))[bd]
    gp = (0.7, -0.4)
    gfun = {"allen_cahn": nonlinear.allen_cahn(gp[0]), "fisher": nonlinear.fisher(gp[0]),
            "burgers": nonlinear.burgers(*gp)}[gname]
    prob = oark.Problem(g, coef, q=qf, f=ff, g=gfun)
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    S = _gpu_solver(torch, n1, n2, p, coef, 0.25 * dt)
    if close == "sweep":
        S.batch_option("edge_projection", 0)
        S.batch_option("fp64_plan_target", 1)  # and another split plan of the FP64 merge applies
    c = hps.hps_ark_abscissae()
    u_or = 0.3 * np.sin(math.pi * X) * np.cos(Y)
    u_or[bd] = ff(0.0)
    u_gpu = to_dev(torch, u_or)
    t = 0.0
    for n in range(5):
        q = to_dev(torch, np.stack([qf(t + cj * dt) for cj in c]).reshape(-1))
        f = to_dev(torch, np.stack([ff(t + cj * dt) for cj in c]).reshape(-1))
        S.ark_step(u_gpu, t, dt, q=q, f=f, g=gname, g_param=gp)
        u_or, _ = oark.ark_step(prob, Hi, Hid, u_or, t, dt)
        t += dt
        assert rel_max(u_gpu.cpu().numpy(), u_or) <= TOL


@pytest.mark.parametrize("n1,n2,p", [(1, 1, 5), (2, 1, 6), (1, 4, 7), (8, 2, 9), (4, 4, 16)])
def test_ark_close_on_degenerate_trees_matches_oracle(n1, n2, p):
    """Step close (edge projection: one tridiagonal system per grid line of shared edges) on a
    single leaf, single rows / columns of leaves, odd p and a rectangle: 3 ARK steps with a
    source and time-dependent boundary data against the oracle."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    dt = 0.02
    g = Grid(n1, n2, p, 0.0, 1.0, 0.0, 0.5)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = {"a11": 0.5, "a22": 0.8, "a1": 0.3, "a0": -0.2}
    qf = lambda t: np.cos(X[I] - t) * np.sin(3 * Y[I])
    ff = lambda t: (np.sin(2 * X + Y) * (1 - t))[bd]
    prob = oark.Problem(g, coef, q=qf, f=ff, g=nonlinear.allen_cahn(0.5))
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    S = _gpu_solver(torch, n1, n2, p, coef, 0.25 * dt, dom=(0.0, 1.0, 0.0, 0.5))
    c = hps.hps_ark_abscissae()
    u_or = 0.2 * np.cos(2 * X) * np.sin(5 * Y)
    u_or[bd] = ff(0.0)
    u_gpu = to_dev(torch, u_or)
    t = 0.0
    for n in range(3):
        q = to_dev(torch, np.stack([qf(t + cj * dt) for cj in c]).reshape(-1))
        f = to_dev(torch, np.stack([ff(t + cj * dt) for cj in c]).reshape(-1))
        S.ark_step(u_gpu, t, dt, q=q, f=f, g="allen_cahn", g_param=(0.5, 0.0))
        u_or, _ = oark.ark_step(prob, Hi, Hid, u_or, t, dt)
        t += dt
        assert rel_max(u_gpu.cpu().numpy(), u_or) <= TOL


def test_ark_rejects_wrong_dt():
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib
    S = _gpu_solver(torch, 2, 2, 6, {"a11": 1.0, "a22": 1.0}, 0.25 * 0.01)
    u = torch.zeros(S.N, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.HPSError) as e:
        S.ark_step(u, 0.0, 0.02)
    assert e.value.code == _lib.HPS_EDT


def test_allen_cahn_full_size_step_matches_oracle():
    """The bench workload (64x64 leaves, p = 16, N = 919,296): one ARK step, every entry
    against the oracle, plus the leaf-local residual of one full-size stage solve."""
    torch = need_gpu()
    wl = workloads.AllenCahn64()
    g = Grid(wl.n1, wl.n2, wl.p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = wl.coef(X[I], Y[I])
    S = _gpu_solver(torch, wl.n1, wl.n2, wl.p, coef, 0.25 * wl.dt)
    # stage-solve residual of eq. sparse_A, evaluated leaf by leaf (no dense matrix)
    rhs = np.random.default_rng(7).standard_normal(g.N_int)
    u = S.solve(to_dev(torch, rhs)).cpu().numpy()
    res = residual.residual(g, coef, 0.25 * wl.dt, u, rhs)
    assert np.abs(res).max() <= 1e-10 * np.abs(u).max()
    # one full ARK step against the oracle
    u0 = wl.u0(X, Y, bd)
    prob = oark.Problem(g, coef, g=nonlinear.allen_cahn(1.0))
    want, _ = oark.ark_step(prob, HPS(g, coef, 0.25 * wl.dt), HPS(g, coef, 0.0), u0, 0.0, wl.dt)
    ug = to_dev(torch, u0)
    S.ark_step(ug, 0.0, wl.dt, g="allen_cahn", g_param=(1.0, 0.0))
    assert rel_max(ug.cpu().numpy(), want) <= TOL
