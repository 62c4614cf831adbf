"""ark_slope_step (slope form, g = 0, penalized interface rows; libhps.so through its C ABI)
against the oracle's slope-form step, element by element; FP64 tolerance 1e-12."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle import ark_slope
from oracle.grid import Grid
from oracle.hps import HPS
from paper_2306_02526_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _solver(torch, g, coef, gdt):
    from paper_2306_02526_gb300 import hps
    tree = hps.Tree(g.n1, g.n2, g.x0, g.x1, g.y0, g.y1)
    cg = {k: (to_dev(torch, v) if np.ndim(v) else float(v)) for k, v in coef.items()}
    return hps.HPSSolver(tree, g.p, cg, gdt)


@pytest.mark.parametrize("nodal", [False, True])
def test_slope_step_with_flux_jumps_matches_oracle(nodal):
    """A state with flux jumps on every shared edge (the penalization acts), a source, zero
    boundary data; constant (fast-diagonalization leaves) or nodal coefficients; 3 steps."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    g = Grid(4, 2, 9)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = workloads.VarCoef128().coef(X[I], Y[I]) if nodal else {"a11": 0.8, "a22": 0.5, "a1": 0.2}
    dt = 0.01
    c = hps.hps_ark_abscissae()
    qf = lambda t: np.cos(X[I] + t) * np.sin(2 * Y[I])
    rng = np.random.default_rng(11)
    u = rng.standard_normal(g.N)
    u[bd] = 0.0
    S = _solver(torch, g, coef, 0.25 * dt)
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    ug = to_dev(torch, u)
    t = 0.0
    for n in range(3):
        S.ark_slope_step(ug, t, dt, q=to_dev(torch, np.stack([qf(t + cj * dt) for cj in c]).reshape(-1)))
        u, _ = ark_slope.ark_slope_step(g, coef, Hi, Hid, u, t, dt, q=qf)
        t += dt
        assert rel_max(ug.cpu().numpy(), u) <= TOL, n
    S.close()


def test_slope_step_with_u_t_boundary_data_matches_oracle():
    """Time-dependent Dirichlet data with the slopes' boundary data u_t (no order reduction)."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    g = Grid(2, 4, 10)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = {"a11": 1.0, "a22": 1.0}
    s2 = (Y - 0.5) ** 2
    ue = lambda t: np.sin(np.pi * X) * np.exp(-t * s2)

    def q(t):
        u = ue(t)
        lap = -np.pi ** 2 * u + np.sin(np.pi * X) * np.exp(-t * s2) * ((2 * t * (Y - 0.5)) ** 2 - 2 * t)
        return (-s2 * u - lap)[I]

    kbc = lambda t: (-s2 * ue(t))[bd]
    dt = 0.05
    c = hps.hps_ark_abscissae()
    S = _solver(torch, g, coef, 0.25 * dt)
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    u = ue(0.0)
    ug = to_dev(torch, u)
    t = 0.0
    for n in range(4):
        S.ark_slope_step(ug, t, dt, q=to_dev(torch, np.stack([q(t + cj * dt) for cj in c]).reshape(-1)),
                         kbc=to_dev(torch, np.stack([kbc(t + cj * dt) for cj in c]).reshape(-1)))
        u, _ = ark_slope.ark_slope_step(g, coef, Hi, Hid, u, t, dt, q=q, kbc=kbc)
        t += dt
        assert rel_max(ug.cpu().numpy(), u) <= TOL, n
    assert np.abs(ug.cpu().numpy() - ue(t)).max() < 1e-5
    S.close()


def test_slope_step_rejects_unsupported_cases():
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib
    S = _solver(torch, Grid(1, 1, 6), {"a11": 1.0, "a22": 1.0}, 0.25 * 0.01)
    u = torch.zeros(S.N, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.HPSError):  # a single leaf has no shared edges
        S.ark_slope_step(u, 0.0, 0.01)
    S.close()


@pytest.mark.parametrize("gname,gp,nodal", [("allen_cahn", (1.5, 0.0), False), ("fisher", (0.8, 0.0), True),
                                            ("burgers", (0.7, -0.4), False)])
def test_slope_step_with_g_matches_oracle(gname, gp, nodal):
    """The slope form with a nonlinear term (eq. slope): a state with flux jumps on every shared
    edge, a source, time-independent (zero) boundary data; 3 steps against the oracle's
    ark_slope_step_g at the FP64 tolerance."""
    torch = need_gpu()
    from oracle import nonlinear
    from paper_2306_02526_gb300 import hps
    g = Grid(4, 2, 10)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = workloads.VarCoef128().coef(X[I], Y[I]) if nodal else {"a11": 0.8, "a22": 0.5, "a1": 0.2, "a0": -0.1}
    gf = {"allen_cahn": lambda: nonlinear.allen_cahn(gp[0]), "fisher": lambda: nonlinear.fisher(gp[0]),
          "burgers": lambda: nonlinear.burgers(gp[0], gp[1])}[gname]()
    dt = 0.01
    c = hps.hps_ark_abscissae()
    qf = lambda t: 0.5 * np.cos(X[I] + t) * np.sin(2 * Y[I])
    u = 0.2 * np.random.default_rng(13).standard_normal(g.N)
    u[bd] = 0.0
    S = _solver(torch, g, coef, 0.25 * dt)
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    ug = to_dev(torch, u)
    t = 0.0
    for n in range(3):
        S.ark_slope_step(ug, t, dt, q=to_dev(torch, np.stack([qf(t + cj * dt) for cj in c]).reshape(-1)),
                         g=gname, g_param=gp)
        u, _, _ = ark_slope.ark_slope_step_g(g, coef, Hi, Hid, u, t, dt, gf, q=qf)
        t += dt
        assert rel_max(ug.cpu().numpy(), u) <= TOL, (n, rel_max(ug.cpu().numpy(), u))
    from paper_2306_02526_gb300 import _lib
    with pytest.raises(_lib.HPSError):  # with g, time-dependent slope boundary data are not accepted
        S.ark_slope_step(ug, t, dt, kbc=torch.zeros(6 * g.boundary_indices().size, dtype=torch.float64,
                                                   device="cuda"), g=gname, g_param=gp)
    S.close()
