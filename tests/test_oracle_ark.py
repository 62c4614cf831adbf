"""Pins for the oracle's additive Runge-Kutta step (eq. ``stage2``) and the stability
statements of Sec. 4: exactness in time, temporal order, the stability theorem."""
import numpy as np
import pytest

from oracle import ark, nonlinear
from oracle.grid import Grid
from oracle.hps import HPS

LAP = {"a11": 1.0, "a22": 1.0}


def run(prob, coef, u0, T, nsteps, **kw):
    dt = T / nsteps
    Hi, Hid = HPS(prob.grid, coef, 0.25 * dt), HPS(prob.grid, coef, 0.0)
    u, t = u0.copy(), 0.0
    for _ in range(nsteps):
        u, _ = ark.ark_step(prob, Hi, Hid, u, t, dt, **kw)
        t += dt
    return u


def test_exact_in_time_polynomial():
    """u = P + t Q with L Q = 0: every stage value is exact (row sums of both tables are c),
    so the step reproduces u to roundoff, including time-dependent boundary data."""
    g = Grid(2, 4, 6, 0.0, 1.0, -0.5, 0.5)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    ue = lambda t: X ** 2 + Y ** 2 + t * (X - Y + X * Y)
    prob = ark.Problem(g, LAP, q=lambda t: (X - Y + X * Y)[I] - 4.0, f=lambda t: ue(t)[bd])
    u = run(prob, LAP, ue(0.0), 0.7, 7)
    assert np.abs(u - ue(0.7)).max() < 1e-12


def heat_problem(g):
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    ue = lambda t: np.sin(np.pi * X) * np.sin(np.pi * Y) * np.exp(-t)
    prob = ark.Problem(g, LAP, q=lambda t: ((2 * np.pi ** 2 - 1) * ue(t))[I], f=lambda t: ue(t)[bd])
    return prob, ue


@pytest.mark.slow
def test_fourth_order_homogeneous_bc():
    """Sec. 5.3: about 4th order in dt for homogeneous boundary data."""
    g = Grid(2, 2, 16)
    prob, ue = heat_problem(g)
    errs = [np.abs(run(prob, LAP, ue(0.0), 1.0, n) - ue(1.0)).max() for n in (16, 32, 64)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 3.6 and rates[-1] < 4.4, (errs, rates)


def test_burgers_type_nonlinearity_fourth_order():
    """g = -u (u_x + u_y) by leaf-local differentiation with a manufactured source: 4th order."""
    g = Grid(2, 2, 12)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    eps = 0.1
    cf = {"a11": eps, "a22": eps}
    ue = lambda t: np.sin(np.pi * X) * np.sin(np.pi * Y) * np.exp(-t)

    def q(t):
        u = ue(t)
        ux = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y) * np.exp(-t)
        uy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.exp(-t)
        return (-u + eps * 2 * np.pi ** 2 * u + u * (ux + uy))[I]

    prob = ark.Problem(g, cf, q=q, f=lambda t: ue(t)[bd], g=nonlinear.burgers(1.0, 1.0))
    errs = [np.abs(run(prob, cf, ue(0.0), 1.0, n) - ue(1.0)).max() for n in (8, 16, 32)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 3.6, (errs, rates)


def _reaction_mms(g_fn, g_closed, kappa):
    """Manufactured solution u = 0.8 sin(pi x) sin(pi y) e^{-t} of u_t = eps Lap u + g(u) + q with
    q = u_t - eps Lap u - g_closed(u): the oracle's g must cancel the source's reaction term exactly,
    so a dropped factor or a wrong sign in g leaves an O(1) error instead of 4th-order convergence."""
    g = Grid(2, 2, 12)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    eps = 0.1
    cf = {"a11": eps, "a22": eps}
    ue = lambda t: 0.8 * np.sin(np.pi * X) * np.sin(np.pi * Y) * np.exp(-t)

    def q(t):
        u = ue(t)
        return (-u + eps * 2 * np.pi ** 2 * u - g_closed(u))[I]

    prob = ark.Problem(g, cf, q=q, f=lambda t: ue(t)[bd], g=g_fn(kappa))
    errs = [np.abs(run(prob, cf, ue(0.0), 1.0, n) - ue(1.0)).max() for n in (8, 16, 32)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    return errs, rates


def test_allen_cahn_manufactured_fourth_order():
    """g = kappa (u - u^3) (Sec. 5: Allen-Cahn reaction), kappa = 2.5: 4th order in dt with the
    manufactured source written from the equation, and small absolute error."""
    k = 2.5
    errs, rates = _reaction_mms(nonlinear.allen_cahn, lambda u: k * (u - u ** 3), k)
    assert rates[-1] > 3.6 and rates[-1] < 4.6, (errs, rates)
    assert errs[-1] < 1e-6, errs


def test_fisher_manufactured_fourth_order():
    """g = kappa u (1 - u) (Fisher-KPP reaction), kappa = 2.5: 4th order in dt with the manufactured
    source written from the equation, and small absolute error."""
    k = 2.5
    errs, rates = _reaction_mms(nonlinear.fisher, lambda u: k * u * (1.0 - u), k)
    assert rates[-1] > 3.6 and rates[-1] < 4.6, (errs, rates)
    assert errs[-1] < 1e-6, errs


def test_reaction_mms_detects_planted_errors():
    """The manufactured test above fails for a g with a dropped kappa or a flipped sign (mistakes
    planted in a copy of the oracle's g, on the CPU)."""
    k = 2.5
    dropped = lambda kappa: nonlinear.fisher(1.0)
    flipped = lambda kappa: (lambda grid, u: -nonlinear.allen_cahn(kappa)(grid, u))
    for bad, closed in ((dropped, lambda u: k * u * (1.0 - u)), (flipped, lambda u: k * (u - u ** 3))):
        errs, rates = _reaction_mms(bad, closed, k)
        assert errs[-1] > 1e-3, errs


def test_inhomogeneous_bc_converges_with_order_reduction():
    """Sec. 3.1.2 / Sec. 5.3: time-dependent Dirichlet data in the stage form loses order."""
    g = Grid(2, 2, 12)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    ue = lambda t: np.sin(np.pi * X) * np.exp(-t * (Y - 0.5) ** 2)

    def q(t):
        s = (Y - 0.5) ** 2
        u = ue(t)
        lap = -np.pi ** 2 * u + np.sin(np.pi * X) * np.exp(-t * s) * ((2 * t * (Y - 0.5)) ** 2 - 2 * t)
        return (-s * u - lap)[I]

    prob = ark.Problem(g, LAP, q=q, f=lambda t: ue(t)[bd])
    errs = [np.abs(run(prob, LAP, ue(0.0), 1.0, n) - ue(1.0)).max() for n in (8, 16, 32)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.6) and np.all(rates < 3.6), (errs, rates)


def test_stage_Lu_identity_matches_differentiation():
    """dt L u_j = (u_j - R_j)/gamma equals leaf-local differentiation of u_j to roundoff."""
    g = Grid(2, 2, 8)
    prob, ue = heat_problem(g)
    prob.g = nonlinear.allen_cahn(0.5)
    u0 = ue(0.0)
    a = run(prob, LAP, u0, 0.1, 2)
    b = run(prob, LAP, u0, 0.1, 2, lu_by_differentiation=True)
    assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


def step_matrix(step, N):
    M = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        M[:, k] = step(e)
    return M


@pytest.mark.parametrize("h", [1.0, 1e-2, 1e-4])
def test_backward_euler_stability_theorem(h):
    """Sec. 4.2 theorem: the BE + HPS time-step map of the heat equation has spectral radius
    <= 1.  Its kernel: every point that is not a leaf-interior point (the step reads u^n only
    at interior points; 2D reading of the zero-eigenvalue count of Sec. 4.2)."""
    g = Grid(2, 2, 6)
    H = HPS(g, LAP, h)
    prob = ark.Problem(g, LAP)
    M = step_matrix(lambda e: ark.backward_euler_step(prob, H, e, 0.0, h), g.N)
    ev = np.linalg.eigvals(M)
    assert np.abs(ev).max() <= 1.0 + 1e-12
    assert (np.abs(ev) < 1e-10).sum() == g.N - g.N_int
    assert np.all(M[:, g.N_int:] == 0.0)


@pytest.mark.parametrize("dt", [1.0, 1e-2, 1e-4])
def test_ark_step_map_eigenvalues(dt):
    """Sec. 4.2 (numerical evidence): eigenvalues of the ARK4 RKHPS step map lie in the unit disc."""
    g = Grid(2, 2, 6)
    Hi, Hid = HPS(g, LAP, 0.25 * dt), HPS(g, LAP, 0.0)
    prob = ark.Problem(g, LAP)
    M = step_matrix(lambda e: ark.ark_step(prob, Hi, Hid, e, 0.0, dt)[0], g.N)
    ev = np.linalg.eigvals(M)
    assert np.abs(ev).max() <= 1.0 + 1e-12
    assert (np.abs(ev) < 1e-10).sum() == g.N - g.N_int


def test_heat_energy_decays():
    """Heat equation, q = f = 0: the discrete 2-norm of smooth data never grows."""
    g = Grid(4, 4, 8)
    X, Y = g.coords()
    u = np.sin(np.pi * X) * np.sin(2 * np.pi * Y) + 0.3 * np.sin(3 * np.pi * X) * np.sin(np.pi * Y)
    prob = ark.Problem(g, LAP)
    dt = 0.01
    Hi, Hid = HPS(g, LAP, 0.25 * dt), HPS(g, LAP, 0.0)
    prev = np.linalg.norm(u)
    for n in range(20):
        u, _ = ark.ark_step(prob, Hi, Hid, u, n * dt, dt)
        cur = np.linalg.norm(u)
        assert cur <= prev * (1 + 1e-13)
        prev = cur


def test_allen_cahn_stays_bounded():
    """u_t = eps Lap u + u - u^3 with |u0| <= 0.1 keeps |u| <= 1 (maximum principle)."""
    g = Grid(4, 4, 8)
    X, Y = g.coords()
    rng = np.random.default_rng(0)
    u = 0.05 * np.sin(np.pi * X) * np.sin(np.pi * Y) + rng.uniform(-0.05, 0.05, g.N)
    u[g.boundary_indices()] = 0.0
    cf = {"a11": 0.01, "a22": 0.01}
    prob = ark.Problem(g, cf, g=nonlinear.allen_cahn(1.0))
    dt = 0.05
    Hi, Hid = HPS(g, cf, 0.25 * dt), HPS(g, cf, 0.0)
    for n in range(40):
        u, _ = ark.ark_step(prob, Hi, Hid, u, n * dt, dt)
        assert np.abs(u).max() <= 1.0
    assert np.abs(u).max() > 0.1  # the reaction term has grown the data
