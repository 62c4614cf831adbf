"""Pins for the oracle's slope-form ARK step (Sec. 3.1, eq. ``slope0``, g = 0) with the
penalized interface conditions: exactness in time, algebraic equivalence with the stage form,
the penalization's effect on flux jumps, and the order with time-dependent boundary data."""
import numpy as np

from oracle import ark, ark_slope
from oracle.grid import Grid
from oracle.hps import HPS
from oracle.residual import flux_jumps

LAP = {"a11": 1.0, "a22": 1.0}


def test_slope_form_exact_in_time_polynomial():
    """u = P + t Q with L Q = 0 and u_t = Q given on the boundary: every slope equals Q exactly
    (row sums of A are c), so the step reproduces u to roundoff."""
    g = Grid(2, 4, 6, 0.0, 1.0, -0.5, 0.5)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    Q = X - Y + X * Y
    ue = lambda t: X ** 2 + Y ** 2 + t * Q
    dt = 0.1
    Hi, Hid = HPS(g, LAP, 0.25 * dt), HPS(g, LAP, 0.0)
    u, t = ue(0.0), 0.0
    for _ in range(7):
        u, ks = ark_slope.ark_slope_step(g, LAP, Hi, Hid, u, t, dt, q=lambda tt: (Q - 4.0)[I],
                                         kbc=lambda tt: Q[bd])
        t += dt
    assert np.abs(u - ue(0.7)).max() < 1e-12
    assert max(np.abs(k - Q).max() for k in ks) < 1e-10


def test_slope_form_equals_stage_form_without_sources():
    """q = g = 0, zero boundary data, a state without flux jumps: the slope and stage forms are
    the same method (k_i = L U_i), so one step agrees to roundoff (1e-12 relative)."""
    g = Grid(4, 2, 10)
    rng = np.random.default_rng(3)
    dt = 0.01
    coef = {"a11": 1.0, "a22": 0.7, "a1": 0.3}
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    u0 = Hid.solve(rng.standard_normal(g.N_int), None)  # flux-continuous, zero on the boundary
    us, _ = ark_slope.ark_slope_step(g, coef, Hi, Hid, u0, 0.0, dt)
    ua, _ = ark.ark_step(ark.Problem(g, coef), Hi, Hid, u0, 0.0, dt)
    assert np.abs(us - ua).max() <= 1e-11 * np.abs(ua).max()


def test_penalization_removes_the_flux_jump():
    """With the penalized interface rows u^{n+1} has no flux jump whatever the jump of u^n;
    without them the jump of u^n is carried over unchanged (Sec. 3.1, penalization)."""
    g = Grid(4, 2, 10)
    rng = np.random.default_rng(5)
    dt = 0.01
    coef = {"a11": 1.0, "a22": 0.7}
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    u = rng.standard_normal(g.N)
    u[g.boundary_indices()] = 0.0
    ii = g.interface_indices()
    j0 = np.abs(flux_jumps(g, u)[ii]).max()
    up, _ = ark_slope.ark_slope_step(g, coef, Hi, Hid, u, 0.0, dt)
    un, _ = ark_slope.ark_slope_step(g, coef, Hi, Hid, u, 0.0, dt, penalize=False)
    assert np.abs(flux_jumps(g, up)[ii]).max() <= 1e-12 * j0
    assert np.abs(flux_jumps(g, un)[ii] - flux_jumps(g, u)[ii]).max() <= 1e-12 * j0


def test_slope_form_with_u_t_boundary_data_avoids_order_reduction():
    """Time-dependent Dirichlet data (the stage form's order-reduction case): slopes with
    boundary data u_t converge at about 4th order and far below the stage form's error."""
    g = Grid(2, 2, 12)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    s2 = (Y - 0.5) ** 2
    ue = lambda t: np.sin(np.pi * X) * np.exp(-t * s2)

    def q(t):
        u = ue(t)
        lap = -np.pi ** 2 * u + np.sin(np.pi * X) * np.exp(-t * s2) * ((2 * t * (Y - 0.5)) ** 2 - 2 * t)
        return (-s2 * u - lap)[I]

    prob = ark.Problem(g, LAP, q=q, f=lambda t: ue(t)[bd])
    es, ea = [], []
    for n in (8, 16, 32):
        dt = 1.0 / n
        Hi, Hid = HPS(g, LAP, 0.25 * dt), HPS(g, LAP, 0.0)
        us, ua, t = ue(0.0), ue(0.0), 0.0
        for _ in range(n):
            us, _ = ark_slope.ark_slope_step(g, LAP, Hi, Hid, us, t, dt, q=q, kbc=lambda tt: (-s2 * ue(tt))[bd])
            ua, _ = ark.ark_step(prob, Hi, Hid, ua, t, dt)
            t += dt
        es.append(np.abs(us - ue(1.0)).max())
        ea.append(np.abs(ua - ue(1.0)).max())
    rates = np.log2(np.array(es[:-1]) / np.array(es[1:]))
    assert rates[-1] > 3.3, (es, rates)
    assert es[-1] < 0.1 * ea[-1], (es, ea)


# ---- the slope form with a nonlinear term (eq. ``slope``, ark_slope_step_g) -----------------
def _g_problem():
    """Manufactured u* = e^-t sin(pi x) sin(pi y) + (x^2 - y^2)/2 (time-independent boundary data,
    the case the paper gives slope boundary conditions for), variable-order L with first and
    zeroth-order terms, Allen-Cahn g with kappa = 0.5: q = u*_t - L u* - g(u*)."""
    from oracle import nonlinear
    g = Grid(2, 2, 16)
    X, Y = g.coords()
    I = np.arange(g.N_int)
    coef = {"a11": 0.2, "a22": 0.15, "a1": 0.1, "a0": -0.3}
    kap = 0.5

    def ue(t):
        return np.exp(-t) * np.sin(np.pi * X) * np.sin(np.pi * Y) + 0.5 * (X ** 2 - Y ** 2)

    def q(t):
        e, s = np.exp(-t), np.sin(np.pi * X) * np.sin(np.pi * Y)
        u = ue(t)
        ux = e * np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y) + X
        uxx, uyy = -e * np.pi ** 2 * s + 1.0, -e * np.pi ** 2 * s - 1.0
        Lu = coef["a11"] * uxx + coef["a22"] * uyy + coef["a1"] * ux + coef["a0"] * u
        return (-e * s - Lu - kap * (u - u ** 3))[I]

    return g, coef, nonlinear.allen_cahn(kap), ue, q


def _g_errors(dts, T=0.4):
    g, coef, gf, ue, q = _g_problem()
    errs = []
    for dt in dts:
        Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
        u, t = ue(0.0), 0.0
        for _ in range(int(round(T / dt))):
            u, _, _ = ark_slope.ark_slope_step_g(g, coef, Hi, Hid, u, t, dt, gf, q=q)
            t += dt
        errs.append(np.abs(u - ue(T)).max())
    return np.array(errs)


def test_slope_form_with_g_converges_at_high_order():
    """Against the manufactured solution the slope form with g converges at order about 3 to 3.5
    (measured 3.0, 3.5, 3.0) and reaches 3e-8 at dt = 0.025 (the stage form on the same problem:
    order about 2, 6e-7)."""
    errs = _g_errors((0.1, 0.05, 0.025))
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates > 2.7), (errs, rates)
    assert errs[-1] < 5e-8, errs


def test_slope_form_with_g_detects_planted_errors(monkeypatch):
    """The same test fails for mistakes planted in the tableau the oracle reads (a copy, on the
    CPU): the explicit table replaced by the implicit one, the explicit table or the explicit
    weights dropped."""
    from oracle import tableau
    A, b, c, Ah, bh = tableau.as_float()
    for bad in ((A, b, c, A, bh), (A, b, c, 0 * Ah, bh), (A, b, c, Ah, 0 * bh)):
        monkeypatch.setattr(tableau, "as_float", lambda bad=bad: bad)
        errs = _g_errors((0.05,))
        assert errs[0] > 1e-4, errs
    monkeypatch.undo()


def test_slope_form_with_g_removes_the_flux_jump_and_reduces_to_slope0():
    """A state with flux jumps on every shared edge: after one step with g the flux jump is gone
    (the l_i carry none, the k_i cancel that of u^n); with g = 0 the step is exactly the g-free
    slope step."""
    from oracle import nonlinear
    g = Grid(4, 2, 10)
    coef = {"a11": 1.0, "a22": 0.7, "a1": 0.3}
    dt = 0.01
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    u = 0.3 * np.random.default_rng(5).standard_normal(g.N)
    u[g.boundary_indices()] = 0.0
    assert np.abs(flux_jumps(g, u)).max() > 1.0
    u1, _, ls = ark_slope.ark_slope_step_g(g, coef, Hi, Hid, u, 0.0, dt, nonlinear.fisher(2.0))
    assert np.abs(flux_jumps(g, u1)).max() < 1e-9 * np.abs(u1).max() * 100
    assert max(np.abs(flux_jumps(g, lf)).max() for lf in ls) < 1e-9
    zero = lambda grid, v: np.zeros(grid.N_int)
    a, _, _ = ark_slope.ark_slope_step_g(g, coef, Hi, Hid, u, 0.0, dt, zero)
    b, _ = ark_slope.ark_slope_step(g, coef, Hi, Hid, u, 0.0, dt)
    assert np.array_equal(a, b)
