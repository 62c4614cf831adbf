"""Pins for the oracle's HPS build and solve (Sec. 2.1, Alg. 1) and its dense system
(eq. ``sparse_A``): brute force, polynomial exactness, spectral convergence, DtN meaning."""
import numpy as np
import pytest

from oracle import dense, residual
from oracle.grid import Grid
from oracle.hps import HPS
from oracle.residual import LeafField

TREES = [(1, 1, 4), (2, 1, 5), (1, 2, 6), (2, 2, 7), (4, 2, 5), (2, 4, 6), (4, 4, 8), (3, 2, 5)]


def random_coef(g, rng):
    return {"a11": 1.0 + 0.5 * rng.random(g.N_int), "a22": 0.6 + 0.4 * rng.random(g.N_int),
            "a1": 0.3 * rng.standard_normal(g.N_int), "a2": 0.25, "a0": -1.0 + 0.2 * rng.random(g.N_int)}


@pytest.mark.parametrize("n1,n2,p", TREES)
def test_hps_equals_dense_solve(n1, n2, p):
    """Sec. 3.1.1: the HPS result equals a direct solve of the global system to machine precision."""
    rng = np.random.default_rng(n1 * 100 + n2 * 10 + p)
    g = Grid(n1, n2, p, -0.3, 1.1, 0.2, 1.0)
    coef = random_coef(g, rng)
    gdt = 0.013
    H = HPS(g, coef, gdt)
    rhs = rng.standard_normal(g.N_int)
    f = rng.standard_normal(g.boundary_indices().size)
    jump = rng.standard_normal(g.N)
    u = H.solve(rhs, f, jump)
    ud = dense.solve(g, coef, gdt, rhs, f, jump)
    assert np.abs(u - ud).max() <= 1e-12 * np.abs(ud).max()
    # the leaf-local residual agrees with the dense residual
    r_loc = residual.residual(g, coef, gdt, u, rhs, f, jump)
    r_den = dense.residual(g, coef, gdt, u, rhs, f, jump)
    assert np.abs(r_loc - r_den).max() <= 1e-10 * (1 + np.abs(r_den).max())
    assert np.abs(r_loc).max() <= 1e-10 * np.abs(ud).max()


def poly_case(g, coef_fn, gdt):
    """u = x^3 y^2 + x y + 2 and the exact rhs of (I - gdt L) u at interior points."""
    X, Y = g.coords()
    u = X ** 3 * Y ** 2 + X * Y + 2.0
    ux, uy = 3 * X ** 2 * Y ** 2 + Y, 2 * X ** 3 * Y + X
    uxx, uyy = 6 * X * Y ** 2, 2 * X ** 3
    I = np.arange(g.N_int)
    c = coef_fn(X[I], Y[I])
    Lu = c["a11"] * uxx[I] + c["a22"] * uyy[I] + c["a1"] * ux[I] + c["a2"] * uy[I] + c["a0"] * u[I]
    rhs = u[I] - gdt * Lu
    return u, rhs, c


def var_coef(x, y):
    return {"a11": 1 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y), "a22": 1 + 0.3 * x * y,
            "a1": 0.5 + np.pi * np.cos(2 * np.pi * x), "a2": -0.25 + y, "a0": -1.0 + 0 * x}


@pytest.mark.parametrize("n1,n2,p", [(1, 1, 4), (2, 2, 5), (4, 2, 6), (4, 4, 8), (8, 8, 4)])
def test_polynomial_exactness(n1, n2, p):
    """A polynomial of degree <= p-1 per variable is reproduced to roundoff (collocation is exact)."""
    g = Grid(n1, n2, p)
    gdt = 0.05
    u, rhs, c = poly_case(g, var_coef, gdt)
    bd = g.boundary_indices()
    H = HPS(g, c, gdt)
    uh = H.solve(rhs, u[bd])
    assert np.abs(uh - u).max() <= 1e-12 * np.abs(u).max() * p ** 2
    if g.N <= 1200:
        ud = dense.solve(g, c, gdt, rhs, u[bd])
        assert np.abs(ud - u).max() <= 1e-12 * np.abs(u).max() * p ** 2


def test_spectral_convergence_in_p():
    """Smooth exact solution of (I - L) u = rhs, L = Laplacian: the error decays exponentially in p."""
    errs = []
    for p in (5, 7, 9, 11, 13):
        g = Grid(2, 2, p)
        X, Y = g.coords()
        u = np.sin(np.pi * X) * np.cosh(Y) + np.exp(X * Y)
        lap = -np.pi ** 2 * np.sin(np.pi * X) * np.cosh(Y) + np.sin(np.pi * X) * np.cosh(Y) \
            + (X ** 2 + Y ** 2) * np.exp(X * Y)
        I = np.arange(g.N_int)
        H = HPS(g, {"a11": 1.0, "a22": 1.0}, 1.0)
        uh = H.solve(u[I] - lap[I], u[g.boundary_indices()])
        errs.append(np.abs(uh - u).max())
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1] / 20.0), errs
    assert errs[-1] < 1e-10


def test_merged_dtn_maps_boundary_data_to_fluxes():
    """T of a merged node is the DtN map (Sec. 2.1): with zero body load, T f equals the
    boundary fluxes (d/dx on vertical sides, d/dy on horizontal ones) of the solution."""
    rng = np.random.default_rng(3)
    g = Grid(2, 2, 6)
    coef = random_coef(g, rng)
    H = HPS(g, coef, 0.02)
    bd = g.boundary_indices()
    root = H.root
    f_box = rng.standard_normal(root.bd.size)
    f = np.zeros(g.N)
    f[root.bd] = f_box
    u = H.solve(np.zeros(g.N_int), f[bd])
    F = LeafField(g, u)
    p, m = g.p, g.m
    flux = []
    # root box order: south, east, north, west; each side leaf by leaf
    for ix in range(g.n1):
        flux.extend(F.Uy[g.leaf_id(ix, 0), 0, 1:-1])
    for iy in range(g.n2):
        flux.extend(F.Ux[g.leaf_id(g.n1 - 1, iy), 1:-1, p - 1])
    for ix in range(g.n1):
        flux.extend(F.Uy[g.leaf_id(ix, g.n2 - 1), p - 1, 1:-1])
    for iy in range(g.n2):
        flux.extend(F.Ux[g.leaf_id(0, iy), 1:-1, 0])
    flux = np.array(flux)
    assert flux.size == 4 * 2 * m
    assert np.abs(root.T @ f_box - flux).max() <= 1e-10 * np.abs(flux).max()


def test_wrong_flux_sign_is_caught():
    """Plant a mistake in a copy of the oracle (flip the sign of one merge's S): the dense pin fails."""
    rng = np.random.default_rng(5)
    g = Grid(2, 2, 5)
    coef = random_coef(g, rng)
    H = HPS(g, coef, 0.01)
    H.root.S = -H.root.S
    rhs = rng.standard_normal(g.N_int)
    f = rng.standard_normal(g.boundary_indices().size)
    u = H.solve(rhs, f)
    ud = dense.solve(g, coef, 0.01, rhs, f)
    assert np.abs(u - ud).max() > 1e-3 * np.abs(ud).max()


def test_grid_counts_and_ordering():
    g = Grid(4, 2, 7)
    assert g.N == (g.p - 2) * (g.p * 4 * 2 + 4 + 2)  # Sec. 2.1
    X, Y = g.coords()
    assert len(set(zip(np.round(X, 14), np.round(Y, 14)))) == g.N  # no duplicate points
    bd = g.boundary_indices()
    on_bd = (np.isclose(X, 0) | np.isclose(X, 1) | np.isclose(Y, 0) | np.isclose(Y, 1))
    assert set(np.nonzero(on_bd)[0].tolist()) == set(bd.tolist())
    assert bd.size == 2 * g.m * (g.n1 + g.n2)
