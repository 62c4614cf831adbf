"""The step close's identity-operator system (Sec. 3.1.1: interior values given, boundary
values given, flux continuity on shared edges) splits, on a uniform leaf grid, into one
tridiagonal system per grid line of shared edges; the CUDA path solves it that way
(k_b_close_leaf + k_b_edge_tridiag).  This restates that formulation in NumPy, step for step
as the kernels take it (leaf flux sums, Thomas factors, forward and back substitution), and
checks it against the oracle's HPS solve with the identity operator."""
import numpy as np
import pytest

from oracle import cheb
from oracle.grid import Grid
from oracle.hps import HPS


def _project(g, rint, fb):
    p, m, q = g.p, g.m, g.m * g.m
    u = np.zeros(g.N)
    u[:g.N_int] = rint
    u[g.boundary_indices()] = fb
    rhs = np.zeros(g.N)
    D = [cheb.diff_matrix(p, g.hx), cheb.diff_matrix(p, g.hy)]
    for iy in range(g.n2):
        for ix in range(g.n1):
            l0 = (iy * g.n1 + ix) * q
            U = u[l0:l0 + q].reshape(m, m)  # [j-1][i-1]
            for r in range(m):
                for d in range(2):
                    line = U[r, :] if d == 0 else U[:, r]
                    f0, fl = D[d][0, 1:p - 1] @ line, D[d][p - 1, 1:p - 1] @ line
                    if d == 0:
                        if ix > 0:
                            rhs[g.vseg(ix, iy, r + 1)] += f0
                        if ix + 1 < g.n1:
                            rhs[g.vseg(ix + 1, iy, r + 1)] -= fl
                    else:
                        if iy > 0:
                            rhs[g.hseg(iy, ix, r + 1)] += f0
                        if iy + 1 < g.n2:
                            rhs[g.hseg(iy + 1, ix, r + 1)] -= fl
    for d in range(2):
        D1, n = D[d], (g.n2 if d else g.n1)
        lo, dd, up = D1[p - 1, 0], D1[p - 1, p - 1] - D1[0, 0], -D1[0, p - 1]
        assert abs(dd) > abs(lo) + abs(up)  # diagonally dominant: elimination without pivoting
        w, ib, b = np.zeros(max(n - 1, 0)), np.zeros(max(n - 1, 0)), dd
        for L in range(n - 1):
            if L > 0:
                w[L] = lo / b
                b = dd - w[L] * up
            ib[L] = 1.0 / b
        for a in range(g.n1 if d else g.n2):
            for node in range(1, m + 1):
                at = (lambda L: g.vseg(L, a, node)) if d == 0 else (lambda L: g.hseg(L, a, node))
                v0, vn, rp, rps = u[at(0)], u[at(n)], 0.0, {}
                for L in range(1, n):
                    r = rhs[at(L)] - (lo * v0 if L == 1 else 0.0) - (up * vn if L == n - 1 else 0.0)
                    rp = r if L == 1 else r - w[L - 1] * rp
                    rps[L] = rp
                v = 0.0
                for L in range(n - 1, 0, -1):
                    v = rps[L] * ib[L - 1] if L == n - 1 else (rps[L] - up * v) * ib[L - 1]
                    u[at(L)] = v
    return u


@pytest.mark.parametrize("n1,n2,p", [(5, 3, 8), (2, 4, 7), (1, 3, 6), (4, 1, 9), (6, 6, 16), (1, 1, 5)])
def test_edge_projection_equals_identity_hps_solve(n1, n2, p):
    g = Grid(n1, n2, p, 0.0, 1.3, -0.2, 0.9)
    rng = np.random.default_rng(n1 * 100 + n2 * 10 + p)
    rint = rng.standard_normal(g.N_int)
    fb = rng.standard_normal(len(g.boundary_indices()))
    ref = HPS(g, {"a11": 1.0, "a22": 1.0}, 0.0).solve(rint, fb)
    got = _project(g, rint, fb)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
