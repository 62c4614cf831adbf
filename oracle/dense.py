"""The global collocation system of eq. ``sparse_A`` (Sec. 2.1), assembled densely.

Row types (one row per global point, corners excluded):
  * leaf interior point  -> (A u)(x_i) with A = I - gamma_dt L, the collocated PDE;
  * edge point shared by two leaves -> flux continuity: the derivative across the edge
    (d/dx on a vertical edge, d/dy on a horizontal one) computed in the west/south leaf
    minus the same derivative computed in the east/north leaf;
  * point on the outer boundary -> u = f.

The paper lists the outer-boundary rows as "+-du/dn"; for the Dirichlet problem solved here
(Alg. 1 sets u = f there) these rows are read as identity rows.  The HPS solver reaches the
solution of exactly this system (Sec. 3.1.1 reports agreement to machine precision), so the
dense solve is the brute-force pin of the whole HPS path.  Only for tiny N.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from .grid import Grid
from .leaf import collocation_L_rows, full_derivatives, local_sets
from .hps import coefficient_slices


def assemble(grid: Grid, coef, gamma_dt):
    """Dense N x N matrix of eq. ``sparse_A`` for the operator I - gamma_dt L."""
    p, m, N = grid.p, grid.m, grid.N
    A = np.zeros((N, N))
    I_loc, _, _ = local_sets(p)
    slices = coefficient_slices(grid, coef)
    Dx, Dy = full_derivatives(p, grid.hx, grid.hy)
    Id = np.eye(p * p)
    filled = np.zeros(N, dtype=bool)
    maps = {}
    for iy in range(grid.n2):
        for ix in range(grid.n1):
            g = grid.local_to_global(ix, iy).reshape(-1)
            maps[(ix, iy)] = g
            rows = Id[I_loc] - gamma_dt * collocation_L_rows(p, grid.hx, grid.hy, slices[(ix, iy)])
            for r, loc in enumerate(I_loc):
                gi = g[loc]
                for col in np.nonzero(rows[r])[0]:
                    assert g[col] >= 0
                    A[gi, g[col]] += rows[r, col]
                filled[gi] = True

    def add_flux_row(row_g, leaf, loc, D, sign):
        g = maps[leaf]
        for col in np.nonzero(D[loc])[0]:
            assert g[col] >= 0
            A[row_g, g[col]] += sign * D[loc, col]

    # vertical interfaces: x-line L between leaf (L-1, iy) (west) and (L, iy) (east)
    for L in range(1, grid.n1):
        for iy in range(grid.n2):
            for j in range(1, m + 1):
                gi = grid.vseg(L, iy, j)
                add_flux_row(gi, (L - 1, iy), j * p + (p - 1), Dx, +1.0)
                add_flux_row(gi, (L, iy), j * p + 0, Dx, -1.0)
                filled[gi] = True
    # horizontal interfaces: y-line L between leaf (ix, L-1) (south) and (ix, L) (north)
    for L in range(1, grid.n2):
        for ix in range(grid.n1):
            for i in range(1, m + 1):
                gi = grid.hseg(L, ix, i)
                add_flux_row(gi, (ix, L - 1), (p - 1) * p + i, Dy, +1.0)
                add_flux_row(gi, (ix, L), 0 * p + i, Dy, -1.0)
                filled[gi] = True
    for gi in grid.boundary_indices():
        A[gi, gi] = 1.0
        filled[gi] = True
    assert filled.all()
    return A


def rhs_vector(grid: Grid, rhs_int, f_bd=None, jump=None):
    b = np.zeros(grid.N)
    b[:grid.N_int] = rhs_int
    if jump is not None:
        iface = grid.interface_indices()
        b[iface] = np.asarray(jump)[iface]
    if f_bd is not None:
        b[grid.boundary_indices()] = f_bd
    return b


def solve(grid: Grid, coef, gamma_dt, rhs_int, f_bd=None, jump=None):
    """Brute-force solve of eq. ``sparse_A`` (numpy.linalg.solve on the dense matrix)."""
    A = assemble(grid, coef, gamma_dt)
    return np.linalg.solve(A, rhs_vector(grid, rhs_int, f_bd, jump))


def residual(grid: Grid, coef, gamma_dt, u, rhs_int, f_bd=None, jump=None):
    """A u - b for the dense system (tiny N only)."""
    A = assemble(grid, coef, gamma_dt)
    return A @ u - rhs_vector(grid, rhs_int, f_bd, jump)
