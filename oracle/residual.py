"""Leaf-local evaluation of the rows of eq. ``sparse_A`` (Sec. 2.1) for any grid size.

Computes A u - b row type by row type without forming A: the collocated PDE rows at
leaf-interior points, the flux-jump rows at shared edges and the Dirichlet rows on the
outer boundary.  Because every row only couples the points of one or two leaves, this is
O(N p) and serves as a size-independent property check (a solution of the system has a
residual at roundoff level) where a dense solve is out of reach.

Also provides ``apply_L_interior``: L u at the interior points by leaf-local Chebyshev
differentiation, used by the time stepper for L u^n and by the nonlinear terms.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from . import cheb
from .grid import Grid


def leaf_gather_index(grid: Grid):
    """(n_leaves, p, p) global indices of every leaf's local nodes (corners -> N, a zero slot).
    Leaves are numbered l = iy*n1 + ix."""
    idx = np.empty((grid.n1 * grid.n2, grid.p, grid.p), dtype=np.int64)
    for iy in range(grid.n2):
        for ix in range(grid.n1):
            g = grid.local_to_global(ix, iy)
            g = np.where(g < 0, grid.N, g)
            idx[grid.leaf_id(ix, iy)] = g
    return idx


class LeafField:
    """Local fields U[l, j, i] of a global vector and their Chebyshev derivatives."""

    def __init__(self, grid: Grid, u, idx=None):
        self.grid = grid
        self.idx = leaf_gather_index(grid) if idx is None else idx
        ext = np.concatenate([np.asarray(u, dtype=np.float64), [0.0]])
        self.U = ext[self.idx]
        D1x = cheb.diff_matrix(grid.p, grid.hx)
        D1y = cheb.diff_matrix(grid.p, grid.hy)
        self.Ux = np.einsum("lji,ki->ljk", self.U, D1x)        # d/dx along i
        self.Uy = np.einsum("lji,kj->lki", self.U, D1y)        # d/dy along j
        self.Uxx = np.einsum("lji,ki->ljk", self.Ux, D1x)
        self.Uyy = np.einsum("lji,kj->lki", self.Uy, D1y)

    def interior(self, arr):
        """Interior block of a (n_leaves, p, p) array, flattened to global interior order."""
        return arr[:, 1:-1, 1:-1].reshape(-1)


def _coef(coef, k, n):
    v = np.asarray(coef.get(k, 0.0), dtype=np.float64)
    return np.full(n, float(v)) if v.ndim == 0 else v


def apply_L_interior(grid: Grid, coef, u, field=None):
    """(L u) at interior points, L = a11 d_xx + a22 d_yy + a1 d_x + a2 d_y + a0."""
    F = LeafField(grid, u) if field is None else field
    n = grid.N_int
    return (_coef(coef, "a11", n) * F.interior(F.Uxx) + _coef(coef, "a22", n) * F.interior(F.Uyy)
            + _coef(coef, "a1", n) * F.interior(F.Ux) + _coef(coef, "a2", n) * F.interior(F.Uy)
            + _coef(coef, "a0", n) * F.interior(F.U))


def flux_jumps(grid: Grid, u, field=None):
    """Length-N array: at every shared edge point, (flux from west/south leaf) - (flux from
    east/north leaf); zero elsewhere."""
    F = LeafField(grid, u) if field is None else field
    out = np.zeros(grid.N)
    p, n1, n2 = grid.p, grid.n1, grid.n2
    for L in range(1, n1):
        for iy in range(n2):
            west = grid.leaf_id(L - 1, iy)
            east = grid.leaf_id(L, iy)
            g = [grid.vseg(L, iy, j) for j in range(1, p - 1)]
            out[g] = F.Ux[west, 1:-1, p - 1] - F.Ux[east, 1:-1, 0]
    for L in range(1, n2):
        for ix in range(n1):
            south = grid.leaf_id(ix, L - 1)
            north = grid.leaf_id(ix, L)
            g = [grid.hseg(L, ix, i) for i in range(1, p - 1)]
            out[g] = F.Uy[south, p - 1, 1:-1] - F.Uy[north, 0, 1:-1]
    return out


def residual(grid: Grid, coef, gamma_dt, u, rhs_int, f_bd=None, jump=None):
    """A u - b for eq. ``sparse_A`` with A = I - gamma_dt L, evaluated leaf by leaf."""
    u = np.asarray(u, dtype=np.float64)
    F = LeafField(grid, u)
    r = np.zeros(grid.N)
    r[:grid.N_int] = F.interior(F.U) - gamma_dt * apply_L_interior(grid, coef, u, F) - rhs_int
    jumps = flux_jumps(grid, u, F)
    iface = grid.interface_indices()
    r[iface] = jumps[iface] - (0.0 if jump is None else np.asarray(jump)[iface])
    bd = grid.boundary_indices()
    r[bd] = u[bd] - (0.0 if f_bd is None else f_bd)
    return r
