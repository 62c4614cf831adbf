"""Leaf collocation operators, eq. ``discretize`` and eq. ``leaf`` of Sec. 2.1.

On one leaf square the operator L u = a11 u_xx + a22 u_yy + a1 u_x + a2 u_y + a0 u
(the elliptic operator of eq. ``operatorA`` with c12 = 0, written with the sign of
u_t = L u) is collocated at the (p-2)^2 interior Chebyshev nodes.  The implicit stage
operator is A = I - gamma*dt*L.  With interior set J_i and edge set J_b (corners dropped):

  S = -A_ii^{-1} A_ib                      (solution operator, eq. ``leaf``)
  T = D S restricted to the edges          (DtN map, eq. ``leaf``), i.e. T = D_bi S + D_bb

where the flux at an edge node is d/dx on a vertical edge and d/dy on a horizontal edge
(Sec. 2.1, the fixed coordinate derivative rather than the outward normal).

Local node (i, j) (i along x) has flat index j*p + i.  Interior order: j-major, i fastest.
Edge order: south (i=1..m, j=0), east (i=p-1, j=1..m), north (i=1..m, j=p-1), west (i=0, j=1..m).

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from . import cheb

COEF_NAMES = ("a11", "a22", "a1", "a2", "a0")


def local_sets(p):
    """(interior flat indices, edge flat indices, edge orientation 'x'/'y') for a p x p leaf."""
    m = p - 2
    I = [j * p + i for j in range(1, m + 1) for i in range(1, m + 1)]
    S = [0 * p + i for i in range(1, m + 1)]
    E = [j * p + (p - 1) for j in range(1, m + 1)]
    N = [(p - 1) * p + i for i in range(1, m + 1)]
    W = [j * p + 0 for j in range(1, m + 1)]
    B = S + E + N + W
    orient = ["y"] * m + ["x"] * m + ["y"] * m + ["x"] * m
    return np.array(I), np.array(B), orient


def full_derivatives(p, hx, hy):
    """Dx, Dy acting on the full p*p local grid (flat index j*p + i)."""
    D1x = cheb.diff_matrix(p, hx)
    D1y = cheb.diff_matrix(p, hy)
    Ip = np.eye(p)
    Dx = np.kron(Ip, D1x)
    Dy = np.kron(D1y, Ip)
    return Dx, Dy


def _coef_vector(c, q):
    c = np.asarray(c, dtype=np.float64)
    if c.ndim == 0:
        return np.full(q, float(c))
    assert c.shape == (q,)
    return c


def collocation_L_rows(p, hx, hy, coef):
    """Rows of L at the interior nodes, as a q x p^2 matrix over the full local grid.

    coef: dict with a11, a22, a1, a2, a0, each a scalar or a length-q array in interior order.
    """
    I, _, _ = local_sets(p)
    q = I.size
    Dx, Dy = full_derivatives(p, hx, hy)
    Dxx = Dx @ Dx
    Dyy = Dy @ Dy
    c = {k: _coef_vector(coef[k], q) for k in COEF_NAMES}
    Id = np.eye(p * p)
    L = (c["a11"][:, None] * Dxx[I] + c["a22"][:, None] * Dyy[I]
         + c["a1"][:, None] * Dx[I] + c["a2"][:, None] * Dy[I] + c["a0"][:, None] * Id[I])
    return L


def flux_rows(p, hx, hy):
    """Rows of the edge-flux operator over the full local grid (b x p^2)."""
    _, B, orient = local_sets(p)
    Dx, Dy = full_derivatives(p, hx, hy)
    rows = np.array([Dx[k] if o == "x" else Dy[k] for k, o in zip(B, orient)])
    return rows


class LeafOps:
    """Everything the HPS build and solve need from one leaf (eq. ``discretize``, eq. ``leaf``)."""

    def __init__(self, p, hx, hy, coef, gamma_dt):
        I, B, _ = local_sets(p)
        self.p, self.I, self.B = p, I, B
        L = collocation_L_rows(p, hx, hy, coef)
        A_rows = np.eye(p * p)[I] - gamma_dt * L          # A = I - gamma dt L at interior rows
        corners = [0, p - 1, (p - 1) * p, p * p - 1]
        assert np.all(A_rows[:, corners] == 0.0), "interior rows must not touch corners (Sec. 2.1)"
        self.A_ii = A_rows[:, I]
        self.A_ib = A_rows[:, B]
        Dflux = flux_rows(p, hx, hy)
        assert np.all(Dflux[:, corners] == 0.0), "edge fluxes must not touch corners (Sec. 2.1)"
        self.D_bi = Dflux[:, I]
        self.D_bb = Dflux[:, B]
        # eq. ``leaf``: S = -A_ii^{-1} A_ib ; T = D S (+ the edge-to-edge part of D)
        self.S = -np.linalg.solve(self.A_ii, self.A_ib)
        self.T = self.D_bi @ self.S + self.D_bb

    def particular(self, rhs):
        """Particular solution w (zero on the edges) of A_ii w = rhs and its edge fluxes h = D_bi w."""
        w = np.linalg.solve(self.A_ii, rhs)
        return w, self.D_bi @ w
