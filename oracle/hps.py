"""Hierarchical Poincare-Steklov (HPS) build and solve, Sec. 2.1.

Tree (Sec. 2.1, Fig. 1: the domain is "halved" repeatedly): a box of a x c leaves is cut
across its longer side (counted in leaves); on a tie the cut is a vertical line (x split).
The west/south half is child alpha, the east/north half child beta.  The paper does not
fix the cut order; this is the reading used throughout.

Build (Sec. 2.1 merge formulas, eq. ``local_operators_children`` / ``local_operators_parent``):
with J1 = alpha-only boundary, J2 = beta-only boundary, J3 = shared interface,

  X   = (T^a_33 - T^b_33)^{-1}
  S^t = X [ -T^a_31 | T^b_32 ]
  T^t = diag(T^a_11, T^b_22) + [T^a_13 ; T^b_23] S^t.

(The beta block equation is printed with alpha superscripts in the paper; it is read
here with beta's blocks, the only reading under which the merge is consistent.)

Solve (Alg. 1 plus the body-load terms the paper defers to Martinsson 2019, ch. 25).
On a leaf u = w + phi with A_ii w = rhs, w = 0 on the edges, phi_i = S u_b, so the edge
flux is v = T u_b + h with h = D_bi w.  Flux continuity on J3, v^a_3 - v^b_3 = jump,
gives
  (T^a_33 - T^b_33) u3 = -T^a_31 u1 + T^b_32 u2 + (h^b_3 - h^a_3 + jump)
hence u3 = S^t [u1; u2] + w3 with w3 = X (h^b_3 - h^a_3 + jump), and the parent's flux
v = T^t [u1; u2] + h^t with h^t = [h^a_1 + T^a_13 w3 ; h^b_2 + T^b_23 w3].
The upward sweep carries w3 and h^t from the leaves to the root; the downward sweep sets
u = f on the outer boundary and applies u3 = S^t u_b + w3 from the root to the leaves,
then u_i = w + S u_b on every leaf.  ``jump`` is zero for the PDE itself; a nonzero jump
is the right-hand side of the interface rows of eq. ``sparse_A``.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from .grid import Grid
from .leaf import LeafOps, COEF_NAMES


class Node:
    def __init__(self, ix0, iy0, a, c, level):
        self.ix0, self.iy0, self.a, self.c, self.level = ix0, iy0, a, c, level
        self.children = None
        self.split = None

    @property
    def is_leaf(self):
        return self.children is None


def build_tree(n1, n2):
    """Binary tree of boxes; returns (root, levels) with levels[l] the nodes of depth l in order."""
    root = Node(0, 0, n1, n2, 0)
    levels = []
    stack = [root]
    while stack:
        nxt = []
        levels.append(stack)
        for nd in stack:
            if nd.a == 1 and nd.c == 1:
                continue
            if nd.a >= nd.c:  # cut across x (vertical interface); ties go to x
                a1 = nd.a // 2
                alpha = Node(nd.ix0, nd.iy0, a1, nd.c, nd.level + 1)
                beta = Node(nd.ix0 + a1, nd.iy0, nd.a - a1, nd.c, nd.level + 1)
                nd.split = "x"
            else:
                c1 = nd.c // 2
                alpha = Node(nd.ix0, nd.iy0, nd.a, c1, nd.level + 1)
                beta = Node(nd.ix0, nd.iy0 + c1, nd.a, nd.c - c1, nd.level + 1)
                nd.split = "y"
            nd.children = (alpha, beta)
            nxt.extend([alpha, beta])
        stack = nxt
    return root, levels


def coefficient_slices(grid, coef):
    """Per-leaf coefficient dicts from global-interior-order arrays (or scalars)."""
    q = grid.m * grid.m
    out = {}
    for iy in range(grid.n2):
        for ix in range(grid.n1):
            l = grid.leaf_id(ix, iy)
            d = {}
            for k in COEF_NAMES:
                v = np.asarray(coef.get(k, 0.0), dtype=np.float64)
                d[k] = v if v.ndim == 0 else v[l * q:(l + 1) * q]
            out[(ix, iy)] = d
    return out


class HPS:
    """Operators of (I - gamma_dt L) on an n1 x n2 leaf grid, built by Sec. 2.1."""

    def __init__(self, grid: Grid, coef, gamma_dt):
        self.grid = grid
        self.gamma_dt = float(gamma_dt)
        self.root, self.levels = build_tree(grid.n1, grid.n2)
        slices = coefficient_slices(grid, coef)
        # every node: its boundary points in box order (south, east, north, west)
        for lev in self.levels:
            for nd in lev:
                nd.bd = grid.box_boundary(nd.ix0, nd.iy0, nd.a, nd.c)
        # leaves (eq. ``leaf``); with scalar coefficients every leaf has the same operators,
        # so they are formed once and shared
        scalar = all(np.ndim(coef.get(k, 0.0)) == 0 for k in COEF_NAMES)
        shared_ops = None
        for lev in self.levels:
            for nd in lev:
                if nd.is_leaf:
                    if scalar and shared_ops is not None:
                        ops = shared_ops
                    else:
                        ops = LeafOps(grid.p, grid.hx, grid.hy, slices[(nd.ix0, nd.iy0)], gamma_dt)
                        shared_ops = ops if scalar else None
                    g = grid.local_to_global(nd.ix0, nd.iy0).reshape(-1)
                    assert np.array_equal(g[ops.B], nd.bd), "leaf edge order must match box order"
                    nd.ops = ops
                    nd.interior = g[ops.I]
                    nd.T = ops.T
        # merges, bottom-up (Sec. 2.1 merge formulas)
        for lev in reversed(self.levels):
            for nd in lev:
                if not nd.is_leaf:
                    self._merge(nd)

    def _merge(self, nd):
        al, be = nd.children
        pos_a = {g: k for k, g in enumerate(al.bd)}
        pos_b = {g: k for k, g in enumerate(be.bd)}
        J3 = [g for g in al.bd if g in pos_b]
        J3_b = [g for g in be.bd if g in pos_a]
        assert J3 == J3_b, "both children list the interface in the same order"
        ia3 = np.array([pos_a[g] for g in J3])
        ib3 = np.array([pos_b[g] for g in J3])
        # parent boundary point -> (child, position in that child); J1 from alpha, J2 from beta
        src_child = np.array([0 if g in pos_a else 1 for g in nd.bd])
        src_pos = np.array([pos_a[g] if g in pos_a else pos_b[g] for g in nd.bd])
        A1 = np.nonzero(src_child == 0)[0]   # parent positions of J1
        B2 = np.nonzero(src_child == 1)[0]   # parent positions of J2
        pa1, pb2 = src_pos[A1], src_pos[B2]
        nb, n3 = len(nd.bd), len(J3)
        M = al.T[np.ix_(ia3, ia3)] - be.T[np.ix_(ib3, ib3)]          # T^a_33 - T^b_33
        Bm = np.empty((n3, nb))                                      # [-T^a_31 | T^b_32]
        Bm[:, A1] = -al.T[np.ix_(ia3, pa1)]
        Bm[:, B2] = be.T[np.ix_(ib3, pb2)]
        Tcat = np.empty((nb, n3))                                    # [T^a_13 ; T^b_23]
        Tcat[A1, :] = al.T[np.ix_(pa1, ia3)]
        Tcat[B2, :] = be.T[np.ix_(pb2, ib3)]
        Tdiag = np.zeros((nb, nb))                                   # diag(T^a_11, T^b_22)
        Tdiag[np.ix_(A1, A1)] = al.T[np.ix_(pa1, pa1)]
        Tdiag[np.ix_(B2, B2)] = be.T[np.ix_(pb2, pb2)]
        X = np.linalg.inv(M)
        S = X @ Bm
        nd.J3 = np.array(J3, dtype=np.int64)
        nd.ia3, nd.ib3 = ia3, ib3
        nd.A1, nd.B2, nd.pa1, nd.pb2 = A1, B2, pa1, pb2
        nd.X, nd.S, nd.Tcat = X, S, Tcat
        nd.T = Tdiag + Tcat @ S

    # ------------------------------------------------------------------------------
    def solve(self, rhs_int, f_bd=None, jump=None):
        """Solve A u = [rhs on interior rows; jump on interface rows; f on boundary rows].

        rhs_int: length N_int (global interior order); f_bd: values at
        grid.boundary_indices() (None = 0); jump: length-N array read at interface points
        (None = 0).  Returns the length-N solution.
        """
        grid = self.grid
        rhs_int = np.asarray(rhs_int, dtype=np.float64)
        u = np.zeros(grid.N)
        w_leaf, h = {}, {}
        # upward sweep: leaves, then merges from the bottom level to the root
        for lev in reversed(self.levels):
            for nd in lev:
                if nd.is_leaf:
                    w, hh = nd.ops.particular(rhs_int[nd.interior])
                    w_leaf[id(nd)], h[id(nd)] = w, hh
                else:
                    al, be = nd.children
                    d = h[id(be)][nd.ib3] - h[id(al)][nd.ia3]
                    if jump is not None:
                        d = d + np.asarray(jump)[nd.J3]
                    nd.w3 = nd.X @ d
                    hc = np.empty(len(nd.bd))
                    hc[nd.A1] = h[id(al)][nd.pa1]
                    hc[nd.B2] = h[id(be)][nd.pb2]
                    h[id(nd)] = hc + nd.Tcat @ nd.w3
        # downward sweep (Alg. 1 with the particular parts added)
        if f_bd is not None:
            u[grid.boundary_indices()] = f_bd
        for lev in self.levels:
            for nd in lev:
                if nd.is_leaf:
                    u[nd.interior] = w_leaf[id(nd)] + nd.ops.S @ u[nd.bd]
                else:
                    u[nd.J3] = nd.S @ u[nd.bd] + nd.w3
        return u
