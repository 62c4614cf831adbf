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
        # leaves (eq. ``leaf``)
        for lev in self.levels:
            for nd in lev:
                if nd.is_leaf:
                    ops = LeafOps(grid.p, grid.hx, grid.hy, slices[(nd.ix0, nd.iy0)], gamma_dt)
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
        src = []  # parent boundary point -> (child, position in that child)
        for g in nd.bd:
            if g in pos_a:
                src.append((0, pos_a[g]))
            else:
                src.append((1, pos_b[g]))
        nb, n3 = len(nd.bd), len(J3)
        M = al.T[np.ix_(ia3, ia3)] - be.T[np.ix_(ib3, ib3)]
        Bm = np.empty((n3, nb))
        Tcat = np.empty((nb, n3))
        Tdiag = np.zeros((nb, nb))
        for k, (ch, pk) in enumerate(src):
            if ch == 0:
                Bm[:, k] = -al.T[ia3, pk]
                Tcat[k, :] = al.T[pk, ia3]
            else:
                Bm[:, k] = be.T[ib3, pk]
                Tcat[k, :] = be.T[pk, ib3]
            for k2, (ch2, pk2) in enumerate(src):
                if ch2 == ch:
                    Tdiag[k, k2] = (al.T if ch == 0 else be.T)[pk, pk2]
        X = np.linalg.inv(M)
        S = X @ Bm
        nd.J3 = np.array(J3, dtype=np.int64)
        nd.ia3, nd.ib3, nd.src = ia3, ib3, src
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
                    hc = np.array([h[id(al) if ch == 0 else id(be)][pk] for ch, pk in nd.src])
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
