"""Global collocation points of Sec. 2.1 and their ordering.

The rectangle [x0, x1] x [y0, y1] is cut into n1 x n2 equal leaves (Sec. 2.1, Fig. 1).
Each leaf carries p x p Chebyshev nodes; the four corner nodes of every leaf are dropped
(Sec. 2.1: they feed no derivative when there is no mixed term), and edge nodes shared
by two leaves are one unknown.  That leaves N = (p-2)(p n1 n2 + n1 + n2) points.

Global ordering (the library's documented convention; m = p - 2):

1. leaf interiors: leaf l = iy*n1 + ix, node (i, j) with i, j in 1..m (i along x),
   index l*m*m + (j-1)*m + (i-1);
2. vertical edge segments: line L = 0..n1 (x = x0 + L*hx), leaf row iy, node j in 1..m,
   index N_int + (L*n2 + iy)*m + (j-1);
3. horizontal edge segments: line L = 0..n2, leaf column ix, node i in 1..m,
   index N_int + N_v + (L*n1 + ix)*m + (i-1).

A leaf's local node (i, j), 0 <= i, j < p, sits at
x = x0 + hx*(ix + (1 + xi_i)/2), y = y0 + hy*(iy + (1 + xi_j)/2).

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from . import cheb


class Grid:
    """Index bookkeeping for an n1 x n2 leaf grid with p Chebyshev nodes per side."""

    def __init__(self, n1, n2, p, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
        if p < 3:
            raise ValueError("p must be >= 3 so that leaves have interior nodes")
        self.n1, self.n2, self.p = int(n1), int(n2), int(p)
        self.m = self.p - 2
        self.x0, self.x1, self.y0, self.y1 = float(x0), float(x1), float(y0), float(y1)
        self.hx = (self.x1 - self.x0) / self.n1
        self.hy = (self.y1 - self.y0) / self.n2
        m = self.m
        self.N_int = self.n1 * self.n2 * m * m
        self.N_v = (self.n1 + 1) * self.n2 * m
        self.N_h = (self.n2 + 1) * self.n1 * m
        self.N = self.N_int + self.N_v + self.N_h
        assert self.N == m * (self.p * self.n1 * self.n2 + self.n1 + self.n2)  # Sec. 2.1 count
        self.xi = cheb.nodes(self.p)

    # --- global index helpers -------------------------------------------------------
    def vseg(self, line, iy, j):
        """Global index of node j (1..m) of the vertical segment on x-line `line`, leaf row iy."""
        return self.N_int + (line * self.n2 + iy) * self.m + (j - 1)

    def hseg(self, line, ix, i):
        """Global index of node i (1..m) of the horizontal segment on y-line `line`, leaf column ix."""
        return self.N_int + self.N_v + (line * self.n1 + ix) * self.m + (i - 1)

    def leaf_id(self, ix, iy):
        return iy * self.n1 + ix

    def local_to_global(self, ix, iy):
        """Array g[j, i] (p x p) with the global index of leaf-local node (i, j); -1 at corners."""
        p, m = self.p, self.m
        g = -np.ones((p, p), dtype=np.int64)
        base = self.leaf_id(ix, iy) * m * m
        for j in range(p):
            for i in range(p):
                if (i in (0, p - 1)) and (j in (0, p - 1)):
                    continue
                if 1 <= i <= m and 1 <= j <= m:
                    g[j, i] = base + (j - 1) * m + (i - 1)
                elif i == 0:
                    g[j, i] = self.vseg(ix, iy, j)
                elif i == p - 1:
                    g[j, i] = self.vseg(ix + 1, iy, j)
                elif j == 0:
                    g[j, i] = self.hseg(iy, ix, i)
                else:
                    g[j, i] = self.hseg(iy + 1, ix, i)
        return g

    def coords(self):
        """x, y coordinates (length N) of every global point."""
        X = np.full(self.N, np.nan)
        Y = np.full(self.N, np.nan)
        for iy in range(self.n2):
            for ix in range(self.n1):
                g = self.local_to_global(ix, iy)
                xs = self.x0 + self.hx * (ix + 0.5 * (1.0 + self.xi))
                ys = self.y0 + self.hy * (iy + 0.5 * (1.0 + self.xi))
                for j in range(self.p):
                    for i in range(self.p):
                        if g[j, i] >= 0:
                            X[g[j, i]] = xs[i]
                            Y[g[j, i]] = ys[j]
        assert not np.isnan(X).any()
        return X, Y

    def boundary_indices(self):
        """Global indices of the points on the outer boundary, ascending."""
        idx = []
        for line in (0, self.n1):
            for iy in range(self.n2):
                idx.extend(self.vseg(line, iy, j) for j in range(1, self.m + 1))
        for line in (0, self.n2):
            for ix in range(self.n1):
                idx.extend(self.hseg(line, ix, i) for i in range(1, self.m + 1))
        return np.array(sorted(idx), dtype=np.int64)

    def interface_indices(self):
        """Global indices of edge points shared by two leaves (not on the outer boundary), ascending."""
        bd = set(self.boundary_indices().tolist())
        all_edges = range(self.N_int, self.N)
        return np.array([k for k in all_edges if k not in bd], dtype=np.int64)

    def interior_indices(self):
        return np.arange(self.N_int, dtype=np.int64)

    def box_boundary(self, ix0, iy0, a, c):
        """Global indices of the boundary points of the box of a x c leaves at leaf (ix0, iy0),
        in the order south (ascending x), east (ascending y), north (ascending x), west (ascending y)."""
        m = self.m
        out = []
        for s in range(a):
            out.extend(self.hseg(iy0, ix0 + s, i) for i in range(1, m + 1))
        for s in range(c):
            out.extend(self.vseg(ix0 + a, iy0 + s, j) for j in range(1, m + 1))
        for s in range(a):
            out.extend(self.hseg(iy0 + c, ix0 + s, i) for i in range(1, m + 1))
        for s in range(c):
            out.extend(self.vseg(ix0, iy0 + s, j) for j in range(1, m + 1))
        return np.array(out, dtype=np.int64)
