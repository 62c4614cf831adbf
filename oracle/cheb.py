"""Chebyshev-Lobatto nodes and the collocation differentiation matrix.

Sec. 2.1 discretizes every leaf square with p x p Chebyshev nodes; Sec. 4.1 names the
1D nodes x_j = cos(j*pi/(p-1)).  The oracle keeps the same point set in ascending order.

The differentiation matrix is written from its plain definition: entry (i, j) is the
derivative at x_i of the j-th Lagrange basis polynomial through all nodes.  It is
formed from barycentric weights, which holds for any distinct nodes; nothing
Chebyshev-specific is used, so a mistake in a closed-form Chebyshev formula elsewhere
cannot be shared with this one.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np


def nodes(p):
    """Chebyshev-Lobatto points on [-1, 1] in ascending order (Sec. 4.1 node formula,
    reversed so that index 0 is the left end)."""
    if p < 2:
        raise ValueError("p must be >= 2")
    j = np.arange(p, dtype=np.float64)
    return -np.cos(j * np.pi / (p - 1))


def lagrange_diff_matrix(x):
    """D[i, j] = l_j'(x_i) for the Lagrange basis {l_j} through the distinct nodes x.

    With barycentric weights w_j = 1 / prod_{k != j} (x_j - x_k):
      l_j'(x_i) = (w_j / w_i) / (x_i - x_j)          for i != j,
      l_i'(x_i) = sum_{k != i} 1 / (x_i - x_k).
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    w = np.empty(n)
    for j in range(n):
        diff = x[j] - np.delete(x, j)
        w[j] = 1.0 / np.prod(diff)
    D = np.empty((n, n))
    for i in range(n):
        s = 0.0
        for j in range(n):
            if i == j:
                continue
            D[i, j] = (w[j] / w[i]) / (x[i] - x[j])
            s += 1.0 / (x[i] - x[j])
        D[i, i] = s
    return D


def diff_matrix(p, length):
    """Differentiation matrix for p Chebyshev nodes mapped affinely onto an interval of
    the given length (d/dx = (2/length) d/dxi)."""
    return (2.0 / length) * lagrange_diff_matrix(nodes(p))
