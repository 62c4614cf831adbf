"""Pins for oracle/cheb.py: nodes and differentiation matrix (Sec. 2.1, Sec. 4.1)."""
import numpy as np
import pytest

from oracle import cheb


@pytest.mark.parametrize("p", [3, 4, 5, 8, 12, 16, 21])
def test_nodes_are_the_cosine_points(p):
    x = cheb.nodes(p)
    ref = np.sort(np.cos(np.arange(p) * np.pi / (p - 1)))  # Sec. 4.1: x_j = cos(j pi/(p-1))
    assert np.allclose(x, ref, atol=1e-15, rtol=0)
    assert x[0] == -1.0 and x[-1] == 1.0
    assert np.all(np.diff(x) > 0)


@pytest.mark.parametrize("p", [3, 4, 6, 8, 12, 16, 21])
def test_diff_matrix_exact_on_polynomials(p):
    """d/dx of every monomial of degree <= p-1 on an interval of length h is exact to roundoff."""
    h = 0.37
    D = cheb.diff_matrix(p, h)
    t = 0.5 * h * (1.0 + cheb.nodes(p))  # points of [0, h]
    for k in range(p):
        v = t ** k
        dv = k * t ** (k - 1) if k > 0 else np.zeros(p)
        scale = max(1.0, np.abs(dv).max())
        assert np.abs(D @ v - dv).max() <= 1e-11 * scale * p ** 2
    # constants are annihilated
    assert np.abs(D @ np.ones(p)).max() < 1e-10 * p ** 2 / h


@pytest.mark.parametrize("p", [4, 8, 16, 21])
def test_diff_matrix_corner_closed_form(p):
    """Textbook Chebyshev value at the right end point: D[N, N] = (2 N^2 + 1) / 6, N = p - 1
    (on [-1, 1]); independent of the barycentric construction."""
    n = p - 1
    D = cheb.lagrange_diff_matrix(cheb.nodes(p))
    assert abs(D[-1, -1] - (2 * n * n + 1) / 6.0) < 1e-10 * n * n
    assert abs(D[0, 0] + (2 * n * n + 1) / 6.0) < 1e-10 * n * n


def test_diff_matrix_not_exact_beyond_degree():
    """Degree p is not reproduced: the check above is discriminating."""
    p = 6
    D = cheb.diff_matrix(p, 2.0)
    x = cheb.nodes(p)
    assert np.abs(D @ x ** p - p * x ** (p - 1)).max() > 1e-3
