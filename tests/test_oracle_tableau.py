"""Pins for oracle/tableau.py (Sec. 3.1, Table ``tbl:butcher``): structure, the order
conditions of additive Runge-Kutta methods up to order 4 in exact arithmetic, L-stability."""
import copy
from fractions import Fraction as F
from functools import lru_cache

import numpy as np

from oracle import tableau as tb

S = tb.S


@lru_cache(None)
def _trees(n):
    """All bi-coloured rooted trees with n vertices: (colour, sorted tuple of child trees)."""
    out = []
    for col in (0, 1):
        for kids in _forests(n - 1):
            out.append((col, kids))
    return tuple(out)


@lru_cache(None)
def _forests(n):
    if n == 0:
        return ((),)
    res = set()
    for k in range(1, n + 1):
        for t in _trees(k):
            for f in _forests(n - k):
                res.add(tuple(sorted((t,) + f)))
    return tuple(sorted(res))


def _density(t):
    r = 1 + sum(_order(k) for k in t[1])
    for k in t[1]:
        r *= _density(k)
    return r


def _order(t):
    return 1 + sum(_order(k) for k in t[1])


def order_residuals(A, Ah, b, bh, max_order):
    """For every bi-coloured tree t up to max_order: sum_i b^{col(root)}_i Phi_i(t) - 1/gamma(t),
    where a child of colour 0 (implicit part) enters through A and colour 1 through A-hat."""
    def phi(t, i):
        r = F(1)
        for k in t[1]:
            M = A if k[0] == 0 else Ah
            r *= sum(M[i][j] * phi(k, j) for j in range(S))
        return r

    out = []
    for n in range(1, max_order + 1):
        for t in _trees(n):
            w = b if t[0] == 0 else bh
            out.append(sum(w[i] * phi(t, i) for i in range(S)) - F(1, _density(t)))
    return out


def test_structure():
    A, Ah, c, b = tb.A_IMPL, tb.A_EXPL, tb.C, tb.B
    assert all(A[0][j] == 0 for j in range(S))                     # explicit first stage
    assert all(A[i][i] == tb.GAMMA for i in range(1, S))            # singly diagonal
    assert all(A[i][j] == 0 for i in range(S) for j in range(i + 1, S))
    assert all(A[S - 1][j] == b[j] for j in range(S))               # stiffly accurate
    assert all(Ah[i][j] == 0 for i in range(S) for j in range(i, S))  # explicit
    assert tb.B_HAT == b and c[0] == 0 and c[-1] == 1
    for i in range(S):
        assert sum(A[i]) == c[i]                                    # row sums = c, exactly
        assert abs(float(sum(Ah[i]) - c[i])) < 1e-24                # shared c (Sec. 3.1)


def test_order_conditions_up_to_four():
    res = order_residuals(tb.A_IMPL, tb.A_EXPL, tb.B, tb.B_HAT, 4)
    assert len(res) == 72
    assert max(abs(float(r)) for r in res) < 1e-24


def test_not_order_five():
    res = order_residuals(tb.A_IMPL, tb.A_EXPL, tb.B, tb.B_HAT, 5)
    assert max(abs(float(r)) for r in res[72:]) > 1e-4


def test_planted_coefficient_error_is_caught():
    A = copy.deepcopy(tb.A_IMPL)
    A[3][1] = -A[3][1]
    res = order_residuals(A, tb.A_EXPL, tb.B, tb.B_HAT, 4)
    assert max(abs(float(r)) for r in res) > 1e-3
    Ah = copy.deepcopy(tb.A_EXPL)
    Ah[4][2] = Ah[4][2] * F(101, 100)
    res = order_residuals(tb.A_IMPL, Ah, tb.B, tb.B_HAT, 4)
    assert max(abs(float(r)) for r in res) > 1e-4


def _stability(z):
    A, b, _, _, _ = tb.as_float()
    e = np.ones(S)
    return 1.0 + z * b @ np.linalg.solve(np.eye(S) - z * A, e)


def test_l_stability():
    """R(z) = 1 + z b^T (I - zA)^{-1} 1 of the implicit table: |R| <= 1 on the left half
    plane and R(z) -> 0 as z -> -infinity."""
    assert abs(_stability(-1e8)) < 1e-6
    for y in np.linspace(0.0, 200.0, 401):
        assert abs(_stability(1j * y)) <= 1.0 + 1e-12
    rng = np.random.default_rng(0)
    for z in -rng.exponential(10, 200) + 1j * rng.normal(0, 30, 200):
        assert abs(_stability(z)) <= 1.0 + 1e-12
