"""Host-side factorization of the constant-coefficient leaf operator by fast diagonalization
(the leaf interior operator is a Kronecker sum of 1-D Chebyshev operators, Sec. 4.2):
A_ii^-1 = (V_y (x) V_x) Lam (V_y^-1 (x) V_x^-1).  hps_fastdiag_check multiplies the factored
inverse by A_ii for every unit vector; no GPU is used."""
import ctypes

import pytest


def _check(p, coef, gdt, hx, hy):
    from paper_2306_02526_gb300 import _lib
    c = (ctypes.c_double * 5)(*coef)
    err = ctypes.c_double(-1.0)
    rc = _lib.lib().hps_fastdiag_check(p, c, gdt, hx, hy, ctypes.byref(err))
    return rc, err.value


@pytest.mark.parametrize("p", [4, 6, 8, 12, 16, 20, 24, 32])
def test_heat_operator_factors(p):
    rc, err = _check(p, (1.0, 1.0, 0.0, 0.0, 0.0), 0.0025, 0.25, 0.25)
    assert rc == 0 and err <= 1e-12


@pytest.mark.parametrize("coef,gdt,hx,hy", [
    ((0.01, 0.01, 0.0, 0.0, 0.0), 2.5e-4, 1 / 64, 1 / 64),      # the Allen-Cahn bench operator
    ((1.0, 0.7, 0.3, 0.0, -0.5), 0.013, 0.125, 0.25),           # anisotropic leaves, first derivative, reaction
    ((1.0, 1.0, 0.5, -0.25, -1.0), 2.5e-4, 1 / 128, 1 / 128),   # cfg3-like constants
])
def test_general_constant_operators_factor(coef, gdt, hx, hy):
    rc, err = _check(16, coef, gdt, hx, hy)
    assert rc == 0 and err <= 1e-12


@pytest.mark.parametrize("coef", [(0.001, 0.001, 100.0, 0.0, 0.0), (0.0, 0.0, 1.0, 0.0, 0.0)])
def test_no_real_decomposition_is_refused(coef):
    """Convection-dominated 1-D operators have complex eigenvalues, a zero operator a repeated
    one: the build falls back to the assembled inverse."""
    rc, _ = _check(16, coef, 0.01, 0.25, 0.25)
    assert rc == -1
