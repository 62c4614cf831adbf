"""Butcher tables of the additive Runge-Kutta pair ARK4(3)6L[2]SA (Kennedy & Carpenter 2003),
the pair the paper uses throughout (Sec. 3.1, Table ``tbl:butcher``).

The paper names the pair but does not print its coefficients.  They are written here as
exact rationals.  Structure (Table ``tbl:butcher``): the implicit table is ESDIRK (zero first
row, a_ii = gamma = 1/4 for i >= 2, last row = b, so the method is stiffly accurate); the
explicit table is strictly lower triangular; both share the abscissae c (Sec. 3.1 assumes
c_j = c-hat_j) and b-hat = b.  The coefficient values are pinned by the order conditions of
additive RK methods up to order 4 (bi-coloured rooted trees) and by L-stability, checked
in exact arithmetic in ``tests/test_oracle_tableau.py``.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from fractions import Fraction as F

import numpy as np

S = 6
GAMMA = F(1, 4)

C = [F(0), F(1, 2), F(83, 250), F(31, 50), F(17, 20), F(1)]

B = [F(82889, 524892), F(0), F(15625, 83664), F(69875, 102672), F(-2260, 8211), F(1, 4)]


def _implicit():
    a = [[F(0)] * S for _ in range(S)]
    a[1][0] = F(1, 4)
    a[2][0], a[2][1] = F(8611, 62500), F(-1743, 31250)
    a[3][0], a[3][1], a[3][2] = F(5012029, 34652500), F(-654441, 2922500), F(174375, 388108)
    a[4][0], a[4][1], a[4][2], a[4][3] = (F(15267082809, 155376265600), F(-71443401, 120774400),
                                          F(730878875, 902184768), F(2285395, 8070912))
    for j in range(S):
        a[5][j] = B[j]
    for i in range(1, S):
        a[i][i] = GAMMA
    return a


def _explicit():
    a = [[F(0)] * S for _ in range(S)]
    a[1][0] = F(1, 2)
    a[2][0], a[2][1] = F(13861, 62500), F(6889, 62500)
    a[3][0], a[3][1], a[3][2] = (F(-116923316275, 2393684061468), F(-2731218467317, 15368042101831),
                                 F(9408046702089, 11113171139209))
    a[4][0], a[4][1], a[4][2], a[4][3] = (F(-451086348788, 2902428689909), F(-2682348792572, 7519795681897),
                                          F(12662868775082, 11960479115383), F(3355817975965, 11060851509271))
    a[5][0], a[5][1], a[5][2], a[5][3], a[5][4] = (F(647845179188, 3216320057751), F(73281519250, 8382639484533),
                                                   F(552539513391, 3454668386233), F(3354512671639, 8306763924573),
                                                   F(4040, 17871))
    return a


A_IMPL = _implicit()
A_EXPL = _explicit()
B_HAT = list(B)


def as_float():
    """(A, b, c, A_hat, b_hat) as float64 numpy arrays."""
    f = lambda M: np.array([[float(x) for x in row] for row in M])
    v = lambda V: np.array([float(x) for x in V])
    return f(A_IMPL), v(B), v(C), f(A_EXPL), v(B_HAT)
