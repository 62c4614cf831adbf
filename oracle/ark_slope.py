"""Slope formulation of the ARK step (Sec. 3.1, eq. ``slope0``) for g = 0, with the flux-jump
penalization of the interface conditions (Sec. 3.1, "Penalization in the slope formulation").

For u_t = L u + q with Dirichlet data f, the slopes k_i approximate u_t at t^n + c_i dt:

  k_1 = L u^n + q_1                                                      (explicit)
  (I - dt gamma L) k_i = L u^n + dt sum_{j<i} a_ij L k_j + q_i,  i = 2..s  (one HPS solve each)
  u^{n+1} = u^n + dt sum_j b_j k_j                                       (at every point)

Readings of the passages (the paper leaves them open or prints them garbled):
  * S1 q in every slope: eq. ``slope0`` prints q only in k_1; it is read as in eq. ``slope``
    (k_i = L U_i + q_i with U_i = u^n + dt sum_j a_ij k_j), so q goes through the implicit table.
  * S2 k_1 is an explicit equation "k = known RHS" (Sec. 3.1.1): its shared-edge values come from
    the same tree solved with the identity operator, like the stage form's close.
  * S3 penalized interface rows: the printed condition [[T k + h^k - dt^-1 h^u]] = 0 is read as
    "the flux jump of every slope equals -1/dt times the flux jump of u^n", i.e. the interface rows
    of each slope system have the right-hand side -J(u^n)/dt, J = (west/south flux) - (east/north
    flux).  Since sum_j b_j = 1, u^{n+1} then has no flux jump whatever the jump of u^n; without
    the penalization (penalize=False) the jump of u^n is carried over unchanged.
  * S4 slope boundary data: u_t(t^n + c_i dt) where the caller knows it (kbc), else zero (the
    case of time-independent data the paper names).
  * S5 dt L k_j: by leaf-local differentiation for j = 1, from the slope equation itself
    for j >= 2, dt L k_j = (k_j - R_j) / gamma (exact algebra, as R9 of the stage form).

With a nonlinear term (eq. ``slope``, ``ark_slope_step_g``) explicit slopes l_i join the k_i:

  k_1 = L u^n + q_1,  l_1 = g(u^n)
  (I - dt gamma L) k_i = L u^n + dt sum_{j<i} a_ij L k_j + dt sum_{j<i} ahat_ij L l_j + q_i
  l_i = g(U_i),  U_i = u^n + dt sum_{j<=i} a_ij k_j + dt sum_{j<i} ahat_ij l_j
  u^{n+1} = u^n + dt sum_j b_j k_j + dt sum_j bhat_j l_j

with three more readings:
  * S6 every l_i is an explicit equation "l = known RHS" like k_1 (S2): g(U_i) at the interior
    points, its shared-edge values from the identity-operator system with a continuous flux (no
    penalization: the l_i carry no flux jump, so with S3 u^{n+1} has none either), zero on the
    boundary; dt L l_j by leaf-local differentiation of that field.
  * S7 boundary data: the paper gives slope boundary conditions with g present only for
    time-independent Dirichlet data (zero for k_i and l_i); other data are rejected.
  * S8 U_i at every point (interior, shared edges, boundary) from the slopes' complete fields, so
    that a g with first derivatives takes them by leaf-local differentiation of U_i.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from . import tableau
from .residual import apply_L_interior, flux_jumps


def ark_slope_step(grid, coef, hps_impl, hps_ident, u, t, dt, q=None, kbc=None, penalize=True):
    """One ARK4(3)6L[2]SA step in slope form; returns (u^{n+1}, slopes).

    q(t): interior source values or None; kbc(t): slope boundary values (u_t on the boundary at
    grid.boundary_indices()) or None for zero; hps_impl: HPS operators of I - gamma dt L;
    hps_ident: those of the identity (gamma dt = 0) on the same grid.
    """
    A, b, c, _, _ = tableau.as_float()
    gam = A[1, 1]
    assert abs(hps_impl.gamma_dt - gam * dt) <= 1e-14 * max(1.0, abs(gam * dt)), "operator built for another dt"
    assert hps_ident.gamma_dt == 0.0
    s = len(c)
    u = np.asarray(u, dtype=np.float64)
    jump = -flux_jumps(grid, u) / dt if penalize else None  # S3
    q_at = (lambda tt: np.zeros(grid.N_int)) if q is None else q
    kb = (lambda tt: None) if kbc is None else kbc
    Lu = apply_L_interior(grid, coef, u)
    slopes, dLk = [], []
    # k_1: explicit, edges by the identity-operator system (S2); dt L k_1 by differentiation (S5)
    k = hps_ident.solve(Lu + q_at(t + c[0] * dt), kb(t + c[0] * dt), jump=jump)
    slopes.append(k)
    dLk.append(dt * apply_L_interior(grid, coef, k))
    for i in range(1, s):
        R = Lu + q_at(t + c[i] * dt)
        for j in range(i):
            R = R + A[i, j] * dLk[j]
        k = hps_impl.solve(R, kb(t + c[i] * dt), jump=jump)
        slopes.append(k)
        dLk.append((k[:grid.N_int] - R) / gam)  # S5
    un = u.copy()
    for j in range(s):
        un = un + dt * b[j] * slopes[j]
    return un, slopes


def ark_slope_step_g(grid, coef, hps_impl, hps_ident, u, t, dt, g, q=None, penalize=True):
    """One ARK4(3)6L[2]SA step in slope form with a nonlinear term g (eq. ``slope``, readings
    S1-S3, S5-S8) for time-independent Dirichlet data; returns (u^{n+1}, k slopes, l slopes).

    g(grid, v) -> interior values of g(v) for a complete field v (``oracle.nonlinear``); q(t):
    interior source values or None."""
    A, b, c, Ah, bh = tableau.as_float()
    gam = A[1, 1]
    assert abs(hps_impl.gamma_dt - gam * dt) <= 1e-14 * max(1.0, abs(gam * dt)), "operator built for another dt"
    assert hps_ident.gamma_dt == 0.0
    s = len(c)
    u = np.asarray(u, dtype=np.float64)
    jump = -flux_jumps(grid, u) / dt if penalize else None  # S3
    q_at = (lambda tt: np.zeros(grid.N_int)) if q is None else q
    Lu = apply_L_interior(grid, coef, u)
    ks, ls, dLk, dLl = [], [], [], []

    def explicit_l(v):  # S6: g at the interior, edges by the identity-operator system, zero boundary
        lf = hps_ident.solve(g(grid, v), None)
        return lf, dt * apply_L_interior(grid, coef, lf)

    k = hps_ident.solve(Lu + q_at(t + c[0] * dt), None, jump=jump)  # S2
    ks.append(k)
    dLk.append(dt * apply_L_interior(grid, coef, k))
    lf, dl = explicit_l(u)
    ls.append(lf)
    dLl.append(dl)
    for i in range(1, s):
        R = Lu + q_at(t + c[i] * dt)
        for j in range(i):
            R = R + A[i, j] * dLk[j] + Ah[i, j] * dLl[j]
        k = hps_impl.solve(R, None, jump=jump)
        ks.append(k)
        dLk.append((k[:grid.N_int] - R) / gam)  # S5
        U = u.copy()  # S8
        for j in range(i + 1):
            U = U + dt * A[i, j] * ks[j]
        for j in range(i):
            U = U + dt * Ah[i, j] * ls[j]
        lf, dl = explicit_l(U)
        ls.append(lf)
        dLl.append(dl)
    un = u.copy()
    for j in range(s):
        un = un + dt * b[j] * ks[j] + dt * bh[j] * ls[j]
    return un, ks, ls
