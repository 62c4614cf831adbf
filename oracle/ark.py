"""Additive Runge-Kutta step in stage form, eq. ``stage`` / eq. ``stage2`` of Sec. 3.1.

For u_t = L u + q + g(u) with u = f on the boundary: the stiff part L u goes through the
ESDIRK table (A, b, c), q + g through the ERK table (A-hat, b-hat, c), with

  u_1 = u^n
  (I - dt gamma L) u_i = u^n + dt sum_{j<i} a_ij L u_j + dt sum_{j<i} ahat_ij (q_j + g_j),  i = 2..s

at the leaf-interior points, u_i = f(t^n + c_i dt) on the boundary and flux continuity on
shared edges (each stage is one HPS solve with the operators of I - gamma dt L).
q_j = q(t^n + c_j dt) (the paper prints c_i in the definition of t^n_j; read as c_j) and
g_j = g(u_j).

The paper leaves two things open, read here as follows:
  * L u_j: for j = 1 by leaf-local differentiation of u^n; for j >= 2 from the stage
    equation itself, dt L u_j = (u_j - R_j) / gamma with R_j its right-hand side (exact
    algebra of eq. ``stage2``; ``lu_by_differentiation=True`` differentiates instead).
  * step close: the standard ARK combination
      u^{n+1} = u^n + dt sum_j b_j L u_j + dt sum_j bhat_j (q_j + g_j)
    at the interior points, u^{n+1} = f(t^{n+1}) on the boundary, and the values on shared
    edges from flux continuity, i.e. the "explicit equation u = known RHS" of Sec. 3.1.1
    solved on the same tree with the identity operator (gamma dt = 0).

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from . import tableau
from .residual import apply_L_interior


class Problem:
    """u_t = L u + q + g(u) on a grid: coef (dict of L's coefficients), q(t) -> interior
    values or None, f(t) -> boundary values (at grid.boundary_indices()) or None,
    g(grid, u) -> interior values or None."""

    def __init__(self, grid, coef, q=None, f=None, g=None):
        self.grid, self.coef, self.q, self.f, self.g = grid, coef, q, f, g

    def explicit_part(self, t, u):
        v = np.zeros(self.grid.N_int)
        if self.q is not None:
            v = v + self.q(t)
        if self.g is not None:
            v = v + self.g(self.grid, u)
        return v

    def bc(self, t):
        return None if self.f is None else self.f(t)


def ark_step(prob: Problem, hps_impl, hps_ident, u, t, dt, lu_by_differentiation=False):
    """One ARK4(3)6L[2]SA step of eq. ``stage2``; returns (u^{n+1}, stage list).

    hps_impl: HPS operators of I - gamma dt L (gamma = 1/4); hps_ident: HPS operators of the
    identity (gamma dt = 0) on the same grid.
    """
    A, b, c, Ah, bh = tableau.as_float()
    gam = A[1, 1]
    assert abs(hps_impl.gamma_dt - gam * dt) <= 1e-14 * max(1.0, abs(gam * dt)), "operator built for another dt"
    assert hps_ident.gamma_dt == 0.0
    grid = prob.grid
    s = len(c)
    u = np.asarray(u, dtype=np.float64)
    un = u[:grid.N_int].copy()
    KL, KE, stages = [], [], [u.copy()]
    # stage 1 is explicit: u_1 = u^n
    KL.append(dt * apply_L_interior(grid, prob.coef, u))
    KE.append(dt * prob.explicit_part(t + c[0] * dt, u))
    for i in range(1, s):
        R = un.copy()
        for j in range(i):
            R += A[i, j] * KL[j] + Ah[i, j] * KE[j]
        ui = hps_impl.solve(R, prob.bc(t + c[i] * dt))
        if lu_by_differentiation:
            KL.append(dt * apply_L_interior(grid, prob.coef, ui))
        else:
            KL.append((ui[:grid.N_int] - R) / gam)
        KE.append(dt * prob.explicit_part(t + c[i] * dt, ui))
        stages.append(ui)
    unew_int = un.copy()
    for j in range(s):
        unew_int += b[j] * KL[j] + bh[j] * KE[j]
    unew = hps_ident.solve(unew_int, prob.bc(t + dt))
    return unew, stages


def backward_euler_step(prob: Problem, hps_be, u, t, dt):
    """(I - dt L) u^{n+1} = u^n + dt q(t^{n+1}) with u^{n+1} = f(t^{n+1}) on the boundary
    (the time discretization of the stability theorem in Sec. 4.2).  hps_be: operators of I - dt L."""
    grid = prob.grid
    rhs = np.asarray(u[:grid.N_int], dtype=np.float64).copy()
    if prob.q is not None:
        rhs += dt * prob.q(t + dt)
    return hps_be.solve(rhs, prob.bc(t + dt))
