"""Nonlinear terms g(u) of eq. ``general`` used by the tests and workloads.

The paper's g may contain first derivatives at most (Sec. 1).  Values are needed only at
leaf-interior points, where the stage equations of eq. ``stage2`` hold; first derivatives
there come from leaf-local Chebyshev differentiation and never touch a dropped corner.

  allen_cahn(kappa):  g = kappa (u - u^3)
  fisher(kappa):      g = kappa u (1 - u)
  burgers(b1, b2):    g = -u (b1 u_x + b2 u_y)   (scalar Burgers-type transport, cf. Sec. 5.4)

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from .residual import LeafField


def none():
    return None


def allen_cahn(kappa=1.0):
    def g(grid, u):
        v = np.asarray(u[:grid.N_int], dtype=np.float64)
        return kappa * (v - v ** 3)
    return g


def fisher(kappa=1.0):
    def g(grid, u):
        v = np.asarray(u[:grid.N_int], dtype=np.float64)
        return kappa * v * (1.0 - v)
    return g


def burgers(b1=1.0, b2=1.0):
    def g(grid, u):
        F = LeafField(grid, u)
        v = F.interior(F.U)
        return -v * (b1 * F.interior(F.Ux) + b2 * F.interior(F.Uy))
    return g
