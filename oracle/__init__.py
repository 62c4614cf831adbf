"""Plain, slow FP64 CPU oracle for the RKHPS method (Chen, Appelo, Babb, Martinsson,
"Fast and high-order approximation of parabolic equations using hierarchical direct
solvers and implicit Runge-Kutta methods").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` use it.  It shares no code with the CUDA implementation under
``paper_2306_02526_gb300/``.

Modules (each function cites the passage of the paper it follows):

* ``cheb``      -- Chebyshev-Lobatto nodes and the Lagrange differentiation matrix (Sec. 2.1).
* ``grid``      -- the global collocation points without corners and their ordering (Sec. 2.1).
* ``leaf``      -- leaf collocation operator, solution operator S and DtN map T (eq. ``leaf``).
* ``hps``       -- hierarchical tree, merge build (Sec. 2.1 merge formulas), upward body-load
                   and downward solve sweeps (Alg. 1 plus the particular-solution terms).
* ``dense``     -- the global collocation system A of eq. ``sparse_A`` assembled and solved
                   densely (brute force for tiny trees).
* ``tableau``   -- ARK4(3)6L[2]SA Butcher tables in exact rational arithmetic (Table ``tbl:butcher``).
* ``ark``       -- the additive Runge-Kutta step in stage form (eq. ``stage2``).
* ``ark_slope`` -- the step in slope form for g = 0 (eq. ``slope0``) with penalized interface
                   conditions (Sec. 3.1, penalization in the slope formulation).
* ``nonlinear`` -- the nonlinear terms g(u) used by the tests (leaf-local differentiation).

Parity status: every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""
