"""Writes varcoef128_ark_step.txt: the oracle's values after one ARK4(3)6L[2]SA step (eq.
``stage2`` with the step close of Sec. 3.1.1) of the variable-coefficient workload -- 128 x 128
leaves, p = 16, a = 1 + 0.5 sin(2 pi x) cos(2 pi y), b = (0.5, -0.25), c = -1, dt = 1e-3, manufactured
u = sin(pi x) sin(pi y) e^{-t} (workloads.VarCoef128) -- at seeded sample points, plus the max-norm
of the whole oracle result, plus the oracle's own sensitivity to rounding: the same step with every
coefficient value moved by one unit in the last place (seeded signs), whose largest change of the
result measures how far two correct FP64 evaluations in different rounding orders may differ on
this discretization (the stage operators I - gamma dt L are ill-conditioned at h = 1/128).  Calls
only oracle/ and the input module; about 10 minutes and 45 GB of host memory.

    python tests/golden/make_varcoef128_step.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ark as oark  # noqa: E402
from oracle.grid import Grid  # noqa: E402
from oracle.hps import HPS  # noqa: E402
from paper_2306_02526_gb300 import workloads  # noqa: E402


def sample_indices(g):
    """3000 seeded points, every interior point of the first and last leaf, the first 300
    vertical-edge and the last 300 horizontal-edge points (global order of the grid)."""
    q = g.m * g.m
    r = np.random.default_rng(128)
    parts = [r.choice(g.N, 3000, replace=False), np.arange(q), np.arange(g.N_int - q, g.N_int),
             np.arange(g.N_int, g.N_int + 300), np.arange(g.N - 300, g.N)]
    return np.unique(np.concatenate(parts))


def main():
    wl = workloads.VarCoef128()
    g = Grid(wl.n1, wl.n2, wl.p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = wl.coef(X[I], Y[I])
    prob = oark.Problem(g, coef, q=lambda t: wl.q(X[I], Y[I], t))
    u0 = wl.u0(X, Y, bd)
    Hi = HPS(g, coef, 0.25 * wl.dt)
    Hid = HPS(g, coef, 0.0)
    u1, _ = oark.ark_step(prob, Hi, Hid, u0, 0.0, wl.dt)
    del Hi, Hid
    # the same step with every coefficient value one ulp away (seeded direction per value)
    r = np.random.default_rng(2306)
    coef_p = {k: np.nextafter(v, np.where(r.random(v.shape) < 0.5, -np.inf, np.inf)) for k, v in coef.items()}
    prob_p = oark.Problem(g, coef_p, q=lambda t: wl.q(X[I], Y[I], t))
    u1p, _ = oark.ark_step(prob_p, HPS(g, coef_p, 0.25 * wl.dt), HPS(g, coef_p, 0.0), u0, 0.0, wl.dt)
    sens = np.abs(u1p - u1).max()
    idx = sample_indices(g)
    with open(os.path.join(HERE, "varcoef128_ark_step.txt"), "w") as fh:
        fh.write("# oracle ARK4(3)6L[2]SA step (eq. stage2, Sec. 3.1.1 close), workloads.VarCoef128: 128x128 leaves,\n")
        fh.write("# p = 16, dt = 1e-3, t = 0 -> dt, u0 = sin(pi x) sin(pi y); global index, value after the step\n")
        fh.write("# written by tests/golden/make_varcoef128_step.py (oracle/ only)\n")
        fh.write("# max_abs %.17e\n" % np.abs(u1).max())
        fh.write("# ulp_sensitivity %.17e (max change of the result when every coefficient moves by one ulp)\n" % sens)
        for i in idx:
            fh.write("%d %.17e\n" % (i, u1[i]))


if __name__ == "__main__":
    main()
