"""Seeded synthetic workloads shaped like the paper's experiments.

Problem data only (coefficients, sources, boundary data, initial states as functions of the
point coordinates and time, and seeded random draws); no step of the solver lives here.
Both the CUDA path and the CPU oracle take their inputs from this module.

  heat_4x4      2D heat u_t = Lap u + q on [0,1]^2, 4x4 leaves, p = 8, dt = 0.01, 100 steps,
                exact u = sin(pi x) sin(pi y) e^{-t} (homogeneous Dirichlet data; cf. Sec. 5.3)
  allen_cahn_64 u_t = 0.01 Lap u + u - u^3, 64x64 leaves, p = 16, dt = 1e-3, 200 steps,
                u0 ~ U[-0.1, 0.1] (seed 0) at every point off the outer boundary, f = 0
  varcoef_128   u_t = div(a grad u) + b.grad u + c u + q, a = 1 + 0.5 sin(2 pi x) cos(2 pi y),
                b = (0.5, -0.25), c = -1, 128x128 leaves, p = 16, dt = 1e-3,
                exact u = sin(pi x) sin(pi y) e^{-t}
  varcoef_64    the same on 64x64 leaves (profiling captures)
  instances     many independent reaction-diffusion instances of uneven sizes (leaf grids 16^2 .. 64^2,
                p in {8, 12, 16}), seeded coefficients a = 1 + alpha sin(2 pi k1 x) cos(2 pi k2 y),
                c ~ U[-2, 0], g = u - u^3, dt = 1e-3, seeded states U[-0.1, 0.1]
"""
import math

import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def uniform_state(seed, N, boundary_index, lo=-0.1, hi=0.1):
    """u0 drawn i.i.d. U[lo, hi] at every point, zero on the outer boundary."""
    u = rng(seed).uniform(lo, hi, N)
    u[np.asarray(boundary_index)] = 0.0
    return u


def random_coefficients(seed, n):
    """Random (non-smooth) coefficients with positive diffusion, for parity tests (values at points)."""
    r = rng(seed)
    return {"a11": 1.0 + 0.5 * r.random(n), "a22": 0.6 + 0.4 * r.random(n), "a1": 0.3 * r.standard_normal(n),
            "a2": 0.2 * r.standard_normal(n), "a0": -1.0 + 0.3 * r.random(n)}


class Workload:
    name = ""
    n1 = n2 = 1
    p = 8
    dt = 1e-2
    steps = 1
    g = None
    g_param = (1.0, 1.0)

    def coef(self, x, y):
        raise NotImplementedError

    def q(self, x, y, t):
        return None

    def f(self, x, y, t):
        return None

    def u0(self, x, y, boundary_index):
        raise NotImplementedError

    def exact(self, x, y, t):
        return None


class Heat4x4(Workload):
    name = "heat_4x4_p8"
    n1 = n2 = 4
    p = 8
    dt = 0.01
    steps = 100

    def coef(self, x, y):
        return {"a11": 1.0, "a22": 1.0, "a1": 0.0, "a2": 0.0, "a0": 0.0}

    def exact(self, x, y, t):
        return np.sin(math.pi * x) * np.sin(math.pi * y) * math.exp(-t)

    def q(self, x, y, t):
        return (2 * math.pi ** 2 - 1.0) * self.exact(x, y, t)

    def u0(self, x, y, boundary_index):
        return self.exact(x, y, 0.0)


class AllenCahn64(Workload):
    name = "allen_cahn_64x64_p16"
    n1 = n2 = 64
    p = 16
    dt = 1e-3
    steps = 200
    eps = 0.01
    g = "allen_cahn"
    g_param = (1.0, 0.0)
    seed = 0

    def coef(self, x, y):
        return {"a11": self.eps, "a22": self.eps, "a1": 0.0, "a2": 0.0, "a0": 0.0}

    def u0(self, x, y, boundary_index):
        return uniform_state(self.seed, x.size, boundary_index)


class VarCoef128(Workload):
    name = "varcoef_128x128_p16"
    n1 = n2 = 128
    p = 16
    dt = 1e-3
    steps = 50
    beta = (0.5, -0.25)
    c0 = -1.0

    def coef(self, x, y):
        a = 1.0 + 0.5 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y)
        ax = math.pi * np.cos(2 * math.pi * x) * np.cos(2 * math.pi * y)
        ay = -math.pi * np.sin(2 * math.pi * x) * np.sin(2 * math.pi * y)
        return {"a11": a, "a22": a, "a1": ax + self.beta[0], "a2": ay + self.beta[1], "a0": self.c0 + 0 * x}

    def exact(self, x, y, t):
        return np.sin(math.pi * x) * np.sin(math.pi * y) * math.exp(-t)

    def q(self, x, y, t):
        c = self.coef(x, y)
        e = math.exp(-t)
        u = np.sin(math.pi * x) * np.sin(math.pi * y) * e
        ux = math.pi * np.cos(math.pi * x) * np.sin(math.pi * y) * e
        uy = math.pi * np.sin(math.pi * x) * np.cos(math.pi * y) * e
        Lu = c["a11"] * (-math.pi ** 2) * u + c["a22"] * (-math.pi ** 2) * u + c["a1"] * ux + c["a2"] * uy + c["a0"] * u
        return -u - Lu

    def u0(self, x, y, boundary_index):
        return self.exact(x, y, 0.0)


class VarCoef64(VarCoef128):
    """The variable-coefficient problem on 64 x 64 leaves (p = 16): a smaller case of the same
    operator for profiling captures that must stay within a few GB of device memory."""
    name = "varcoef_64x64_p16"
    n1 = n2 = 64


WORKLOADS = {w.name: w for w in (Heat4x4(), AllenCahn64(), VarCoef128(), VarCoef64())}


class Instance(Workload):
    """One instance of the many-instance workload: u_t = div(a grad u) + c u + u - u^3 on [0,1]^2,
    a = 1 + alpha sin(2 pi k1 x) cos(2 pi k2 y), written as a11 = a22 = a, a1 = a_x, a2 = a_y, a0 = c."""
    dt = 1e-3
    g = "allen_cahn"
    g_param = (1.0, 0.0)

    def __init__(self, n, p, alpha, k1, k2, c0, index):
        self.n1 = self.n2 = int(n)
        self.p = int(p)
        self.alpha, self.k1, self.k2, self.c0 = float(alpha), int(k1), int(k2), float(c0)
        self.name = "instance_%d_%dx%d_p%d" % (index, n, n, p)

    def coef(self, x, y):
        s1, c1 = np.sin(2 * math.pi * self.k1 * x), np.cos(2 * math.pi * self.k1 * x)
        s2, c2 = np.sin(2 * math.pi * self.k2 * y), np.cos(2 * math.pi * self.k2 * y)
        a = 1.0 + self.alpha * s1 * c2
        ax = self.alpha * 2 * math.pi * self.k1 * c1 * c2
        ay = -self.alpha * 2 * math.pi * self.k2 * s1 * s2
        return {"a11": a, "a22": a, "a1": ax, "a2": ay, "a0": self.c0 + 0 * x}

    def u0(self, x, y, boundary_index):
        return uniform_state(0, x.size, boundary_index)


def instances(count=64, seed=0, grids=(16, 32, 64), orders=(8, 12, 16)):
    """`count` seeded instances: leaf grid n x n with n from `grids`, p from `orders`,
    alpha ~ U[0.1, 0.5], k1, k2 in {1, 2, 3}, c ~ U[-2, 0]."""
    r = rng(seed)
    out = []
    for i in range(count):
        out.append(Instance(int(r.choice(grids)), int(r.choice(orders)), r.uniform(0.1, 0.5), int(r.integers(1, 4)),
                            int(r.integers(1, 4)), r.uniform(-2.0, 0.0), i))
    return out
