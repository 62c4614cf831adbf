"""A caller-supplied nonlinear term g (HPS_G_USER): the library calls the hook on its stream for
every stage value and adds dt g(u_j) to the stage's explicit term (eq. stage2).  A hook that
computes Allen-Cahn must agree with the preset to rounding; a g the presets do not have
(0.7 sin u) must match the oracle stepping the same g; with graphs on, the replayed steps
(the hook's work recorded with them) must equal the eager ones; a hook that fails ends the
step with an error."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle import ark as oark
from oracle.grid import Grid
from oracle.hps import HPS

pytestmark = pytest.mark.gpu

COEF = {"a11": 0.05, "a22": 0.03, "a1": 0.1, "a0": -0.2}


class _SinG:
    """g(u) = 0.7 sin(u) at the interior points, allocation-free (out= forms)."""

    def __init__(self, n_int):
        self.n_int = n_int
        self.calls = 0

    def __call__(self, u, g_out):
        import torch
        self.calls += 1
        torch.sin(u[: self.n_int], out=g_out)
        g_out.mul_(0.7)


class _AllenCahnG:
    def __init__(self, torch, n_int, kappa):
        self.n_int, self.kappa = n_int, kappa
        self.tmp = torch.empty(n_int, dtype=torch.float64, device="cuda")

    def __call__(self, u, g_out):
        import torch
        v = u[: self.n_int]
        torch.mul(v, v, out=self.tmp)
        self.tmp.mul_(v)
        torch.sub(v, self.tmp, out=g_out)
        g_out.mul_(self.kappa)


def _setup(torch, n1=8, n2=4, p=10, dt=0.02):
    from paper_2306_02526_gb300 import hps
    tree = hps.Tree(n1, n2)
    S = hps.HPSSolver(tree, p, COEF, 0.25 * dt)
    x, y = hps.hps_coords(tree, p)
    u0 = 0.4 * np.sin(np.pi * x) * np.sin(np.pi * y) + 0.1 * x * (1.0 - x) * y
    u0[hps.hps_boundary_index(tree, p)] = 0.0
    return S, u0, dt


def test_user_g_matches_preset_allen_cahn():
    torch = need_gpu()
    S, u0, dt = _setup(torch)
    a = to_dev(torch, u0)
    b = to_dev(torch, u0)
    hook = _AllenCahnG(torch, S.N_int, 1.5)
    for n in range(6):
        S.ark_step(a, n * dt, dt, g="allen_cahn", g_param=(1.5, 0.0))
        S.ark_step(b, n * dt, dt, g=hook)
    assert rel_max(b.cpu().numpy(), a.cpu().numpy()) <= 1e-13
    S.close()


def test_user_g_matches_oracle():
    torch = need_gpu()
    S, u0, dt = _setup(torch)
    hook = _SinG(S.N_int)
    u = to_dev(torch, u0)
    steps = 4
    for n in range(steps):
        S.ark_step(u, n * dt, dt, g=hook)
    assert hook.calls == 6 * steps  # stage 1 and the five implicit stages of every step
    g = Grid(8, 4, 10)
    prob = oark.Problem(g, COEF, g=lambda grid, v: 0.7 * np.sin(np.asarray(v[: grid.N_int])))
    Hi, Hid = HPS(g, COEF, 0.25 * dt), HPS(g, COEF, 0.0)
    v = u0.copy()
    for n in range(steps):
        v, _ = oark.ark_step(prob, Hi, Hid, v, n * dt, dt)
    assert rel_max(u.cpu().numpy(), v) <= 1e-12
    S.close()


def test_user_g_graph_replay_equals_eager():
    torch = need_gpu()
    S, u0, dt = _setup(torch, 16, 16, 12, 0.01)
    hook = _SinG(S.N_int)
    eager = to_dev(torch, u0)
    for n in range(5):
        S.ark_step(eager, n * dt, dt, g=hook)
    calls_eager = hook.calls
    S.set_graph(True)
    graphed = to_dev(torch, u0)
    for n in range(5):  # eager, recorded, then three replays that do not call the hook
        S.ark_step(graphed, n * dt, dt, g=hook)
    torch.cuda.synchronize()
    assert hook.calls - calls_eager == 2 * 6
    assert torch.equal(graphed, eager)
    S.close()


def test_failing_user_g_raises():
    torch = need_gpu()
    S, u0, dt = _setup(torch, 2, 2, 8)

    def bad(u, g_out):
        raise ValueError("no g here")

    u = to_dev(torch, u0)
    with pytest.raises(ValueError):
        S.ark_step(u, 0.0, dt, g=bad)
    torch.cuda.synchronize()
    S.ark_step(u, 0.0, dt, g="fisher")  # the handle stays usable
    from paper_2306_02526_gb300 import _lib
    with pytest.raises(_lib.HPSError):  # the batched path has no hook
        S.batch_reserve(4)
        ub = torch.zeros((S.N, 4), dtype=torch.float64, device="cuda")
        S.ark_step_batch(ub, 0.0, dt, g="allen_cahn", g_param=(1.0, 0.0), refine=1)
        import ctypes
        t = _lib.hps_ark_terms()
        t.g_kind = _lib.HPS_G_USER
        t.g_fn = ctypes.cast(S._g_hook(_SinG(S.N_int)), ctypes.c_void_p)
        from paper_2306_02526_gb300._lib import check, lib
        check(lib().ark_step_batch(S._h, 4, ctypes.c_void_p(ub.data_ptr()), ctypes.c_double(0.0),
                                   ctypes.c_double(dt), ctypes.byref(t), 1,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "ark_step_batch")
    S.close()
