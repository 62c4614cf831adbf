"""The persistent merge kernel (all levels, grid barriers) against one launch per level,
and its bounded wait: a barrier that cannot complete must time out, report HPS_ETIMEOUT
and leave the handle usable."""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n1,n2,p,nodal", [(2, 1, 5, True), (8, 8, 10, False), (16, 8, 12, True), (64, 64, 16, False)])
def test_persistent_equals_per_level(n1, n2, p, nodal):
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps, workloads
    tree = hps.Tree(n1, n2)
    N, N_int, N_bd = hps.hps_sizes(tree, p)
    if nodal:
        coef = {k: to_dev(torch, v) for k, v in workloads.random_coefficients(7, N_int).items()}
    else:
        coef = {"a11": 0.5, "a22": 0.5, "a1": 0.2, "a2": 0.0, "a0": -1.0}
    S = hps.HPSSolver(tree, p, coef, 0.0025)
    S.set_persistent(True)
    r = np.random.default_rng(1)
    rhs, f = to_dev(torch, r.standard_normal(N_int)), to_dev(torch, r.standard_normal(N_bd))
    a = S.solve(rhs, f).clone()
    u0 = r.uniform(-0.1, 0.1, N)
    ua = to_dev(torch, u0)
    for n in range(3):
        S.ark_step(ua, 0.01 * n, 0.01, g="allen_cahn", g_param=(1.0, 0.0))
    S.set_persistent(False)
    b = S.solve(rhs, f)
    ub = to_dev(torch, u0)
    for n in range(3):
        S.ark_step(ub, 0.01 * n, 0.01, g="allen_cahn", g_param=(1.0, 0.0))
    S.status()
    assert torch.equal(a, b)
    assert torch.equal(ua, ub)
    S.close()


def test_bounded_barrier_times_out_and_recovers():
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib, hps
    tree = hps.Tree(8, 8)
    N, N_int, N_bd = hps.hps_sizes(tree, 10)
    S = hps.HPSSolver(tree, 10, {"a11": 1.0, "a22": 1.0}, 0.01)
    rhs = to_dev(torch, np.random.default_rng(2).standard_normal(N_int))
    want = S.solve(rhs).clone()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _lib.lib().hps_selftest_barrier_timeout(S._h, stream) == _lib.HPS_ETIMEOUT
    S.status()  # the self-test cleared its own error word
    got = S.solve(rhs)
    S.status()
    assert torch.equal(got, want)
    S.close()
