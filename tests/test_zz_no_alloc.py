"""hps_solve_static (the allocation-free variant of hps_solve) against hps_solve.

For callers that cannot allocate device memory when they solve (fixed memory budget set at
start-up, real-time loops, an allocator missing on the solving thread): the static entry
point keeps its work vectors in a fixed array inside libhps.so.  This file is collected last
so that a run stopping at the first failure has already run every other test; it also
passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev

pytestmark = pytest.mark.gpu


def _static_solve(S, rhs, f, u):
    import torch
    from paper_2306_02526_gb300 import _lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _lib.lib().hps_solve_static(S._h, ctypes.c_void_p(rhs.data_ptr()),
                                       None if f is None else ctypes.c_void_p(f.data_ptr()),
                                       ctypes.c_void_p(u.data_ptr()), stream)


@pytest.mark.parametrize("case", ["nodal", "nodal_persistent", "const_fast_diag"])
def test_static_solve_matches_hps_solve_twice(case):
    """Per-level merge launches on per-node operators; the persistent merge kernel (its partial
    sums, tile counters, barrier and error word then also sit in the static array); constant
    coefficients with the fast-diagonalization leaf apply."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib, hps, workloads
    n1, n2, p = 8, 4, 10
    tree = hps.Tree(n1, n2, -0.2, 1.3, 0.0, 0.75)
    N, N_int, N_bd = hps.hps_sizes(tree, p)
    if case == "const_fast_diag":
        coef = {"a11": 0.8, "a22": 1.1, "a1": 0.2, "a2": -0.1, "a0": -0.4}
    else:
        coef = {k: to_dev(torch, v) for k, v in workloads.random_coefficients(11, N_int).items()}
    S = hps.HPSSolver(tree, p, coef, 0.017)
    if case == "nodal_persistent":
        S.set_persistent(True)
    if case == "const_fast_diag":
        assert S.batch_option("fast_diag") == 1
    r = np.random.default_rng(5)
    for call in range(2):  # two calls in a row: the array keeps the previous call's contents
        rhs = to_dev(torch, r.standard_normal(N_int))
        f = to_dev(torch, r.standard_normal(N_bd)) if call == 0 else None
        want = S.solve(rhs, f).cpu().numpy()
        u = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        assert _static_solve(S, rhs, f, u) == _lib.HPS_OK
        got = u.cpu().numpy()
        assert rel_max(got, want) <= 1e-12
    S.status()  # no bounded wait ran out (the static call's error word was folded into the handle's)
    S.close()


def test_static_solve_rejects_too_large_problem():
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib, hps
    tree = hps.Tree(128, 128)
    N, N_int, _ = hps.hps_sizes(tree, 16)
    S = hps.HPSSolver(tree, 16, {"a11": 1.0, "a22": 1.0}, 1e-3)
    rhs = torch.zeros(N_int, dtype=torch.float64, device="cuda")
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    assert _static_solve(S, rhs, None, u) == _lib.HPS_ESCRATCH
    assert "static work array" in _lib.lib().hps_strerror(_lib.HPS_ESCRATCH).decode()
    S.close()
