"""Leaf apply with per-node operators on the 5th-generation tensor cores (tcgen05.mma kind::tf32,
3xTF32 products, accumulator in tensor memory, operator boxes by TMA): the first sweep of every
batched solve on a variable-coefficient handle with 16 or 32 columns.  Checked against the FP32
FFMA leaf apply (option umma_leaf = 0) and, after refinement, against the FP64 path."""
import math

import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from paper_2306_02526_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _nodal_solver(torch, n1, n2, p, gdt, seed):
    from paper_2306_02526_gb300 import hps
    tree = hps.Tree(n1, n2, -0.5, 0.5, 0.0, 1.0)
    N, N_int, N_bd = hps.hps_sizes(tree, p)
    coef = {k: to_dev(torch, v) for k, v in workloads.random_coefficients(seed, N_int).items()}
    return hps.HPSSolver(tree, p, coef, gdt), N, N_int, N_bd


# (n1, n2, p, R): two row tiles and 7 column boxes (p = 16), one row tile (p = 12, 8), padding
# columns (R = 13 -> 16, R = 29 -> 32), a leaf count below and above the SM count
@pytest.mark.parametrize("n1,n2,p,R", [(8, 4, 16, 32), (16, 16, 16, 16), (4, 4, 12, 13), (32, 16, 8, 29),
                                       (64, 32, 16, 32), (2, 1, 18, 16)])
def test_umma_first_sweep_matches_ffma_and_refines_to_fp64(n1, n2, p, R):
    torch = need_gpu()
    S, N, N_int, N_bd = _nodal_solver(torch, n1, n2, p, 0.013, p + R)
    S.batch_reserve(R)
    assert S.batch_option("umma_leaf") == 1
    r = np.random.default_rng(R * 7 + p)
    rhs = to_dev(torch, r.standard_normal((N_int, R)))
    f = to_dev(torch, r.standard_normal((N_bd, R)))
    u_tc0 = S.solve_batch(rhs, f, refine=0).cpu().numpy()
    u_tc2 = S.solve_batch(rhs, f, refine=2).cpu().numpy()
    S.batch_option("umma_leaf", 0)
    u_ff0 = S.solve_batch(rhs, f, refine=0).cpu().numpy()
    S.batch_option("umma_leaf", 1)
    S.status()  # no bounded wait of the tensor-core kernel ran out
    want = np.stack([S.solve(rhs[:, j].contiguous(), f[:, j].contiguous()).cpu().numpy() for j in range(R)], axis=1)
    e_tc0, e_ff0 = rel_max(u_tc0, want), rel_max(u_ff0, want)
    assert e_tc0 < 1e-4 and e_ff0 < 1e-4, (e_tc0, e_ff0)
    assert not np.array_equal(u_tc0, u_ff0)        # the tensor-core kernel ran (it rounds differently)
    assert rel_max(u_tc0, u_ff0) < 1e-4
    assert rel_max(u_tc2, want) <= TOL
    S.close()


@pytest.mark.parametrize("mode,refine", [(1, 1), (2, 2)])
def test_umma_ark_batch_matches_fp64(mode, refine):
    """Batched ARK steps with per-node operators and 32 states against the FP64 step column by
    column: tensor-core first sweeps with one refinement sweep (option 1), and tensor cores in every
    sweep with two refinement sweeps (option 2)."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    n1, n2, p, dt, R = 16, 8, 16, 0.01, 32
    S, N, N_int, N_bd = _nodal_solver(torch, n1, n2, p, 0.25 * dt, 3)
    x, y = hps.hps_coords(S.tree, p)
    bd = hps.hps_boundary_index(S.tree, p)
    S.batch_reserve(R)
    S.batch_option("umma_leaf", mode)
    u0 = np.stack([0.3 * np.sin(math.pi * (j % 5 + 1) * (x + 0.5)) * np.sin(math.pi * y) + 0.01 * j for j in range(R)],
                  axis=1)
    u0[bd, :] = 0.0
    ub = to_dev(torch, u0)
    us = [to_dev(torch, u0[:, j].copy()) for j in range(R)]
    for n in range(3):
        S.ark_step_batch(ub, n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0), refine=refine)
        for j in range(R):
            S.ark_step(us[j], n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0))
    S.status()
    got = ub.cpu().numpy()
    err = max(rel_max(got[:, j], us[j].cpu().numpy()) for j in range(R))
    S.close()
    assert err <= TOL, err


@pytest.mark.parametrize("n1,n2,p,R", [(8, 4, 16, 32), (16, 16, 12, 16)])
def test_bf16_trial_first_sweep_is_coarse_and_refines(n1, n2, p, R):
    """BF16 trial (option umma_leaf = 3): the first sweep's per-node leaf applies as one BF16
    product on the tensor cores.  Its unrefined error sits at BF16 level (well above the FP32
    sweep's), and FP32 refinement sweeps still bring the solve to the mixed-precision tolerance."""
    torch = need_gpu()
    S, N, N_int, N_bd = _nodal_solver(torch, n1, n2, p, 0.013, 7 * p + R)
    S.batch_reserve(R)
    r = np.random.default_rng(R + p)
    rhs = to_dev(torch, r.standard_normal((N_int, R)))
    f = to_dev(torch, r.standard_normal((N_bd, R)))
    want = np.stack([S.solve(rhs[:, j].contiguous(), f[:, j].contiguous()).cpu().numpy() for j in range(R)], axis=1)
    e_tf = rel_max(S.solve_batch(rhs, f, refine=0).cpu().numpy(), want)
    S.batch_option("umma_leaf", 3)
    e_bf = [rel_max(S.solve_batch(rhs, f, refine=k).cpu().numpy(), want) for k in (0, 1, 2, 3)]
    S.status()
    S.close()
    assert 10 * e_tf < e_bf[0] < 5e-2, (e_tf, e_bf)
    assert e_bf[1] < e_bf[0] and min(e_bf[2], e_bf[3]) <= TOL, e_bf
