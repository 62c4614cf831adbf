"""Batched mixed precision (FP32 sweeps + FP64 refinement, R right-hand sides) against the
FP64 path and the oracle.  Tolerance of the mixed path: 1e-10 relative max-norm."""
import math

import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle import ark as oark
from oracle import nonlinear
from oracle.grid import Grid
from oracle.hps import HPS
from paper_2306_02526_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _solver(torch, n1, n2, p, coef, gdt, dom=(0.0, 1.0, 0.0, 1.0)):
    from paper_2306_02526_gb300 import hps
    tree = hps.Tree(n1, n2, *dom)
    cg = {k: (to_dev(torch, v) if np.ndim(v) else float(v)) for k, v in coef.items()}
    return hps.HPSSolver(tree, p, cg, gdt)


@pytest.mark.parametrize("n1,n2,p,R,nodal", [(1, 1, 5, 1, False), (2, 2, 7, 3, True), (8, 4, 9, 8, True),
                                             (16, 16, 12, 32, False), (8, 16, 16, 5, True), (16, 8, 16, 1, True),
                                             (4, 4, 13, 4, True)])
def test_solve_batch_matches_fp64(n1, n2, p, R, nodal):
    torch = need_gpu()
    g = Grid(n1, n2, p, -0.5, 0.5, 0.0, 1.0)
    coef = workloads.random_coefficients(p, g.N_int) if nodal else {"a11": 1.0, "a22": 0.7, "a1": 0.3, "a2": 0.0,
                                                                    "a0": -0.5}
    S = _solver(torch, n1, n2, p, coef, 0.013, (-0.5, 0.5, 0.0, 1.0))
    S.batch_reserve(R)
    r = np.random.default_rng(R + p)
    rhs = r.standard_normal((g.N_int, R))
    f = r.standard_normal((g.boundary_indices().size, R))
    errs = []
    for refine in (0, 1, 2):
        u = S.solve_batch(to_dev(torch, rhs), to_dev(torch, f), refine=refine).cpu().numpy()
        err = 0.0
        for j in range(R):
            want = S.solve(to_dev(torch, rhs[:, j].copy()), to_dev(torch, f[:, j].copy())).cpu().numpy()
            err = max(err, rel_max(u[:, j], want))
        errs.append(err)
    assert errs[0] < 1e-4               # FP32 sweep alone
    assert errs[2] <= TOL, errs         # refined to FP64 accuracy
    assert errs[2] < errs[0]
    if g.N <= 1500:
        want = HPS(g, coef, 0.013).solve(rhs[:, 0], f[:, 0])
        assert rel_max(S.solve_batch(to_dev(torch, rhs), to_dev(torch, f), refine=2).cpu().numpy()[:, 0], want) <= TOL
    S.close()


def test_ark_batch_heat_matches_oracle():
    """4 different initial states of the heat problem (4x4 leaves, p = 8), 20 ARK steps."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    wl = workloads.Heat4x4()
    g = Grid(wl.n1, wl.n2, wl.p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = wl.coef(X[I], Y[I])
    R = 4
    S = _solver(torch, wl.n1, wl.n2, wl.p, coef, 0.25 * wl.dt)
    S.batch_reserve(R)
    c = hps.hps_ark_abscissae()
    u0 = np.stack([wl.u0(X, Y, bd) * (1 + 0.25 * j) + 0.01 * j * np.sin(3 * X) * np.sin(2 * math.pi * Y)
                   for j in range(R)], axis=1)
    for j in range(R):
        u0[bd, j] = 0.0
    ug = to_dev(torch, u0)
    prob = oark.Problem(g, coef, q=lambda t: wl.q(X, Y, t)[I])
    Hi, Hid = HPS(g, coef, 0.25 * wl.dt), HPS(g, coef, 0.0)
    uo = [u0[:, j].copy() for j in range(R)]
    t = 0.0
    for n in range(20):
        q = np.stack([np.repeat(wl.q(X, Y, t + cj * wl.dt)[I][:, None], R, axis=1) for cj in c])
        S.ark_step_batch(ug, t, wl.dt, q=to_dev(torch, q), refine=2)
        for j in range(R):
            uo[j], _ = oark.ark_step(prob, Hi, Hid, uo[j], t, wl.dt)
        t += wl.dt
    got = ug.cpu().numpy()
    for j in range(R):
        assert rel_max(got[:, j], uo[j]) <= TOL
    S.close()


@pytest.mark.parametrize("gname,R,groups", [("allen_cahn", 6, 1), ("burgers", 6, 1), ("burgers", 10, 3)])
def test_ark_batch_varcoef_inhomogeneous_matches_fp64(gname, R, groups):
    """Stage sources q and boundary data f per column; with groups the columns run as column
    groups (4, 4, 2 of 10) on their own streams, reading q and f in place."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    n1, n2, p, dt = 8, 4, 10, 0.02
    g = Grid(n1, n2, p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = workloads.VarCoef128().coef(X[I], Y[I])
    S = _solver(torch, n1, n2, p, coef, 0.25 * dt)
    S.batch_reserve(R, groups=groups)
    c = hps.hps_ark_abscissae()
    gp = (0.8, -0.3)
    qf = lambda t, j: np.cos(X[I] + t + 0.1 * j) * np.sin(2 * Y[I])
    ff = lambda t, j: (np.sin(X + 2 * Y - 0.2 * j) * (1 + t))[bd]
    u0 = np.stack([0.3 * np.sin(math.pi * X) * np.cos(Y + j) for j in range(R)], axis=1)
    for j in range(R):
        u0[bd, j] = ff(0.0, j)
    ub = to_dev(torch, u0)
    us = [to_dev(torch, u0[:, j].copy()) for j in range(R)]
    t = 0.0
    for n in range(4):
        qb = np.stack([np.stack([qf(t + cj * dt, j) for j in range(R)], axis=1) for cj in c])
        fb = np.stack([np.stack([ff(t + cj * dt, j) for j in range(R)], axis=1) for cj in c])
        S.ark_step_batch(ub, t, dt, q=to_dev(torch, qb), f=to_dev(torch, fb), g=gname, g_param=gp, refine=2)
        for j in range(R):
            S.ark_step(us[j], t, dt, q=to_dev(torch, qb[:, :, j].reshape(-1).copy()),
                       f=to_dev(torch, fb[:, :, j].reshape(-1).copy()), g=gname, g_param=gp)
        t += dt
    got = ub.cpu().numpy()
    for j in range(R):
        assert rel_max(got[:, j], us[j].cpu().numpy()) <= TOL
    S.close()


@pytest.mark.parametrize("gname,groups", [("allen_cahn", 1), ("allen_cahn", 3), ("fisher", 2)])
def test_fused_stage_epilogue_with_sources(gname, groups):
    """Constant coefficients (the persistent leaf solve that writes the stage epilogue), stage
    sources q and boundary data f per column, column groups reading q at their column offset:
    the fused epilogue against the separate pass (to rounding) and against the FP64 path."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    n1, n2, p, dt, R = 8, 4, 10, 0.02, 10
    g = Grid(n1, n2, p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    c = hps.hps_ark_abscissae()
    gp = (0.8, 0.0)
    qf = lambda t, j: np.cos(X[I] + t + 0.1 * j) * np.sin(2 * Y[I])
    ff = lambda t, j: (np.sin(X + 2 * Y - 0.2 * j) * (1 + t))[bd]
    u0 = np.stack([0.3 * np.sin(math.pi * X) * np.cos(Y + j) for j in range(R)], axis=1)
    for j in range(R):
        u0[bd, j] = ff(0.0, j)
    outs = []
    for fuse in (1, 0):
        S = _solver(torch, n1, n2, p, {"a11": 0.03, "a22": 0.02}, 0.25 * dt)
        S.batch_reserve(R, groups=groups)
        S.batch_option("fuse_epilogue", fuse)
        ub = to_dev(torch, u0)
        t = 0.0
        for n in range(3):
            qb = np.stack([np.stack([qf(t + cj * dt, j) for j in range(R)], axis=1) for cj in c])
            fb = np.stack([np.stack([ff(t + cj * dt, j) for j in range(R)], axis=1) for cj in c])
            S.ark_step_batch(ub, t, dt, q=to_dev(torch, qb), f=to_dev(torch, fb), g=gname, g_param=gp, refine=1)
            t += dt
        outs.append(ub.cpu().numpy())
        if fuse:
            us = [to_dev(torch, u0[:, j].copy()) for j in range(R)]
            t = 0.0
            for n in range(3):
                for j in range(R):
                    qj = np.stack([qf(t + cj * dt, j) for cj in c]).reshape(-1)
                    fj = np.stack([ff(t + cj * dt, j) for cj in c]).reshape(-1)
                    S.ark_step(us[j], t, dt, q=to_dev(torch, qj), f=to_dev(torch, fj), g=gname, g_param=gp)
                t += dt
            for j in range(R):
                assert rel_max(outs[0][:, j], us[j].cpu().numpy()) <= TOL
        S.close()
    assert rel_max(outs[0], outs[1]) <= 1e-13


@pytest.mark.parametrize("n1,n2,p,R", [(1, 1, 6, 3), (1, 4, 7, 5), (8, 2, 9, 6), (2, 2, 16, 33), (2, 1, 26, 16)])
def test_ark_batch_close_on_degenerate_trees_matches_oracle(n1, n2, p, R):
    """Batched step (constant coefficients, a source, boundary data) on a single leaf, a column
    of leaves, odd p and a rectangle, R not a multiple of 4 (and > 32): 2 steps against the
    oracle, column by column."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    dt = 0.02
    g = Grid(n1, n2, p)
    X, Y = g.coords()
    I, bd = np.arange(g.N_int), g.boundary_indices()
    coef = {"a11": 0.5, "a22": 0.8}
    S = _solver(torch, n1, n2, p, coef, 0.25 * dt)
    S.batch_reserve(R)
    c = hps.hps_ark_abscissae()
    qf = lambda t, j: np.cos(X[I] - t + 0.1 * j) * np.sin(3 * Y[I])
    ff = lambda t, j: (np.sin(2 * X + Y - 0.05 * j) * (1 - t))[bd]
    u0 = np.stack([0.2 * np.cos(2 * X + 0.1 * j) * np.sin(5 * Y) for j in range(R)], axis=1)
    for j in range(R):
        u0[bd, j] = ff(0.0, j)
    ug = to_dev(torch, u0)
    Hi, Hid = HPS(g, coef, 0.25 * dt), HPS(g, coef, 0.0)
    uo = [u0[:, j].copy() for j in range(R)]
    t = 0.0
    for n in range(2):
        qb = np.stack([np.stack([qf(t + cj * dt, j) for j in range(R)], axis=1) for cj in c])
        fb = np.stack([np.stack([ff(t + cj * dt, j) for j in range(R)], axis=1) for cj in c])
        S.ark_step_batch(ug, t, dt, q=to_dev(torch, qb), f=to_dev(torch, fb), g="fisher", g_param=(0.7, 0.0),
                         refine=2)
        for j in range(R):
            prob = oark.Problem(g, coef, q=lambda tt, j=j: qf(tt, j), f=lambda tt, j=j: ff(tt, j),
                                g=nonlinear.fisher(0.7))
            uo[j], _ = oark.ark_step(prob, Hi, Hid, uo[j], t, dt)
        t += dt
    got = ug.cpu().numpy()
    for j in range(R):
        assert rel_max(got[:, j], uo[j]) <= TOL
    S.close()


def test_ark_batch_full_size_allen_cahn():
    """The bench workload (64x64 leaves, p = 16) with 8 seeded states: 2 batched mixed steps
    against the FP64 path column by column."""
    torch = need_gpu()
    wl = workloads.AllenCahn64()
    from paper_2306_02526_gb300 import hps
    tree = hps.Tree(wl.n1, wl.n2)
    N, N_int, N_bd = hps.hps_sizes(tree, wl.p)
    x, y = hps.hps_coords(tree, wl.p)
    bidx = hps.hps_boundary_index(tree, wl.p)
    S = hps.HPSSolver(tree, wl.p, {"a11": wl.eps, "a22": wl.eps}, 0.25 * wl.dt)
    R = 8
    S.batch_reserve(R)
    u0 = np.stack([workloads.uniform_state(j, N, bidx) for j in range(R)], axis=1)
    ub = to_dev(torch, u0)
    us = [to_dev(torch, u0[:, j].copy()) for j in range(R)]
    for n in range(2):
        S.ark_step_batch(ub, n * wl.dt, wl.dt, g="allen_cahn", g_param=(1.0, 0.0), refine=2)
        for j in range(R):
            S.ark_step(us[j], n * wl.dt, wl.dt, g="allen_cahn", g_param=(1.0, 0.0))
    got = ub.cpu().numpy()
    for j in range(R):
        assert rel_max(got[:, j], us[j].cpu().numpy()) <= TOL
    S.close()


@pytest.mark.parametrize("graph", [False, True])
def test_grouped_solve_batch_matches_ungrouped(graph):
    """Column groups on their own streams (eager, and recorded into a CUDA graph and replayed)
    give the ungrouped result to rounding and the FP64 solve to the mixed tolerance."""
    torch = need_gpu()
    n1, n2, p, R = 16, 8, 12, 13
    g = Grid(n1, n2, p, -0.5, 0.5, 0.0, 1.0)
    coef = workloads.random_coefficients(p, g.N_int)
    S1 = _solver(torch, n1, n2, p, coef, 0.013, (-0.5, 0.5, 0.0, 1.0))
    SG = _solver(torch, n1, n2, p, coef, 0.013, (-0.5, 0.5, 0.0, 1.0))
    S1.batch_reserve(R)
    SG.batch_reserve(R, groups=2)
    if graph:
        SG.set_graph(True)
    r = np.random.default_rng(7)
    rhs = to_dev(torch, r.standard_normal((g.N_int, R)))
    f = to_dev(torch, r.standard_normal((g.boundary_indices().size, R)))
    want = S1.solve_batch(rhs, f, refine=2).cpu().numpy()
    u = torch.zeros((g.N, R), dtype=torch.float64, device="cuda")
    for _ in range(3):  # eager; recorded + replayed; replayed
        u.zero_()
        SG.solve_batch(rhs, f, u=u, refine=2)
        torch.cuda.synchronize()
        got = u.cpu().numpy()
        assert rel_max(got, want) <= 1e-11
        for j in (0, 7, R - 1):
            ref = S1.solve(rhs[:, j].contiguous(), f[:, j].contiguous()).cpu().numpy()
            assert rel_max(got[:, j], ref) <= TOL
    S1.close()
    SG.close()


def _ark_pair(torch, n1, n2, p, R, dt, opt=None, val=None, autotune=False):
    """Two batched ARK steps (Allen-Cahn, constant coefficients: the shared-operator kernels)
    against the FP64 single-column path, column by column."""
    from paper_2306_02526_gb300 import hps
    g = Grid(n1, n2, p)
    X, Y = g.coords()
    bd = g.boundary_indices()
    S = _solver(torch, n1, n2, p, {"a11": 0.02, "a22": 0.02}, 0.25 * dt)
    S.batch_reserve(R)
    tuned = None
    if opt is not None:
        S.batch_option(opt, val)
        assert S.batch_option(opt) == val
    if autotune:
        tuned = S.batch_autotune(R, refine=1)
    u0 = np.stack([0.3 * np.sin(math.pi * (j + 1) * X) * np.sin(math.pi * Y) for j in range(R)], axis=1)
    u0[bd, :] = 0.0
    ub = to_dev(torch, u0)
    us = [to_dev(torch, u0[:, j].copy()) for j in range(R)]
    for n in range(2):
        S.ark_step_batch(ub, n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0), refine=1)
        for j in range(R):
            S.ark_step(us[j], n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0))
    got = ub.cpu().numpy()
    err = max(rel_max(got[:, j], us[j].cpu().numpy()) for j in range(R))
    S.close()
    return err, tuned


@pytest.mark.parametrize("opt,val", [("tensor_leaf", 0), ("even_odd", 0), ("flow_levels", 3), ("flow_levels", 8),
                                     ("cluster_splitk", 1), ("plan_target", 4), ("plan_kmin", 8),
                                     ("plan_npc_max", 1), ("split_rhs", 1), ("fp64_ctas_per_sm", 2),
                                     ("fast_diag", 0), ("last_cta_sum", 16), ("plan_tile_cols", 8),
                                     ("plan_tile_cols", 4), ("plan_tile_cols", 2), ("fuse_epilogue", 0),
                                     ("fuse_jump", 0), ("fold_scale", 0), ("sa_close", 0),
                                     ("edge_projection", 0), ("eo_cols", 5), ("eo_cols", 8),
                                     ("tile_cols_down", 4), ("tile_cols_h", 8), ("sub_levels", 3),
                                     ("sub_levels", 6), ("pdl", 1)])
def test_batch_option_variants_match_fp64(opt, val):
    """Every kernel variant of the batched path (handle options) gives the FP64 result to the
    mixed-precision tolerance; flow_levels = 8 puts every level of the 16 x 8 tree, root
    included, into the dataflow kernels."""
    torch = need_gpu()
    err, _ = _ark_pair(torch, 16, 8, 12, 16, 0.01, opt, val)
    assert err <= TOL, (opt, val, err)


def test_batch_autotune_keeps_a_correct_configuration():
    torch = need_gpu()
    err, tuned = _ark_pair(torch, 16, 16, 12, 16, 0.01, autotune=True)
    assert len(tuned) == 8 and all(t["ms"] > 0 for t in tuned)
    assert err <= TOL


def test_host_buffer_steps_equal_device_steps():
    """ark_step_host / ark_step_batch_host (states in page-locked host memory, copies inside the
    call) give bit for bit the states of ark_step / ark_step_batch on device buffers."""
    torch = need_gpu()
    n1, n2, p, dt, R = 4, 2, 10, 0.02, 6
    g = Grid(n1, n2, p)
    X, Y = g.coords()
    bd = g.boundary_indices()
    S = _solver(torch, n1, n2, p, {"a11": 0.3, "a22": 0.5}, 0.25 * dt)
    S.batch_reserve(R)
    u0 = np.stack([0.2 * np.cos(2 * X + 0.3 * j) * np.sin(4 * Y) for j in range(R)], axis=1)
    u0[bd, :] = 0.0
    ud = to_dev(torch, u0)
    uh = torch.tensor(u0, dtype=torch.float64).pin_memory()
    vd = to_dev(torch, u0[:, 0].copy())
    vh = torch.tensor(u0[:, 0].copy(), dtype=torch.float64).pin_memory()
    for n in range(3):
        S.ark_step_batch(ud, n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0), refine=1)
        S.ark_step_batch_host(uh, n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0), refine=1)
        S.ark_step(vd, n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0))
        S.ark_step_host(vh, n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0))
    torch.cuda.synchronize()
    assert torch.equal(ud.cpu(), uh)
    assert torch.equal(vd.cpu(), vh)
    S.close()
