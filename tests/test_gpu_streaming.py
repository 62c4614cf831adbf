"""The HBM-bound form of the batched path: one to four right-hand sides with per-node operators
(nodal coefficients).  Its kernels -- leaf applies streamed by bulk copies through persistent
CTAs (option stream_leaf, with or without the per-leaf register loads and fused one-column sums of
stream_prefetch), one-column merge applies (one_column_merge) with in-kernel split-K sums
(one_column_sum) -- and the general kernels they replace must all give the FP64 result after
refinement (1e-10 relative max-norm) and agree with each other in the FP32 sweep alone."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev
from oracle.grid import Grid
from oracle.hps import HPS
from paper_2306_02526_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10
VARIANTS = [dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1),
            dict(stream_leaf=1, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1),
            dict(stream_leaf=4, stream_chunk_kb=8, one_column_merge=1, one_column_sum=1),
            dict(stream_leaf=2, stream_chunk_kb=64, one_column_merge=1, one_column_sum=1),
            dict(stream_leaf=0, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=0),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=0, one_column_sum=0),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1, pdl=1),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1, eo_threads=256),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1, eo_threads=64),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1, prefetch_next=1),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=0, one_column_sum=0, prefetch_next=1),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1, b1_roll=1),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1, b1_roll=1, b1_kw=2),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=0, b1_roll=0, b1_kw=1),
            dict(stream_leaf=3, stream_chunk_kb=24, one_column_merge=1, one_column_sum=1, stream_prefetch=0),
            dict(stream_leaf=4, stream_chunk_kb=8, one_column_merge=1, one_column_sum=1, stream_prefetch=1),
            dict(stream_leaf=1, stream_chunk_kb=64, one_column_merge=1, one_column_sum=1, stream_prefetch=1)]


def _nodal_solver(torch, n1, n2, p, gdt, seed=0):
    from paper_2306_02526_gb300 import hps
    g = Grid(n1, n2, p)
    coef = workloads.random_coefficients(seed, g.N_int)
    S = hps.HPSSolver(hps.Tree(n1, n2), p, {k: to_dev(torch, v) for k, v in coef.items()}, gdt)
    return g, coef, S


def _set(S, opts):
    for k, v in opts.items():
        S.batch_option(k, v)
        assert S.batch_option(k) == v


@pytest.mark.parametrize("n1,n2,p,R", [(16, 16, 12, 1), (16, 16, 12, 2), (32, 8, 16, 4), (4, 2, 9, 3),
                                       (1, 1, 6, 1), (2, 2, 32, 1)])
def test_streaming_variants_match_fp64(n1, n2, p, R):
    """(16, 16): 256 leaves, more than one per persistent CTA; (32, 8, 16): q = 196, several
    chunks per leaf operator and a partial last chunk; (2, 2, 32): the largest p, q = 900 rows
    on one K slice, 4 operator columns per chunk."""
    torch = need_gpu()
    g, coef, S = _nodal_solver(torch, n1, n2, p, 0.011, seed=n1 + p)
    S.batch_reserve(R)
    r = np.random.default_rng(7 * R + p)
    rhs = to_dev(torch, r.standard_normal((g.N_int, R)))
    f = to_dev(torch, r.standard_normal((g.boundary_indices().size, R)))
    want = np.stack([S.solve(rhs[:, j].contiguous(), f[:, j].contiguous()).cpu().numpy() for j in range(R)], axis=1)
    sweeps = []
    for opts in VARIANTS:
        _set(S, opts)
        u0 = S.solve_batch(rhs, f, refine=0).cpu().numpy()
        u2 = S.solve_batch(rhs, f, refine=2).cpu().numpy()
        assert rel_max(u0, want) < 1e-4, opts
        assert rel_max(u2, want) <= TOL, (opts, rel_max(u2, want))
        sweeps.append(u0)
    for u0 in sweeps[1:]:  # the FP32 sweeps differ only in the order of their FP32 sums
        assert rel_max(u0, sweeps[0]) < 1e-5
    S.status()
    if g.N <= 3000:
        ref = HPS(g, coef, 0.011).solve(rhs[:, 0].cpu().numpy(), f[:, 0].cpu().numpy())
        assert rel_max(S.solve_batch(rhs, f, refine=2).cpu().numpy()[:, 0], ref) <= TOL
    S.close()


@pytest.mark.parametrize("stream_leaf", [3, 0])
def test_streaming_ark_step_batch_matches_fp64(stream_leaf):
    """ark_step_batch with 3 states on per-node operators (stage right-hand sides of several
    terms in the streaming particular solve, Allen-Cahn epilogue) against ark_step."""
    torch = need_gpu()
    dt = 0.01
    g, coef, S = _nodal_solver(torch, 16, 8, 10, 0.25 * dt, seed=3)
    S.batch_reserve(3)
    S.batch_option("stream_leaf", stream_leaf)
    X, Y = g.coords()
    bd = g.boundary_indices()
    u0 = np.stack([0.3 * np.sin(np.pi * (j + 1) * X) * np.sin(np.pi * Y) for j in range(3)], axis=1)
    u0[bd, :] = 0.0
    ub = to_dev(torch, u0)
    us = [to_dev(torch, u0[:, j].copy()) for j in range(3)]
    for n in range(3):
        S.ark_step_batch(ub, n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0), refine=2)
        for j in range(3):
            S.ark_step(us[j], n * dt, dt, g="allen_cahn", g_param=(1.0, 0.0))
    got = ub.cpu().numpy()
    for j in range(3):
        assert rel_max(got[:, j], us[j].cpu().numpy()) <= TOL
    S.status()
    S.close()


def test_streaming_single_rhs_full_size():
    """The single-right-hand-side sweep at full size (128 x 128 leaves, p = 16, variable
    coefficients, 16,384 per-leaf operators streamed): one refinement sweep, as timed, against
    the FP64 solve; replayed from a CUDA graph it gives the same values."""
    torch = need_gpu()
    from paper_2306_02526_gb300 import hps
    wl = workloads.VarCoef128()
    tree = hps.Tree(wl.n1, wl.n2)
    N, N_int, N_bd = hps.hps_sizes(tree, wl.p)
    x, y = hps.hps_coords(tree, wl.p)
    I = np.arange(N_int)
    S = hps.HPSSolver(tree, wl.p, {k: to_dev(torch, v) for k, v in wl.coef(x[I], y[I]).items()}, 0.25 * wl.dt)
    S.batch_reserve(1)
    rhs = to_dev(torch, np.random.default_rng(11).uniform(-0.1, 0.1, (N_int, 1)))
    want = S.solve(rhs[:, 0].contiguous())
    u = torch.empty((N, 1), dtype=torch.float64, device="cuda")
    S.solve_batch(rhs, u=u, refine=1)
    eager = u.clone()
    assert float((u[:, 0] - want).abs().max() / want.abs().max()) <= TOL
    S.set_graph(True)
    for _ in range(3):
        S.solve_batch(rhs, u=u, refine=1)
    assert torch.equal(u, eager)
    S.status()
    S.close()
