"""Served jobs with nodal (variable) coefficients and with sources q and boundary data f filled
by a per-step callback (hps_job_desc.a11 .. a0, .terms).

Manufactured solution u*(x, y, t) = e^{-t} sin(pi x) sin(pi y) + (1 + t) x y on [0, 1]^2 with
smooth variable coefficients and Fisher's g: q = u*_t - L u* - g(u*) at the interior points and
f = u* on the boundary, both at the stage times t + c_j dt (eq. stage2).  A served job must equal
the direct ark_step with the same q and f arrays bit for bit (per-job FP64 path), be close to
u*(T) (a q or f taken at a wrong stage time misses by O(dt)), share the factorization of another
job whose coefficient arrays hold the same values, and in batched serving agree with its FP64
served result to the mixed-precision tolerance."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_max, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-10
KAPPA = 0.5


def _coef_fns(x, y):
    return {"a11": 1.0 + 0.3 * np.sin(x + 0.5 * y), "a22": 0.8 + 0.2 * y * y, "a1": 0.1 * x,
            "a2": -0.2 + 0.0 * x, "a0": -0.5 + 0.1 * np.cos(y)}


def _exact(x, y, t, amp):
    s = np.sin(np.pi * x) * np.sin(np.pi * y)
    return amp * (np.exp(-t) * s + (1.0 + t) * x * y)


def _source(x, y, t, amp):
    """u*_t - L u* - kappa u* (1 - u*) at points (x, y)."""
    e = np.exp(-t)
    sx, cx, sy, cy = np.sin(np.pi * x), np.cos(np.pi * x), np.sin(np.pi * y), np.cos(np.pi * y)
    u = amp * (e * sx * sy + (1.0 + t) * x * y)
    ut = amp * (-e * sx * sy + x * y)
    ux = amp * (e * np.pi * cx * sy + (1.0 + t) * y)
    uy = amp * (e * np.pi * sx * cy + (1.0 + t) * x)
    uxx = amp * (-e * np.pi ** 2 * sx * sy)
    uyy = uxx
    c = _coef_fns(x, y)
    Lu = c["a11"] * uxx + c["a22"] * uyy + c["a1"] * ux + c["a2"] * uy + c["a0"] * u
    return ut - Lu - KAPPA * u * (1.0 - u)


class _Problem:
    def __init__(self, n1, n2, p, amp):
        from paper_2306_02526_gb300 import hps
        self.tree = hps.Tree(n1, n2)
        self.p = p
        self.amp = amp
        self.N, self.N_int, self.N_bd = hps.hps_sizes(self.tree, p)
        self.x, self.y = hps.hps_coords(self.tree, p)
        self.bd = hps.hps_boundary_index(self.tree, p)
        self.c = hps.hps_ark_abscissae()
        xi, yi = self.x[: self.N_int], self.y[: self.N_int]
        self.coef = _coef_fns(xi, yi)

    def arrays(self, t, dt):
        """q (6, N_int) and f (6, N_bd) of the step that starts at t."""
        xi, yi = self.x[: self.N_int], self.y[: self.N_int]
        xb, yb = self.x[self.bd], self.y[self.bd]
        q = np.stack([_source(xi, yi, t + cj * dt, self.amp) for cj in self.c])
        f = np.stack([_exact(xb, yb, t + cj * dt, self.amp) for cj in self.c])
        return q, f

    def fill(self, t, dt, q, f):  # the serving callback: torch copies on the job's stream
        import torch
        qa, fa = self.arrays(t, dt)
        q.copy_(torch.from_numpy(qa))
        f.copy_(torch.from_numpy(fa))

    def u0(self, t0):
        return _exact(self.x, self.y, t0, self.amp)

    def job(self, dt, steps, t0=0.0, arrival_s=0.0, coef=None):
        return dict(tree=self.tree, p=self.p, coef=self.coef if coef is None else coef, dt=dt, steps=steps,
                    u0=self.u0(t0), g="fisher", g_param=(KAPPA, 0.0), t0=t0, arrival_s=arrival_s, terms=self.fill)


def _serve(jobs, batch_cols=0, refine=-1):
    from paper_2306_02526_gb300.serve import Server
    S = Server(16 << 30, 8, batch_cols=batch_cols, refine=refine)
    ids = [S.submit(**j) for j in jobs]
    S.run()
    res = [S.result(i).copy() for i in ids]
    stats = [S.job_stats(i) for i in ids]
    summ = S.summary()
    S.close()
    return res, stats, summ


def _direct(torch, P, dt, steps, t0=0.0):
    from paper_2306_02526_gb300 import hps
    S = hps.HPSSolver(P.tree, P.p, {k: to_dev(torch, v) for k, v in P.coef.items()}, 0.25 * dt)
    u = to_dev(torch, P.u0(t0))
    for n in range(steps):
        qa, fa = P.arrays(t0 + n * dt, dt)
        S.ark_step(u, t0 + n * dt, dt, q=to_dev(torch, qa), f=to_dev(torch, fa), g="fisher", g_param=(KAPPA, 0.0))
    out = u.cpu().numpy()
    S.close()
    return out


def test_served_nodal_job_with_terms_equals_direct_and_manufactured():
    torch = need_gpu()
    P = _Problem(8, 8, 12, 1.0)
    dt, steps = 0.01, 10
    res, stats, summ = _serve([P.job(dt, steps, t0=0.2)])
    assert stats[0]["state"] == 2 and stats[0]["status"] == 0 and stats[0]["steps_done"] == steps
    assert np.array_equal(res[0], _direct(torch, P, dt, steps, t0=0.2))
    exact = _exact(P.x, P.y, 0.2 + steps * dt, 1.0)
    assert rel_max(res[0], exact) < 1e-6, rel_max(res[0], exact)


def test_equal_coefficient_arrays_share_a_factorization():
    need_gpu()
    P = _Problem(8, 4, 10, 1.0)
    copy = {k: np.array(v, copy=True) for k, v in P.coef.items()}  # other arrays, same values
    other = dict(copy, a0=copy["a0"] + 1e-3)                         # a different operator
    jobs = [P.job(0.01, 6), P.job(0.01, 6, arrival_s=0.02, coef=copy), P.job(0.01, 6, arrival_s=0.03, coef=other)]
    res, stats, summ = _serve(jobs)
    assert [s["state"] for s in stats] == [2, 2, 2]
    assert stats[1]["shared_operators"] == 1 and stats[2]["shared_operators"] == 0
    assert summ["factorizations_built"] == 2
    assert np.array_equal(res[0], res[1])
    assert not np.array_equal(res[0], res[2])


def test_batched_nodal_jobs_with_terms_match_fp64_served():
    """Three jobs of one nodal operation with terms (different amplitudes and start times) share a
    batch; a job of the same operator without terms runs in a batch of its own."""
    need_gpu()
    P = [_Problem(16, 8, 10, a) for a in (1.0, 0.5, 2.0)]
    jobs = [P[0].job(0.005, 12), P[1].job(0.005, 8, t0=0.1, arrival_s=0.01), P[2].job(0.005, 10, t0=0.3,
                                                                                         arrival_s=0.02)]
    plain = dict(P[0].job(0.005, 6, arrival_s=0.005), terms=None)
    plain["u0"] = plain["u0"].copy()
    plain["u0"][P[0].bd] = 0.0
    jobs.append(plain)
    ref, ref_stats, _ = _serve(jobs)
    got, stats, summ = _serve(jobs, batch_cols=8)
    assert all(s["state"] == 2 and s["status"] == 0 for s in stats)
    assert summ["batches_formed"] == 2 and summ["mean_batch_cols"] > 1.5
    for a, b, j in zip(got, ref, jobs):
        assert rel_max(a, b) <= TOL
    for k in range(3):  # and near the manufactured solution
        T = jobs[k]["t0"] + jobs[k]["steps"] * jobs[k]["dt"]
        assert rel_max(got[k], _exact(P[k].x, P[k].y, T, P[k].amp)) < 1e-6


def test_failing_terms_callback_ends_the_job():
    need_gpu()
    from paper_2306_02526_gb300.serve import Server
    P = _Problem(4, 4, 8, 1.0)
    calls = []

    def bad(t, dt, q, f):
        calls.append(t)
        if len(calls) == 3:
            raise RuntimeError("source unavailable")
        P.fill(t, dt, q, f)

    S = Server(4 << 30, 4)
    jid = S.submit(**dict(P.job(0.01, 8), terms=bad))
    with pytest.raises(RuntimeError):
        S.run()
    st = S.job_stats(jid)
    S.close()
    assert st["state"] == 2 and st["status"] != 0 and st["steps_done"] == 2
