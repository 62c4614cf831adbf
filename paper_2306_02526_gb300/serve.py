"""Python binding of the serving loop (hps_server_* in include/hps.h).

Jobs carry host arrays (numpy float64) for their initial and final states; the loop itself
runs natively (admission by device memory, one CUDA stream per job or per batch, graph-replayed
steps).  batch_cols > 0 coalesces jobs of the same operation into batched mixed-precision steps
(hps_server_set_batching).

Jobs may carry nodal coefficients (host arrays at the interior points) and a `terms` callable
(t, dt, q, f) that fills the step's sources q (6 x N_int) and boundary data f (6 x N_bd), given as
CUDA tensors, for the stage times t + c_j dt; it runs with the job's CUDA stream as torch's
current stream, so its tensor operations are ordered before the step."""
import ctypes

import numpy as np

from . import _lib
from ._lib import check, lib
from .hps import G_KINDS, DeviceArray, Tree, _torch_stream, hps_sizes


class Server:
    def __init__(self, mem_budget_bytes, max_active=8, batch_cols=0, refine=-1):
        h = ctypes.c_void_p()
        check(lib().hps_server_create(int(mem_budget_bytes), int(max_active), ctypes.byref(h)), "hps_server_create")
        self._h = h
        if batch_cols:
            check(lib().hps_server_set_batching(h, int(batch_cols), int(refine)), "hps_server_set_batching")
        self._keep = []
        self._errors = []
        self.jobs = []

    def submit(self, tree: Tree, p, coef, dt, steps, u0, g=None, g_param=(1.0, 1.0), t0=0.0, arrival_s=0.0,
               terms=None):
        """Queue a job; returns its id.  coef: dict of a11, a22, a1, a2, a0, all constants or
        (nodal) arrays of N_int values at the interior points, a missing one zero.  terms: None
        (q = 0, f = 0) or a callable (t, dt, q, f) filling the CUDA tensors q (6, N_int) and
        f (6, N_bd) in place with q(t + c_j dt) and f(t + c_j dt), j = 1..6."""
        N, N_int, N_bd = hps_sizes(tree, p)
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        if u0.size != N:
            raise ValueError("u0 has %d entries, expected %d" % (u0.size, N))
        out = np.empty(N)
        d = _lib.hps_job_desc()
        d.tree = tree.c
        d.p = int(p)
        keep = [u0, out]
        if any(np.ndim(v) for v in coef.values()):
            for k in ("a11", "a22", "a1", "a2", "a0"):
                if k in coef:
                    a = np.ascontiguousarray(np.broadcast_to(np.asarray(coef[k], dtype=np.float64), (N_int,)))
                    keep.append(a)
                    setattr(d, k, a.ctypes.data)
        else:
            for k in ("a11", "a22", "a1", "a2", "a0"):
                setattr(d, "c_" + k, float(coef.get(k, 0.0)))
        if terms is not None:
            cb = _lib.TERMS_FN(self._terms_callback(terms, N_int, N_bd))
            keep.append(cb)
            d.terms = ctypes.cast(cb, ctypes.c_void_p)
        d.dt, d.t0, d.steps = float(dt), float(t0), int(steps)
        d.g_kind = G_KINDS[g]
        d.g_param[0], d.g_param[1] = float(g_param[0]), float(g_param[1])
        d.u0 = u0.ctypes.data_as(ctypes.c_void_p)
        d.u_out = out.ctypes.data_as(ctypes.c_void_p)
        d.arrival_s = float(arrival_s)
        jid = ctypes.c_int()
        check(lib().hps_server_submit(self._h, ctypes.byref(d), ctypes.byref(jid)), "hps_server_submit")
        self._keep.append(keep)
        self.jobs.append(out)
        return jid.value

    def _terms_callback(self, fn, N_int, N_bd):
        def call(user, t, dt, q, f, stream):
            try:
                import torch
                qt = torch.as_tensor(DeviceArray(q, (6, N_int)), device="cuda")
                ft = torch.as_tensor(DeviceArray(f, (6, N_bd)), device="cuda")
                with torch.cuda.stream(_torch_stream(stream)):
                    fn(t, dt, qt, ft)
                return 0
            except Exception as e:  # the job ends with this status; the exception is raised by run()
                self._errors.append(e)
                return _lib.HPS_EINVAL
        return call

    def evict_after(self, job_id, steps):
        """Checkpoint job `job_id` to host memory after `steps` steps, release it, queue it again."""
        check(lib().hps_server_evict_after(self._h, int(job_id), int(steps)), "hps_server_evict_after")

    def run(self):
        self._errors = getattr(self, "_errors", [])
        rc = lib().hps_server_run(self._h)
        if self._errors:
            raise self._errors[0]
        check(rc, "hps_server_run")

    def result(self, job_id):
        return self.jobs[job_id]

    def job_stats(self, job_id):
        s = _lib.hps_job_stats()
        check(lib().hps_server_job_stats(self._h, int(job_id), ctypes.byref(s)), "hps_server_job_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def summary(self):
        s = _lib.hps_server_stats()
        check(lib().hps_server_summary(self._h, ctypes.byref(s)), "hps_server_summary")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().hps_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

