"""Python binding of libhps.so: the names of include/hps.h over torch device tensors.

PyTorch provides device memory and the current CUDA stream; every step of the solve runs
in the library's CUDA kernels.  Vectors use the library's global ordering (include/hps.h).
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import check, lib

G_KINDS = {None: _lib.HPS_G_NONE, "none": _lib.HPS_G_NONE, "allen_cahn": _lib.HPS_G_ALLEN_CAHN,
           "fisher": _lib.HPS_G_FISHER, "burgers": _lib.HPS_G_BURGERS}
COEF_NAMES = ("a11", "a22", "a1", "a2", "a0")


def _tree(n1, n2, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
    return _lib.hps_tree(int(n1), int(n2), float(x0), float(x1), float(y0), float(y1))


class Tree:
    """n1 x n2 equal leaves on [x0, x1] x [y0, y1] (n1, n2 powers of two)."""

    def __init__(self, n1, n2, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
        self.n1, self.n2, self.x0, self.x1, self.y0, self.y1 = int(n1), int(n2), x0, x1, y0, y1
        self.c = _tree(n1, n2, x0, x1, y0, y1)


def hps_sizes(tree: Tree, p):
    N, Ni, Nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().hps_sizes(ctypes.byref(tree.c), int(p), ctypes.byref(N), ctypes.byref(Ni), ctypes.byref(Nb)),
          "hps_sizes")
    return N.value, Ni.value, Nb.value


def hps_coords(tree: Tree, p):
    N, _, _ = hps_sizes(tree, p)
    x = np.empty(N)
    y = np.empty(N)
    check(lib().hps_coords(ctypes.byref(tree.c), int(p), x.ctypes.data_as(_lib.c_double_p),
                           y.ctypes.data_as(_lib.c_double_p)), "hps_coords")
    return x, y


def hps_boundary_index(tree: Tree, p):
    _, _, Nb = hps_sizes(tree, p)
    idx = np.empty(Nb, dtype=np.int64)
    check(lib().hps_boundary_index(ctypes.byref(tree.c), int(p), idx.ctypes.data_as(_lib.c_int64_p)),
          "hps_boundary_index")
    return idx


def hps_bytes(tree: Tree, p, nodal=False, per_node=False):
    return int(lib().hps_bytes(ctypes.byref(tree.c), int(p), _lib.HPS_COEF_NODAL if nodal else _lib.HPS_COEF_CONST,
                               _lib.HPS_FLAG_PER_NODE if per_node else 0))


def hps_ark_abscissae():
    c = (ctypes.c_double * 6)()
    check(lib().hps_ark_abscissae(c), "hps_ark_abscissae")
    return np.array(list(c))


def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, n, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    if t.numel() != n:
        raise ValueError("%s has %d entries, expected %d" % (name, t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t, n, name):
    """Host pointer of a contiguous float64 CPU tensor (page-locked for asynchronous copies)."""
    import torch
    if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CPU tensor" % name)
    if t.numel() != n:
        raise ValueError("%s has %d entries, expected %d" % (name, t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


class HPSSolver:
    """A built handle: the HPS operators of I - gamma_dt L (plus the identity set).

    coef: dict with a11, a22, a1, a2, a0; all Python scalars -> constant coefficients,
    otherwise float64 CUDA tensors of N_int values (interior order; scalars are broadcast).
    """

    def __init__(self, tree: Tree, p, coef, gamma_dt, per_node=False, stream=None):
        import torch
        self.tree, self.p, self.gamma_dt = tree, int(p), float(gamma_dt)
        self.N, self.N_int, self.N_bd = hps_sizes(tree, p)
        nodal = any(isinstance(coef.get(k, 0.0), torch.Tensor) for k in COEF_NAMES)
        c = _lib.hps_coeffs()
        keep = []
        if nodal:
            c.kind = _lib.HPS_COEF_NODAL
            for k in COEF_NAMES:
                v = coef.get(k, 0.0)
                if not isinstance(v, torch.Tensor):
                    v = torch.full((self.N_int,), float(v), dtype=torch.float64, device="cuda")
                v = v.to(device="cuda", dtype=torch.float64).contiguous()
                keep.append(v)
                setattr(c, k, _dptr(v, self.N_int, k))
        else:
            c.kind = _lib.HPS_COEF_CONST
            for k in COEF_NAMES:
                setattr(c, "c_" + k, float(coef.get(k, 0.0)))
        self.nodal = nodal
        h = ctypes.c_void_p()
        check(lib().hps_build(ctypes.byref(tree.c), self.p, ctypes.byref(c), self.gamma_dt,
                              _lib.HPS_FLAG_PER_NODE if per_node else 0, _stream_ptr(stream), ctypes.byref(h)),
              "hps_build")
        self._h = h
        del keep

    def close(self):
        if getattr(self, "_h", None):
            lib().hps_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_graph(self, enable=True):
        """Record ark_step / hps_solve into CUDA graphs and replay them (hps_set_graph)."""
        check(lib().hps_set_graph(self._h, 1 if enable else 0), "hps_set_graph")

    def set_persistent(self, enable=True):
        """All merge levels in one persistent kernel per direction (default) or one launch per level."""
        check(lib().hps_set_persistent(self._h, 1 if enable else 0), "hps_set_persistent")

    def trace_tasks(self, enable=None):
        """enable True/False: start/stop per-task stamping; None: (up_us, down_us) of the last sweep."""
        if enable is not None:
            check(lib().hps_trace_tasks(self._h, 1 if enable else 0, 0, None, 0), "hps_trace_tasks")
            return None
        out = []
        for up in (1, 0):
            buf = (ctypes.c_double * 64)()
            n = lib().hps_trace_tasks(self._h, -1, up, buf, 64)
            if n < 0:
                check(n, "hps_trace_tasks")
            out.append(list(buf)[:n])
        return tuple(out)

    def status(self, stream=None):
        """Raise HPSError if a bounded device wait ran out since the last check (hps_status)."""
        check(lib().hps_status(self._h, _stream_ptr(stream)), "hps_status")

    def trace_enable(self, kernels=()):
        """Reset the per-kernel counters; time the named kernels (see _lib.KERNELS) with CUDA events."""
        mask = 0
        for k in kernels:
            mask |= 1 << _lib.KERNELS.index(k)
        check(lib().hps_trace_enable(self._h, mask), "hps_trace_enable")

    def trace_read(self):
        """{kernel: (launches, launches timed, total ms)} since the last trace_enable."""
        out = {}
        for i, name in enumerate(_lib.KERNELS):
            n, nt, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
            check(lib().hps_trace_read(self._h, i, ctypes.byref(n), ctypes.byref(nt), ctypes.byref(ms)),
                  "hps_trace_read")
            out[name] = (n.value, nt.value, ms.value)
        return out

    def solve(self, rhs, f=None, u=None, stream=None):
        """u (length N) solving (I - gamma_dt L) u = rhs, u = f on the boundary (hps_solve)."""
        import torch
        if u is None:
            u = torch.empty(self.N, dtype=torch.float64, device="cuda")
        check(lib().hps_solve(self._h, _dptr(rhs, self.N_int, "rhs"), _dptr(f, self.N_bd, "f"),
                              _dptr(u, self.N, "u"), _stream_ptr(stream)), "hps_solve")
        return u

    def ark_step(self, u, t, dt, q=None, f=None, g=None, g_param=(1.0, 1.0), stream=None):
        """One ARK4(3)6L[2]SA step in place on u (ark_step).  q: (6, N_int) stage sources or
        None; f: (6, N_bd) stage boundary data or None; g: None, 'allen_cahn', 'fisher', 'burgers',
        or a callable g(u_j, g_out) (HPS_G_USER) on CUDA tensors -- the stage value (N,) and
        g(u_j) at the interior points (N_int,), to be written in place -- that runs with the
        step's stream as torch's current stream.  With graphs on (set_graph) the step is recorded
        with the callable's work and replayed without calling it again: it must then do the same
        work each time and allocate nothing (out= forms into tensors made beforehand)."""
        terms = _lib.hps_ark_terms()
        terms.q = _dptr(q, 6 * self.N_int, "q")
        terms.f = _dptr(f, 6 * self.N_bd, "f")
        if callable(g):
            terms.g_kind = _lib.HPS_G_USER
            terms.g_fn = ctypes.cast(self._g_hook(g), ctypes.c_void_p)
        else:
            terms.g_kind = G_KINDS[g]
            terms.g_param[0], terms.g_param[1] = float(g_param[0]), float(g_param[1])
        rc = lib().ark_step(self._h, _dptr(u, self.N, "u"), float(t), float(dt), ctypes.byref(terms),
                            _stream_ptr(stream))
        errs = self.__dict__.setdefault("_hook_errors", [])
        if errs:
            e = errs[0]
            errs.clear()
            raise e
        check(rc, "ark_step")
        return u

    def _g_hook(self, fn):
        """The C hook of a Python g, one per callable (a stable pointer: graph replays match it)."""
        hooks = self.__dict__.setdefault("_g_hooks", {})
        if id(fn) not in hooks:
            N, Ni, errs = self.N, self.N_int, self.__dict__.setdefault("_hook_errors", [])

            def call(user, u, gout, stream):
                try:
                    import torch
                    ut = torch.as_tensor(DeviceArray(u, (N,)), device="cuda")
                    gt = torch.as_tensor(DeviceArray(gout, (Ni,)), device="cuda")
                    with torch.cuda.stream(_torch_stream(stream)):
                        fn(ut, gt)
                    return 0
                except Exception as e:  # the step returns an error; ark_step raises this
                    errs.append(e)
                    return _lib.HPS_EINVAL
            hooks[id(fn)] = (fn, _lib.G_FN(call))
        return hooks[id(fn)][1]

    def ark_slope_step(self, u, t, dt, q=None, kbc=None, g=None, g_param=(1.0, 1.0), stream=None):
        """One ARK step in slope form (ark_slope_step) in place on u: q (6, N_int) stage sources or
        None; kbc (6, N_bd) slope boundary data (u_t at the stage times) or None (zero); g a preset
        (then kbc must be None: time-independent boundary data)."""
        terms = _lib.hps_ark_terms()
        terms.q = _dptr(q, 6 * self.N_int, "q")
        terms.f = _dptr(kbc, 6 * self.N_bd, "kbc")
        terms.g_kind = G_KINDS[g]
        terms.g_param[0], terms.g_param[1] = float(g_param[0]), float(g_param[1])
        check(lib().ark_slope_step(self._h, _dptr(u, self.N, "u"), float(t), float(dt), ctypes.byref(terms),
                                   _stream_ptr(stream)), "ark_slope_step")
        return u

    def ark_step_host(self, u_host, t, dt, q=None, f=None, g=None, g_param=(1.0, 1.0), stream=None):
        """ark_step on a state in host memory (ark_step_host): u_host is a float64 CPU tensor of
        N entries (pin_memory() for asynchronous copies), updated once the stream is done; q, f
        on the device as for ark_step."""
        terms = _lib.hps_ark_terms()
        terms.q = _dptr(q, 6 * self.N_int, "q")
        terms.f = _dptr(f, 6 * self.N_bd, "f")
        terms.g_kind = G_KINDS[g]
        terms.g_param[0], terms.g_param[1] = float(g_param[0]), float(g_param[1])
        check(lib().ark_step_host(self._h, _hptr(u_host, self.N, "u_host"), float(t), float(dt), ctypes.byref(terms),
                                  _stream_ptr(stream)), "ark_step_host")
        return u_host

    # ---- batched mixed precision -----------------------------------------------------------
    def batch_reserve(self, R, groups=None):
        """FP32 operator copies and R-column work buffers (hps_batch_reserve); with `groups`,
        the columns of later calls run as that many column groups on their own streams
        (hps_batch_reserve_groups)."""
        if groups is None:
            check(lib().hps_batch_reserve(self._h, int(R)), "hps_batch_reserve")
        else:
            check(lib().hps_batch_reserve_groups(self._h, int(R), int(groups)), "hps_batch_reserve_groups")

    def batch_option(self, name, value=None):
        """Get (value None) or set a kernel option of the batched path (hps_batch_get/set_option;
        the step-close option edge_projection applies to the FP64 ark_step too); names
        in _lib.BATCH_OPTIONS."""
        opt = _lib.BATCH_OPTIONS.index(name)
        if value is not None:
            check(lib().hps_batch_set_option(self._h, opt, int(value)), "hps_batch_set_option")
        out = ctypes.c_int()
        check(lib().hps_batch_get_option(self._h, opt, ctypes.byref(out)), "hps_batch_get_option")
        return out.value

    def batch_autotune(self, R, refine=1, stream=None):
        """Time the candidate kernel configurations on this operator, keep the fastest
        (hps_batch_autotune); returns one dict per candidate."""
        res = (_lib.hps_tune_result * 32)()
        n = ctypes.c_int()
        check(lib().hps_batch_autotune(self._h, int(R), int(refine), _stream_ptr(stream), res, 32, ctypes.byref(n)),
              "hps_batch_autotune")
        return [{"tile_cols": r.tile_cols, "flow_levels": r.flow_levels, "plan_target": r.plan_target,
                 "plan_kmin": r.plan_kmin, "ms": r.ms} for r in res[:n.value]]

    def solve_batch(self, rhs, f=None, u=None, refine=2, stream=None):
        """R solves at once: rhs (N_int, R), f (N_bd, R) or None -> u (N, R) (hps_solve_batch)."""
        import torch
        R = rhs.shape[1]
        if u is None:
            u = torch.empty((self.N, R), dtype=torch.float64, device="cuda")
        check(lib().hps_solve_batch(self._h, R, _dptr(rhs, self.N_int * R, "rhs"), _dptr(f, self.N_bd * R, "f"),
                                    _dptr(u, self.N * R, "u"), int(refine), _stream_ptr(stream)), "hps_solve_batch")
        return u

    def ark_step_batch(self, u, t, dt, q=None, f=None, g=None, g_param=(1.0, 1.0), refine=2, stream=None):
        """ARK step on R states u (N, R) in place (ark_step_batch); q (6, N_int, R), f (6, N_bd, R)."""
        R = u.shape[1]
        terms = _lib.hps_ark_terms()
        terms.q = _dptr(q, 6 * self.N_int * R, "q")
        terms.f = _dptr(f, 6 * self.N_bd * R, "f")
        terms.g_kind = G_KINDS[g]
        terms.g_param[0], terms.g_param[1] = float(g_param[0]), float(g_param[1])
        check(lib().ark_step_batch(self._h, R, _dptr(u, self.N * R, "u"), float(t), float(dt), ctypes.byref(terms),
                                   int(refine), _stream_ptr(stream)), "ark_step_batch")
        return u

    def ark_slope_step_batch(self, u, t, dt, q=None, kbc=None, g=None, g_param=(1.0, 1.0), refine=2, stream=None):
        """ark_slope_step on R states u (N, R) in place, mixed precision (ark_slope_step_batch):
        q (6, N_int, R) stage sources, kbc (6, N_bd, R) slope boundary data (u_t), or None; g a
        preset (then kbc must be None)."""
        R = u.shape[1]
        terms = _lib.hps_ark_terms()
        terms.q = _dptr(q, 6 * self.N_int * R, "q")
        terms.f = _dptr(kbc, 6 * self.N_bd * R, "kbc")
        terms.g_kind = G_KINDS[g]
        terms.g_param[0], terms.g_param[1] = float(g_param[0]), float(g_param[1])
        check(lib().ark_slope_step_batch(self._h, R, _dptr(u, self.N * R, "u"), float(t), float(dt),
                                         ctypes.byref(terms), int(refine), _stream_ptr(stream)), "ark_slope_step_batch")
        return u

    def ark_step_batch_host(self, u_host, t, dt, q=None, f=None, g=None, g_param=(1.0, 1.0), refine=2, stream=None):
        """ark_step_batch on R states in host memory (ark_step_batch_host): u_host (N, R) float64
        CPU tensor (pin_memory() for asynchronous copies), updated once the stream is done."""
        R = u_host.shape[1]
        terms = _lib.hps_ark_terms()
        terms.q = _dptr(q, 6 * self.N_int * R, "q")
        terms.f = _dptr(f, 6 * self.N_bd * R, "f")
        terms.g_kind = G_KINDS[g]
        terms.g_param[0], terms.g_param[1] = float(g_param[0]), float(g_param[1])
        check(lib().ark_step_batch_host(self._h, R, _hptr(u_host, self.N * R, "u_host"), float(t), float(dt),
                                        ctypes.byref(terms), int(refine), _stream_ptr(stream)), "ark_step_batch_host")
        return u_host


class MultiStep:
    """Several independent instances (HPSSolver objects, each reserved for its column count)
    advanced together by one batched ARK step each per call, concurrently (hps_multi_*)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        h = ctypes.c_void_p()
        check(lib().hps_multi_create(arr, len(self.solvers), ctypes.byref(h)), "hps_multi_create")
        self._h = h

    def set_graph(self, enable=True):
        check(lib().hps_multi_set_graph(self._h, 1 if enable else 0), "hps_multi_set_graph")

    def set_lockstep(self, enable=True):
        """One grouped merge launch per tree level for all instances (every solver with one
        column group)."""
        check(lib().hps_multi_set_lockstep(self._h, 1 if enable else 0), "hps_multi_set_lockstep")

    def ark_step(self, us, dt, g=None, g_param=(1.0, 1.0), refine=1, stream=None):
        """us: one (N_i, R_i) float64 CUDA tensor per instance, advanced in place."""
        n = len(self.solvers)
        if len(us) != n:
            raise ValueError("expected %d states" % n)
        up = (ctypes.c_void_p * n)(*[_dptr(u, s.N * u.shape[1], "u").value for u, s in zip(us, self.solvers)])
        R = (ctypes.c_int * n)(*[int(u.shape[1]) for u in us])
        terms = (_lib.hps_ark_terms * n)()
        for t in terms:
            t.q = None
            t.f = None
            t.g_kind = G_KINDS[g]
            t.g_param[0], t.g_param[1] = float(g_param[0]), float(g_param[1])
        check(lib().hps_multi_ark_step(self._h, up, R, ctypes.cast(terms, ctypes.c_void_p), float(dt), int(refine),
                                       _stream_ptr(stream)), "hps_multi_ark_step")
        return us

    def close(self):
        if getattr(self, "_h", None):
            lib().hps_multi_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _torch_stream(ptr):
    """torch's view of a CUDA stream handed over by the library (NULL: the legacy default stream)."""
    import torch
    return torch.cuda.ExternalStream(ptr) if ptr else torch.cuda.default_stream()


class DeviceArray:
    """A device buffer of float64 seen through the CUDA array interface (no copy)."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}
