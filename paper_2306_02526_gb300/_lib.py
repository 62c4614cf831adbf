"""ctypes declarations of the C ABI in include/hps.h (argument marshalling only)."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhps.so")

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int64_p = ctypes.POINTER(ctypes.c_int64)

HPS_OK, HPS_EINVAL, HPS_ENOMEM, HPS_ESINGULAR, HPS_ETIMEOUT, HPS_ECUDA, HPS_EDT, HPS_ESCRATCH = 0, -1, -2, -3, -4, -5, -6, -7
HPS_COEF_CONST, HPS_COEF_NODAL = 0, 1
HPS_FLAG_PER_NODE = 1
HPS_G_NONE, HPS_G_ALLEN_CAHN, HPS_G_FISHER, HPS_G_BURGERS, HPS_G_USER = 0, 1, 2, 3, 4
KERNELS = ("leaf_up", "merge_up_w3", "merge_up_h", "merge_down", "leaf_down", "leaf_eval", "set_boundary",
           "merge_up_all", "merge_down_all", "residual", "jump", "finish", "close")


class hps_tree(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double)]


class hps_coeffs(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("c_a11", ctypes.c_double), ("c_a22", ctypes.c_double),
                ("c_a1", ctypes.c_double), ("c_a2", ctypes.c_double), ("c_a0", ctypes.c_double),
                ("a11", ctypes.c_void_p), ("a22", ctypes.c_void_p), ("a1", ctypes.c_void_p),
                ("a2", ctypes.c_void_p), ("a0", ctypes.c_void_p)]


class hps_ark_terms(ctypes.Structure):
    _fields_ = [("q", ctypes.c_void_p), ("f", ctypes.c_void_p), ("g_kind", ctypes.c_int),
                ("g_param", ctypes.c_double * 2), ("g_fn", ctypes.c_void_p), ("g_user", ctypes.c_void_p)]


# int (*)(void *user, const double *u, double *g_out, hps_stream_t stream)
G_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class hps_job_desc(ctypes.Structure):
    _fields_ = [("tree", hps_tree), ("p", ctypes.c_int), ("c_a11", ctypes.c_double), ("c_a22", ctypes.c_double),
                ("c_a1", ctypes.c_double), ("c_a2", ctypes.c_double), ("c_a0", ctypes.c_double),
                ("dt", ctypes.c_double), ("t0", ctypes.c_double), ("steps", ctypes.c_int), ("g_kind", ctypes.c_int),
                ("g_param", ctypes.c_double * 2), ("u0", ctypes.c_void_p), ("u_out", ctypes.c_void_p),
                ("arrival_s", ctypes.c_double), ("a11", ctypes.c_void_p), ("a22", ctypes.c_void_p),
                ("a1", ctypes.c_void_p), ("a2", ctypes.c_void_p), ("a0", ctypes.c_void_p),
                ("terms", ctypes.c_void_p), ("terms_user", ctypes.c_void_p)]


# int (*)(void *user, double t, double dt, double *q, double *f, hps_stream_t stream)
TERMS_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_void_p)


class hps_job_stats(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("arrival_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double), ("steps_done", ctypes.c_int),
                ("shared_operators", ctypes.c_int), ("work_bytes", ctypes.c_size_t),
                ("step_ms_mean", ctypes.c_double), ("step_ms_p50", ctypes.c_double), ("step_ms_p99", ctypes.c_double),
                ("evictions", ctypes.c_int)]


class hps_tune_result(ctypes.Structure):
    _fields_ = [("tile_cols", ctypes.c_int), ("flow_levels", ctypes.c_int), ("plan_target", ctypes.c_int),
                ("plan_kmin", ctypes.c_int), ("ms", ctypes.c_float)]


BATCH_OPTIONS = ("tensor_leaf", "even_odd", "flow_levels", "flow_n3_max", "cluster_splitk", "plan_target",
                 "plan_kmin", "plan_npc_max", "split_rhs", "fp64_ctas_per_sm", "group_offset", "last_cta_sum",
                 "fast_diag", "plan_tile_cols", "fuse_epilogue",
                 "fuse_jump", "fold_scale", "sa_close", "edge_projection",
                 "eo_cols", "tile_cols_w3", "tile_cols_h", "tile_cols_down",
                 "fp64_plan_target", "umma_leaf", "one_column_merge",
                 "one_column_sum", "stream_leaf",
                 "stream_chunk_kb", "sub_levels", "pdl",
                 "eo_threads", "prefetch_next", "b1_roll", "b1_kw", "stream_prefetch")


class hps_server_stats(ctypes.Structure):
    _fields_ = [("jobs_done", ctypes.c_int), ("jobs_rejected", ctypes.c_int), ("makespan_s", ctypes.c_double),
                ("dof_stages_per_s", ctypes.c_double), ("steps", ctypes.c_int64), ("step_ms_p50", ctypes.c_double),
                ("step_ms_p99", ctypes.c_double), ("max_concurrent", ctypes.c_int), ("peak_bytes", ctypes.c_size_t),
                ("factorizations_built", ctypes.c_int), ("factorizations_shared", ctypes.c_int), ("batches_formed", ctypes.c_int),
                ("mean_batch_cols", ctypes.c_double)]


# name -> (restype, argtypes); the list is also the set of exported symbols include/hps.h declares
SIGNATURES = {
    "hps_sizes": (ctypes.c_int, [ctypes.POINTER(hps_tree), ctypes.c_int, c_int64_p, c_int64_p, c_int64_p]),
    "hps_coords": (ctypes.c_int, [ctypes.POINTER(hps_tree), ctypes.c_int, c_double_p, c_double_p]),
    "hps_boundary_index": (ctypes.c_int, [ctypes.POINTER(hps_tree), ctypes.c_int, c_int64_p]),
    "hps_bytes": (ctypes.c_size_t, [ctypes.POINTER(hps_tree), ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "hps_build": (ctypes.c_int, [ctypes.POINTER(hps_tree), ctypes.c_int, ctypes.POINTER(hps_coeffs), ctypes.c_double,
                                 ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hps_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "hps_solve_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "hps_ark_abscissae": (ctypes.c_int, [c_double_p]),
    "ark_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(hps_ark_terms), ctypes.c_void_p]),
    "hps_set_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hps_set_persistent": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hps_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hps_trace_tasks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, c_double_p, ctypes.c_int]),
    "hps_selftest_barrier_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hps_selftest_conversions": (ctypes.c_int, [ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, c_int64_p]),
    "hps_trace_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint]),
    "hps_trace_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int64_p, c_int64_p,
                                      ctypes.POINTER(ctypes.c_double)]),
    "hps_batch_reserve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hps_batch_reserve_groups": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "hps_batch_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "hps_fastdiag_check": (ctypes.c_int, [ctypes.c_int, c_double_p, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, c_double_p]),
    "hps_batch_get_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "hps_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(hps_tune_result), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
    "hps_solve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "ark_step_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(hps_ark_terms), ctypes.c_int, ctypes.c_void_p]),
    "ark_slope_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(hps_ark_terms), ctypes.c_void_p]),
    "ark_slope_step_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                            ctypes.c_double, ctypes.POINTER(hps_ark_terms), ctypes.c_int,
                                            ctypes.c_void_p]),
    "ark_step_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(hps_ark_terms), ctypes.c_void_p]),
    "ark_step_batch_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                           ctypes.c_double, ctypes.POINTER(hps_ark_terms), ctypes.c_int,
                                           ctypes.c_void_p]),
    "hps_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "hps_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hps_job_desc), ctypes.POINTER(ctypes.c_int)]),
    "hps_server_run": (ctypes.c_int, [ctypes.c_void_p]),
    "hps_server_set_batching": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "hps_server_evict_after": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "hps_multi_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "hps_multi_set_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hps_multi_set_lockstep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hps_multi_ark_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                          ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "hps_multi_free": (None, [ctypes.c_void_p]),
    "hps_server_job_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(hps_job_stats)]),
    "hps_server_summary": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hps_server_stats)]),
    "hps_server_free": (None, [ctypes.c_void_p]),
    "hps_free": (None, [ctypes.c_void_p]),
    "hps_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def lib():
    """Load libhps.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhps.so is not built (run `python -m paper_2306_02526_gb300.build` "
                               "or __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class HPSError(RuntimeError):
    def __init__(self, code, what):
        msg = lib().hps_strerror(code).decode()
        super().__init__("%s failed: %s (%d)" % (what, msg, code))
        self.code = code


def check(code, what):
    if code != HPS_OK:
        raise HPSError(code, what)
