"""Python binding of the C ABI in include/sdsl.h (ctypes; marshalling only).

Every function here has the name of the C entry point it wraps and does
nothing but convert arguments: all computation happens in ``libsdsl.so``.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); the
binding derives ``mem_space`` from them.  The library must have been built
(``python -c "import __graft_entry__ as g; g.build()"``); loading fails
loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdsl.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_STATE = range(8)
FORM_CSR, FORM_NORMAL, FORM_AUGMENTED = 0, 1, 2
BJ_PCG, BBD_GMRES, BJ_BICGSTAB, BBD_GCR = 0, 1, 2, 3
MEM_HOST, MEM_DEVICE = 0, 1


class sdsl_options(C.Structure):
    _fields_ = [
        ("form", C.c_int), ("method", C.c_int), ("nblocks", C.c_int64), ("block_ptr", C.c_void_p),
        ("col_block_ptr", C.c_void_p), ("border", C.c_int64), ("tau", C.c_double), ("delta", C.c_double),
        ("rho", C.c_double), ("factor_prec", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int64),
        ("restart", C.c_int), ("refactor_ratio", C.c_double), ("mem_space", C.c_int), ("stream", C.c_void_p),
        ("graph_iters", C.c_int), ("tune", C.c_int), ("profile", C.c_int), ("apply_prec", C.c_int),
        ("flexible", C.c_int), ("solve_kernel", C.c_int), ("spmv_form", C.c_int), ("orthog", C.c_int),
        ("sweep_warps", C.c_int), ("sweep_backoff_ns", C.c_int), ("sweep_lane_entries", C.c_int),
        ("schur_lu", C.c_int), ("sweep_wait", C.c_int), ("wait_limit", C.c_int), ("sweep_far_gap", C.c_int),
        ("tau_switch_step", C.c_int64),
        ("tau_after", C.c_double), ("tau_relax", C.c_double), ("sweep_slots", C.c_int), ("wait_test", C.c_int),
    ]


class sdsl_stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int64), ("restarts", C.c_int64), ("rebuilt", C.c_int), ("status", C.c_int),
        ("rel_res_true", C.c_double), ("rel_res_rec", C.c_double), ("ms_setup", C.c_double),
        ("ms_factor", C.c_double), ("ms_solve", C.c_double), ("ms_update", C.c_double), ("n", C.c_int64),
        ("nnz_system", C.c_int64), ("nnz_precond", C.c_int64), ("nnz_factor", C.c_int64),
        ("levels_lower", C.c_int64), ("levels_upper", C.c_int64), ("max_levels", C.c_int64),
        ("shifted_blocks", C.c_int64), ("builds", C.c_int64), ("bytes_per_iter", C.c_double),
        ("kernel_ms", C.c_double * 4), ("kernel_launches", C.c_int64 * 4), ("kernel_bytes", C.c_double * 4),
        ("spmv_lanes", C.c_int64), ("solve_lanes", C.c_int64), ("tuned_spmv_lanes", C.c_int64),
        ("product_lanes", C.c_int64 * 2), ("ms_schur", C.c_double), ("ms_dense_lu", C.c_double),
        ("ms_dense_inverse", C.c_double), ("tau_used", C.c_double), ("ms_tune", C.c_double), ("sweep_shape", C.c_int64 * 2),
        ("product_kind", C.c_int64), ("iters_discarded", C.c_int64),
    ]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        return d


class sdsl_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz_system", C.c_int64), ("nnz_precond", C.c_int64), ("nblocks", C.c_int64),
                ("border", C.c_int64), ("levels_lower", C.c_int64), ("levels_upper", C.c_int64),
                ("factored", C.c_int), ("device_bytes", C.c_int64), ("peak_device_bytes", C.c_int64)]


_lib = None
_VP = C.c_void_p
_I64 = C.c_int64


def load():
    """Load libsdsl.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2604_23979_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    H = C.c_void_p
    L.sdsl_default_options.argtypes = [C.POINTER(sdsl_options)]
    L.sdsl_default_options.restype = None
    L.sdsl_setup.argtypes = [C.POINTER(sdsl_options), _I64, _I64, _VP, _VP, _VP, _VP, C.POINTER(H)]
    L.sdsl_factor.argtypes = [H]
    L.sdsl_solve.argtypes = [H, _VP, _VP, C.c_int, C.POINTER(sdsl_stats)]
    L.sdsl_update_diag.argtypes = [H, _VP]
    L.sdsl_set_tau.argtypes = [H, C.c_double]
    L.sdsl_batch_solve.argtypes = [C.c_int, _VP, _VP, _VP, C.c_int, _VP]
    L.sdsl_batch_create.argtypes = [C.c_int, C.POINTER(C.c_void_p)]
    L.sdsl_batch_add.argtypes = [_VP, _VP, _VP, _VP, C.c_int]
    L.sdsl_batch_step.argtypes = [_VP, C.c_int, _VP, _VP, C.c_int, C.POINTER(C.c_int)]
    L.sdsl_batch_size.argtypes = [_VP]
    L.sdsl_batch_size.restype = C.c_int
    L.sdsl_batch_free.argtypes = [_VP]
    L.sdsl_free.argtypes = [H]
    L.sdsl_get_stats.argtypes = [H, C.POINTER(sdsl_stats)]
    L.sdsl_get_info.argtypes = [H, C.POINTER(sdsl_info)]
    L.sdsl_export_system.argtypes = [H, _VP, _VP, _VP]
    L.sdsl_export_precond.argtypes = [H, _VP, _VP, _VP, _VP, _VP]
    L.sdsl_export_levels.argtypes = [H, C.c_int, _VP, _VP, _VP]
    L.sdsl_export_schur.argtypes = [H, _VP]
    L.sdsl_export_schur_lu.argtypes = [H, _VP, _VP]
    L.sdsl_spmv.argtypes = [H, _VP, _VP]
    L.sdsl_precond_apply.argtypes = [H, _VP, _VP]
    L.sdsl_normal_spmv_noalloc.argtypes = [_I64, _I64, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, C.c_double,
                                           _VP, _VP, _VP]
    L.sdsl_status_str.argtypes = [C.c_int]
    L.sdsl_status_str.restype = C.c_char_p
    L.sdsl_kernel_launches.argtypes = []
    L.sdsl_kernel_launches.restype = C.c_int64
    L.sdsl_last_error.argtypes = []
    L.sdsl_last_error.restype = C.c_char_p
    for f in ("sdsl_setup", "sdsl_factor", "sdsl_solve", "sdsl_batch_solve", "sdsl_batch_create", "sdsl_batch_add",
              "sdsl_batch_step", "sdsl_batch_free", "sdsl_update_diag", "sdsl_set_tau", "sdsl_free", "sdsl_get_stats",
              "sdsl_get_info", "sdsl_export_system", "sdsl_export_precond", "sdsl_export_levels",
              "sdsl_export_schur", "sdsl_export_schur_lu", "sdsl_spmv", "sdsl_precond_apply", "sdsl_normal_spmv_noalloc"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


class SdslError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(st, allow=()):
    if st != OK and st not in allow:
        L = load()
        raise SdslError(st, f"{L.sdsl_status_str(st).decode()}: {L.sdsl_last_error().decode()}")
    return st


def _ptr(a):
    """(pointer, is_device, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, None, None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            a = np.ascontiguousarray(a)
        return a.ctypes.data, False, a
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.is_cuda, a
    raise TypeError(f"unsupported array type {type(a)}")


def sdsl_default_options() -> sdsl_options:
    o = sdsl_options()
    load().sdsl_default_options(C.byref(o))
    return o


def sdsl_setup(opt: sdsl_options, m, n, rowptr, col, val, theta=None):
    keep = []
    ptrs = []
    dev = None
    for a in (rowptr, col, val, theta):
        p, d, k = _ptr(a)
        keep.append(k)
        ptrs.append(p)
        if d is not None:
            if dev is not None and d != dev:
                raise ValueError("all arrays must live in the same memory space")
            dev = d
    opt.mem_space = MEM_DEVICE if dev else MEM_HOST
    h = C.c_void_p()
    _check(load().sdsl_setup(C.byref(opt), int(m), int(n), ptrs[0], ptrs[1], ptrs[2], ptrs[3], C.byref(h)))
    return h


def sdsl_factor(h):
    return _check(load().sdsl_factor(h))


def sdsl_solve(h, b, x, x0_zero=True, allow=(ERR_NOT_CONVERGED,)):
    st = sdsl_stats()
    pb, _, kb = _ptr(b)
    px, _, kx = _ptr(x)
    rc = load().sdsl_solve(h, pb, px, 1 if x0_zero else 0, C.byref(st))
    _check(rc, allow)
    return st


def sdsl_batch_solve(hs, bs, xs, x0_zero=True, allow=(ERR_NOT_CONVERGED,)):
    """Solve len(hs) systems together (each handle with its own b and x);
    returns the list of per-request statistics."""
    n = len(hs)
    for x in xs:
        if (isinstance(x, np.ndarray) and not x.flags.c_contiguous) or (hasattr(x, "is_contiguous")
                                                                         and not x.is_contiguous()):
            raise ValueError("x arrays must be contiguous (they receive the solutions)")
    pb = [_ptr(b) for b in bs]  # keeps any contiguous copy of b alive for the call
    px = [_ptr(x) for x in xs]
    H = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    B = (C.c_void_p * n)(*[p[0] for p in pb])
    X = (C.c_void_p * n)(*[p[0] for p in px])
    st = (sdsl_stats * n)()
    rc = load().sdsl_batch_solve(n, C.cast(H, C.c_void_p), C.cast(B, C.c_void_p), C.cast(X, C.c_void_p),
                                 1 if x0_zero else 0, C.cast(st, C.c_void_p))
    _check(rc, allow)
    return list(st)


def sdsl_batch_create(graph_iters=16):
    B = C.c_void_p()
    _check(load().sdsl_batch_create(int(graph_iters), C.byref(B)))
    return B


def sdsl_batch_add(B, h, b, x, x0_zero=True):
    """Add a request (factored handle h, right-hand side b, solution x) to the
    batch; b and x must stay alive until the request is handed back."""
    if (isinstance(x, np.ndarray) and not x.flags.c_contiguous) or (hasattr(x, "is_contiguous")
                                                                     and not x.is_contiguous()):
        raise ValueError("x must be contiguous (it receives the solution)")
    pb, px = _ptr(b), _ptr(x)
    if pb[2] is not b:
        raise ValueError("b must be contiguous (it is read while the batch runs)")
    return _check(load().sdsl_batch_add(B, h, pb[0], px[0], 1 if x0_zero else 0))


def sdsl_batch_step(B, max_graphs=1, cap=64):
    """Launch the batch until a request finishes (or max_graphs graph
    launches); returns [(handle value, stats)] of the requests that left."""
    hs = (C.c_void_p * cap)()
    st = (sdsl_stats * cap)()
    nd = C.c_int(0)
    _check(load().sdsl_batch_step(B, int(max_graphs), C.cast(hs, C.c_void_p), C.cast(st, C.c_void_p), int(cap),
                                  C.byref(nd)))
    return [(hs[k], st[k]) for k in range(nd.value)]


def sdsl_batch_size(B):
    return int(load().sdsl_batch_size(B))


def sdsl_batch_free(B):
    return _check(load().sdsl_batch_free(B))


def sdsl_update_diag(h, theta):
    p, _, k = _ptr(theta)
    return _check(load().sdsl_update_diag(h, p))


def sdsl_set_tau(h, tau):
    return _check(load().sdsl_set_tau(h, float(tau)))


def sdsl_free(h):
    return _check(load().sdsl_free(h))


def sdsl_get_stats(h) -> sdsl_stats:
    st = sdsl_stats()
    _check(load().sdsl_get_stats(h, C.byref(st)))
    return st


def sdsl_get_info(h) -> sdsl_info:
    info = sdsl_info()
    _check(load().sdsl_get_info(h, C.byref(info)))
    return info


def sdsl_export_system(h):
    info = sdsl_get_info(h)
    rp = np.zeros(info.n + 1, np.int64)
    ci = np.zeros(max(info.nnz_system, 1), np.int32)
    v = np.zeros(max(info.nnz_system, 1), np.float64)
    _check(load().sdsl_export_system(h, rp.ctypes.data, ci.ctypes.data, v.ctypes.data))
    return rp, ci[: info.nnz_system], v[: info.nnz_system]


def sdsl_export_precond(h):
    info = sdsl_get_info(h)
    nnz = info.nnz_precond
    rp = np.zeros(info.n + 1, np.int64)
    ci = np.zeros(max(nnz, 1), np.int32)
    pv = np.zeros(max(nnz, 1))
    fv = np.zeros(max(nnz, 1))
    al = np.zeros(max(info.nblocks, 1))
    _check(load().sdsl_export_precond(h, rp.ctypes.data, ci.ctypes.data, pv.ctypes.data, fv.ctypes.data,
                                      al.ctypes.data))
    return rp, ci[:nnz], pv[:nnz], fv[:nnz], al[: info.nblocks]


def sdsl_export_levels(h, which):
    info = sdsl_get_info(h)
    tot = info.levels_lower if which == 0 else info.levels_upper
    nlev = np.zeros(max(info.nblocks, 1), np.int32)
    lptr = np.zeros(tot + 1, np.int64)
    rows = np.zeros(max(info.n, 1), np.int32)
    _check(load().sdsl_export_levels(h, int(which), nlev.ctypes.data, lptr.ctypes.data, rows.ctypes.data))
    return nlev[: info.nblocks], lptr, rows


def sdsl_kernel_launches() -> int:
    return int(load().sdsl_kernel_launches())


def sdsl_export_schur_lu(h, nbord):
    """(ipiv, pivots) of the border Schur LU (host arrays of nbord entries)."""
    ipiv = np.zeros(max(nbord, 1), np.int32)
    piv = np.zeros(max(nbord, 1))
    _check(load().sdsl_export_schur_lu(h, ipiv.ctypes.data, piv.ctypes.data))
    return ipiv[:nbord], piv[:nbord]


def sdsl_spmv(h, x, y):
    return _check(load().sdsl_spmv(h, _ptr(x)[0], _ptr(y)[0]))


def sdsl_precond_apply(h, r, z):
    return _check(load().sdsl_precond_apply(h, _ptr(r)[0], _ptr(z)[0]))


def sdsl_status_str_py(status) -> str:
    """Name of a status code."""
    return load().sdsl_status_str(int(status)).decode()


NOALLOC_MAX_COLS = 1 << 19


def sdsl_normal_spmv_noalloc(m, n, nnz, a_rowptr, a_col, a_val, at_rowptr, at_col, at_val, theta, rho, x, y,
                             stream=0):
    """y = A (theta o (A^T x)) + rho x without any device allocation (all
    arrays are device tensors of the current device; stream is a raw
    cudaStream_t handle, 0 for the legacy default stream)."""
    ptrs = [_ptr(a)[0] for a in (a_rowptr, a_col, a_val, at_rowptr, at_col, at_val, theta, x, y)]
    return _check(load().sdsl_normal_spmv_noalloc(m, n, nnz, *ptrs[:7], float(rho), ptrs[7], ptrs[8], stream or None))


def options_for(prob, method=BJ_PCG, factor_prec=64, graph_iters=16, stream=None):
    """Options (and the keep-alive block-pointer arrays) for a workloads problem."""
    o = sdsl_default_options()
    o.method = method
    o.factor_prec = factor_prec
    o.graph_iters = graph_iters
    o.tau, o.delta, o.rho, o.rtol, o.maxit = prob.tau, prob.delta, prob.rho, prob.rtol, prob.maxit
    keep = []
    if hasattr(prob, "block_ptr"):
        o.form = FORM_NORMAL
        bp = np.ascontiguousarray(prob.block_ptr, dtype=np.int64)
        keep.append(bp)
        o.nblocks = len(bp) - 1
        o.block_ptr = bp.ctypes.data
    else:
        o.form = FORM_AUGMENTED
        o.method = BBD_GMRES
        rbp = np.ascontiguousarray(prob.row_block_ptr, dtype=np.int64)
        cbp = np.ascontiguousarray(prob.col_block_ptr, dtype=np.int64)
        keep += [rbp, cbp]
        o.nblocks = len(rbp) - 1
        o.block_ptr = rbp.ctypes.data
        o.col_block_ptr = cbp.ctypes.data
        o.border = prob.nlink
        o.restart = prob.restart
    if stream is not None:
        o.stream = stream
    return o, keep
