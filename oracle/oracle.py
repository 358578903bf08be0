"""ctypes wrapper of the C oracle (FP64, single thread).

TEST INFRASTRUCTURE ONLY.  Allocation and marshalling live here; every step
of the arithmetic is in ``sdsl_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

_lib = None

_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_I64 = C.c_int64
_F64 = C.c_double
_VP = C.c_void_p

OK, ARG, OOM, BREAKDOWN, NOT_CONVERGED = 0, 1, 2, 4, 5


def threads() -> int:
    """Host threads the oracle's parallel block and row loops use (1 without OpenMP)."""
    return int(lib().or_threads())


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(_build.build()))
    return _lib


class use_library:
    """Context manager that routes the wrapper to another build of the oracle
    (the mutation tests load deliberately broken copies through it)."""

    def __init__(self, path):
        self.L = _bind(C.CDLL(path))

    def __enter__(self):
        global _lib
        self.saved, _lib = lib(), self.L
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _bind(L):
    if True:
        L.or_transpose.argtypes = [_I64, _I64, _i64p, _i32p, _f64p, _i64p, _i32p, _f64p]
        L.or_normal_pattern.argtypes = [_I64, _I64, _i64p, _i32p, _i64p, _i32p, _i64p, _VP]
        L.or_normal_pattern.restype = _I64
        L.or_normal_values.argtypes = [_I64, _I64, _i64p, _i32p, _f64p, _f64p, _F64, _i64p, _i32p, _f64p]
        L.or_bbd_order.argtypes = [_I64, _I64, _I64, _i64p, _i64p, _i64p, _i64p]
        L.or_augmented.argtypes = [_I64, _I64, _i64p, _i32p, _f64p, _i64p, _i32p, _f64p, _f64p, _F64,
                                   _i64p, _i64p, _VP, _VP]
        L.or_augmented.restype = _I64
        L.or_filter_correct.argtypes = [_I64, _i64p, _i32p, _f64p, _I64, _i64p, C.c_int, _F64, _F64,
                                        _i64p, _VP, _VP]
        L.or_filter_correct.restype = _I64
        L.or_levels.argtypes = [_I64, _i64p, _i32p, _I64, _i64p, _i32p, _i32p]
        L.or_level_lists.argtypes = [_I64, _i64p, _i32p, _i32p, _VP, _VP]
        L.or_ic0.argtypes = [_I64, _i64p, _i32p, _f64p, _I64, _i64p, _f64p, C.c_int, _f64p, _f64p]
        L.or_ic0.restype = C.c_int
        L.or_ilu0.argtypes = L.or_ic0.argtypes
        L.or_ilu0.restype = C.c_int
        L.or_ic0_apply.argtypes = [_I64, _i64p, _i32p, _f64p, _I64, _i64p, _f64p, _f64p]
        L.or_ilu0_apply.argtypes = L.or_ic0_apply.argtypes
        L.or_spmv.argtypes = [_I64, _i64p, _i32p, _f64p, _f64p, _f64p]
        L.or_threads.argtypes = []
        L.or_threads.restype = C.c_int
        L.or_dense_lu.argtypes = [_I64, _f64p, _i32p]
        L.or_dense_lu.restype = C.c_int
        L.or_dense_lu_solve.argtypes = [_I64, _f64p, _i32p, _f64p]
        L.or_bbd_schur.argtypes = [_I64, _i64p, _i32p, _f64p, _f64p, _I64, _i64p, _f64p]
        L.or_bbd_apply.argtypes = [_I64, _i64p, _i32p, _f64p, _f64p, _I64, _i64p, _f64p, _i32p, _f64p, _f64p]
        L.or_pcg_bj.argtypes = [_I64, _i64p, _i32p, _f64p, _i64p, _i32p, _f64p, _I64, _i64p, _f64p, _f64p,
                                _F64, _I64, _i64p, _f64p]
        L.or_pcg_bj.restype = C.c_int
        L.or_gmres_pre.argtypes = [C.c_int, _I64, _i64p, _i32p, _f64p, _i64p, _i32p, _VP, _VP, _I64, _VP,
                                   _VP, _VP, _f64p, _f64p, _F64, _I64, _I64, _i64p, _f64p]
        L.or_gmres_pre.restype = C.c_int
        L.or_precond_apply.argtypes = [C.c_int, _I64, _i64p, _i32p, _VP, _VP, _I64, _VP, _VP, _VP, _f64p, _f64p]
        L.or_bicgstab_pre.argtypes = [C.c_int, _I64, _i64p, _i32p, _f64p, _i64p, _i32p, _VP, _VP, _I64, _VP,
                                      _f64p, _f64p, _F64, _I64, _i64p, _f64p]
        L.or_bicgstab_pre.restype = C.c_int
        L.or_gcr_pre.argtypes = L.or_gmres_pre.argtypes
        L.or_gcr_pre.restype = C.c_int
    return L


@dataclasses.dataclass
class Mat:
    """CSR matrix (int64 row pointers, int32 sorted columns, float64 values)."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def dense(self):
        d = np.zeros((self.nrows, self.ncols))
        for i in range(self.nrows):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            d[i, self.col[s:e]] = self.val[s:e]
        return d


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def as_mat(A) -> Mat:
    return Mat(int(A.nrows), int(A.ncols), _c(A.rowptr, np.int64), _c(A.col, np.int32), _c(A.val, np.float64))


def from_dense(d: np.ndarray) -> Mat:
    """CSR of the nonzero pattern of a dense array (test helper)."""
    d = np.asarray(d, dtype=np.float64)
    rows, cols = np.nonzero(d)
    rowptr = np.zeros(d.shape[0] + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=d.shape[0]), out=rowptr[1:])
    return Mat(d.shape[0], d.shape[1], rowptr, cols.astype(np.int32), d[rows, cols].copy())


def _ptr(p):
    return p.ctypes.data_as(_VP) if p is not None else None


def transpose(A) -> Mat:
    A = as_mat(A)
    trp = np.zeros(A.ncols + 1, np.int64)
    tci = np.zeros(max(A.nnz, 1), np.int32)
    tv = np.zeros(max(A.nnz, 1), np.float64)
    lib().or_transpose(A.nrows, A.ncols, A.rowptr, A.col, A.val, trp, tci, tv)
    return Mat(A.ncols, A.nrows, trp, tci[: A.nnz], tv[: A.nnz])


def normal_pattern(A) -> Mat:
    A = as_mat(A)
    T = transpose(A)
    srp = np.zeros(A.nrows + 1, np.int64)
    nnz = lib().or_normal_pattern(A.nrows, A.ncols, A.rowptr, A.col, T.rowptr, _c(T.col, np.int32), srp, None)
    sci = np.zeros(max(nnz, 1), np.int32)
    lib().or_normal_pattern(A.nrows, A.ncols, A.rowptr, A.col, T.rowptr, _c(T.col, np.int32), srp, _ptr(sci))
    return Mat(A.nrows, A.nrows, srp, sci[:nnz], np.zeros(nnz))


def normal_values(A, theta, rho, pattern: Mat) -> np.ndarray:
    A = as_mat(A)
    sv = np.zeros(max(pattern.nnz, 1))
    lib().or_normal_values(A.nrows, A.ncols, A.rowptr, A.col, A.val, _c(theta, np.float64), float(rho),
                           pattern.rowptr, _c(pattern.col, np.int32), sv)
    return sv[: pattern.nnz]


def normal_matrix(A, theta, rho) -> Mat:
    """S = A diag(theta) A^T + rho I (Eq. schur) with the fixed rounding order."""
    S = normal_pattern(A)
    S.val = normal_values(A, theta, rho, S)
    return S


def bbd_order(m, n, row_block_ptr, col_block_ptr):
    nblocks = len(row_block_ptr) - 1
    pos = np.zeros(n + m, np.int64)
    kbp = np.zeros(nblocks + 1, np.int64)
    lib().or_bbd_order(m, n, nblocks, _c(row_block_ptr, np.int64), _c(col_block_ptr, np.int64), pos, kbp)
    return pos, kbp


def augmented(A, theta, rho, row_block_ptr, col_block_ptr):
    """K = [[-diag(1/theta), A^T], [A, rho I]] in BBD order; returns (K, pos, kblock_ptr)."""
    A = as_mat(A)
    T = transpose(A)
    pos, kbp = bbd_order(A.nrows, A.ncols, row_block_ptr, col_block_ptr)
    N = A.nrows + A.ncols
    krp = np.zeros(N + 1, np.int64)
    args = (A.nrows, A.ncols, A.rowptr, A.col, A.val, T.rowptr, _c(T.col, np.int32), _c(T.val, np.float64),
            _c(theta, np.float64), float(rho), pos, krp)
    nnz = lib().or_augmented(*args, None, None)
    kci = np.zeros(max(nnz, 1), np.int32)
    kv = np.zeros(max(nnz, 1))
    lib().or_augmented(*args, _ptr(kci), _ptr(kv))
    return Mat(N, N, krp, kci[:nnz], kv[:nnz]), pos, kbp


def filter_correct(S, block_ptr, tau, delta, whole=False) -> Mat:
    """Preconditioner matrix P: Eq. (filter) then Eq. (diagcorr)."""
    S = as_mat(S)
    bp = _c(block_ptr, np.int64)
    prp = np.zeros(S.nrows + 1, np.int64)
    args = (S.nrows, S.rowptr, S.col, S.val, len(bp) - 1, bp, int(bool(whole)), float(tau), float(delta), prp)
    nnz = lib().or_filter_correct(*args, None, None)
    pci = np.zeros(max(nnz, 1), np.int32)
    pv = np.zeros(max(nnz, 1))
    lib().or_filter_correct(*args, _ptr(pci), _ptr(pv))
    return Mat(S.nrows, S.ncols, prp, pci[:nnz], pv[:nnz])


def levels(P, block_ptr):
    P = as_mat(P)
    bp = _c(block_ptr, np.int64)
    lo = np.zeros(P.nrows, np.int32)
    up = np.zeros(P.nrows, np.int32)
    lib().or_levels(P.nrows, P.rowptr, P.col, len(bp) - 1, bp, lo, up)
    return lo, up


def level_lists(block_ptr, lev):
    """(nlev per block, level_ptr, level_rows) with rows ascending in each level."""
    bp = _c(block_ptr, np.int64)
    nb = len(bp) - 1
    nlev = np.zeros(max(nb, 1), np.int32)
    lev = _c(lev, np.int32)
    lib().or_level_lists(nb, bp, lev, nlev, None, None)
    total = int(nlev[:nb].sum())
    lptr = np.zeros(total + 1, np.int64)
    rows = np.zeros(max(int(bp[-1] - bp[0]), 1), np.int32)
    lib().or_level_lists(nb, bp, lev, nlev, _ptr(lptr), _ptr(rows))
    return nlev[:nb], lptr, rows[: int(bp[-1] - bp[0])]


DEFAULT_SHIFTS = (0.0, 1e-3, 1e-2, 1e-1, 1.0)


def ic0(P, block_ptr, shifts=DEFAULT_SHIFTS):
    """Per-block IC(0) with the shift-retry rule; returns (F, alpha, status)."""
    P = as_mat(P)
    bp = _c(block_ptr, np.int64)
    F = np.zeros(max(P.nnz, 1))
    alpha = np.zeros(max(len(bp) - 1, 1))
    sh = _c(shifts, np.float64)
    st = lib().or_ic0(P.nrows, P.rowptr, P.col, P.val, len(bp) - 1, bp, sh, len(sh), F, alpha)
    return F[: P.nnz], alpha[: len(bp) - 1], st


def ilu0(P, block_ptr, shifts=DEFAULT_SHIFTS):
    P = as_mat(P)
    bp = _c(block_ptr, np.int64)
    F = np.zeros(max(P.nnz, 1))
    alpha = np.zeros(max(len(bp) - 1, 1))
    sh = _c(shifts, np.float64)
    st = lib().or_ilu0(P.nrows, P.rowptr, P.col, P.val, len(bp) - 1, bp, sh, len(sh), F, alpha)
    return F[: P.nnz], alpha[: len(bp) - 1], st


def ic0_apply(P, F, block_ptr, r):
    P = as_mat(P)
    bp = _c(block_ptr, np.int64)
    z = np.zeros(P.nrows)
    lib().or_ic0_apply(P.nrows, P.rowptr, P.col, _c(F, np.float64), len(bp) - 1, bp, _c(r, np.float64), z)
    return z


def ilu0_apply(P, F, block_ptr, r):
    P = as_mat(P)
    bp = _c(block_ptr, np.int64)
    z = np.zeros(P.nrows)
    lib().or_ilu0_apply(P.nrows, P.rowptr, P.col, _c(F, np.float64), len(bp) - 1, bp, _c(r, np.float64), z)
    return z


def spmv(S, x):
    S = as_mat(S)
    y = np.zeros(S.nrows)
    lib().or_spmv(S.nrows, S.rowptr, S.col, S.val, _c(x, np.float64), y)
    return y


def dense_lu(a):
    a = _c(a, np.float64).copy()
    nb = a.shape[0]
    ipiv = np.zeros(max(nb, 1), np.int32)
    st = lib().or_dense_lu(nb, a, ipiv)
    return a, ipiv[:nb], st


def dense_lu_solve(lu, ipiv, b):
    x = _c(b, np.float64).copy()
    lib().or_dense_lu_solve(lu.shape[0], _c(lu, np.float64), _c(ipiv, np.int32), x)
    return x


def bbd_schur(P, F, block_ptr):
    P = as_mat(P)
    bp = _c(block_ptr, np.int64)
    nb = P.nrows - int(bp[-1])
    SB = np.zeros(max(nb * nb, 1))
    lib().or_bbd_schur(P.nrows, P.rowptr, P.col, P.val, _c(F, np.float64), len(bp) - 1, bp, SB)
    return SB[: nb * nb].reshape(nb, nb)


def bbd_apply(P, F, block_ptr, lu, ipiv, r):
    P = as_mat(P)
    bp = _c(block_ptr, np.int64)
    z = np.zeros(P.nrows)
    lib().or_bbd_apply(P.nrows, P.rowptr, P.col, P.val, _c(F, np.float64), len(bp) - 1, bp,
                       _c(lu, np.float64).reshape(-1), _c(ipiv, np.int32), _c(r, np.float64), z)
    return z


@dataclasses.dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    relres_true: float
    relres_rec: float
    status: int


def pcg_bj(S, P, F, block_ptr, b, x0=None, rtol=1e-8, maxit=2000) -> SolveResult:
    """Block-Jacobi IC(0) preconditioned CG (Sec. 2.3)."""
    S, P = as_mat(S), as_mat(P)
    bp = _c(block_ptr, np.int64)
    x = np.zeros(S.nrows) if x0 is None else _c(x0, np.float64).copy()
    it = np.zeros(1, np.int64)
    out = np.zeros(2)
    st = lib().or_pcg_bj(S.nrows, S.rowptr, S.col, S.val, P.rowptr, P.col, _c(F, np.float64), len(bp) - 1, bp,
                         _c(b, np.float64), x, float(rtol), int(maxit), it, out)
    return SolveResult(x, int(it[0]), float(out[0]), float(out[1]), st)


PRE_NONE, PRE_BJ_IC0, PRE_BJ_ILU0, PRE_BBD = 0, 1, 2, 3


def gmres(K, b, kind=PRE_NONE, P=None, F=None, block_ptr=None, lu=None, ipiv=None, x0=None, rtol=1e-8,
          maxit=3000, restart=30) -> SolveResult:
    """Right-preconditioned GMRES(restart) with modified Gram-Schmidt."""
    K = as_mat(K)
    x = np.zeros(K.nrows) if x0 is None else _c(x0, np.float64).copy()
    it = np.zeros(1, np.int64)
    out = np.zeros(2)
    keep = []

    def p(a, dt):
        if a is None:
            return None
        a = _c(a, dt)
        keep.append(a)
        return a.ctypes.data_as(_VP)

    Pm = as_mat(P) if P is not None else K
    bp = _c(block_ptr if block_ptr is not None else np.zeros(1, np.int64), np.int64)
    st = lib().or_gmres_pre(int(kind), K.nrows, K.rowptr, K.col, K.val, Pm.rowptr, Pm.col, p(Pm.val, np.float64),
                            p(F, np.float64), len(bp) - 1, p(bp, np.int64), p(None if lu is None else np.asarray(lu).reshape(-1), np.float64),
                            p(ipiv, np.int32), _c(b, np.float64), x, float(rtol), int(maxit), int(restart), it, out)
    return SolveResult(x, int(it[0]), float(out[0]), float(out[1]), st)


def bicgstab(S, b, kind=PRE_NONE, P=None, F=None, block_ptr=None, x0=None, rtol=1e-8,
             maxit=2000) -> SolveResult:
    """Right-preconditioned BiCGSTAB (the Block-Jacobi pairing of Sec. 4.3);
    kind is PRE_NONE, PRE_BJ_IC0 or PRE_BJ_ILU0."""
    S = as_mat(S)
    x = np.zeros(S.nrows) if x0 is None else _c(x0, np.float64).copy()
    it = np.zeros(1, np.int64)
    out = np.zeros(2)
    keep = []

    def p(a, dt):
        if a is None:
            return None
        a = _c(a, dt)
        keep.append(a)
        return a.ctypes.data_as(_VP)

    Pm = as_mat(P) if P is not None else S
    bp = _c(block_ptr if block_ptr is not None else np.zeros(1, np.int64), np.int64)
    st = lib().or_bicgstab_pre(int(kind), S.nrows, S.rowptr, S.col, S.val, Pm.rowptr, Pm.col,
                               p(Pm.val, np.float64), p(F, np.float64), len(bp) - 1, p(bp, np.int64),
                               _c(b, np.float64), x, float(rtol), int(maxit), it, out)
    return SolveResult(x, int(it[0]), float(out[0]), float(out[1]), st)


def gcr(K, b, kind=PRE_NONE, P=None, F=None, block_ptr=None, lu=None, ipiv=None, x0=None, rtol=1e-8,
        maxit=3000, restart=30) -> SolveResult:
    """Restarted right-preconditioned GCR(restart), the "IGCR(m)" of Sec. 4.3."""
    K = as_mat(K)
    x = np.zeros(K.nrows) if x0 is None else _c(x0, np.float64).copy()
    it = np.zeros(1, np.int64)
    out = np.zeros(2)
    keep = []

    def p(a, dt):
        if a is None:
            return None
        a = _c(a, dt)
        keep.append(a)
        return a.ctypes.data_as(_VP)

    Pm = as_mat(P) if P is not None else K
    bp = _c(block_ptr if block_ptr is not None else np.zeros(1, np.int64), np.int64)
    st = lib().or_gcr_pre(int(kind), K.nrows, K.rowptr, K.col, K.val, Pm.rowptr, Pm.col, p(Pm.val, np.float64),
                          p(F, np.float64), len(bp) - 1, p(bp, np.int64),
                          p(None if lu is None else np.asarray(lu).reshape(-1), np.float64), p(ipiv, np.int32),
                          _c(b, np.float64), x, float(rtol), int(maxit), int(restart), it, out)
    return SolveResult(x, int(it[0]), float(out[0]), float(out[1]), st)


def precond_apply(kind, P, F, block_ptr, r, lu=None, ipiv=None):
    P = as_mat(P)
    bp = _c(block_ptr, np.int64)
    z = np.zeros(P.nrows)
    keep = [_c(P.val, np.float64), _c(F, np.float64)]
    lu_a = None if lu is None else _c(np.asarray(lu).reshape(-1), np.float64)
    ip_a = None if ipiv is None else _c(ipiv, np.int32)
    lib().or_precond_apply(int(kind), P.nrows, P.rowptr, P.col, keep[0].ctypes.data_as(_VP),
                           keep[1].ctypes.data_as(_VP), len(bp) - 1, bp.ctypes.data_as(_VP),
                           _ptr(lu_a), _ptr(ip_a), _c(r, np.float64), z)
    return z


# ---------------------------------------------------------------------------
# whole pipelines
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class BJState:
    S: Mat
    P: Mat
    F: np.ndarray
    alpha: np.ndarray
    status: int
    lev_lo: np.ndarray
    lev_up: np.ndarray


def bj_setup_factor(A, theta, rho, block_ptr, tau, delta) -> BJState:
    """Eq. (schur) -> Eq. (filter) -> Eq. (diagcorr) -> levels -> IC(0)."""
    S = normal_matrix(A, theta, rho)
    P = filter_correct(S, block_ptr, tau, delta)
    lo, up = levels(P, block_ptr)
    F, alpha, st = ic0(P, block_ptr)
    return BJState(S, P, F, alpha, st, lo, up)


def bj_solve(prob, x0=None) -> tuple[BJState, SolveResult]:
    st = bj_setup_factor(prob.A, prob.theta, prob.rho, prob.block_ptr, prob.tau, prob.delta)
    res = pcg_bj(st.S, st.P, st.F, prob.block_ptr, prob.b, x0, prob.rtol, prob.maxit)
    return st, res
