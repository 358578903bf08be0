"""Seeded synthetic inputs shaped like the interior-point systems of the paper.

This module only draws structure, values, scalings (theta) and right-hand
sides.  It contains none of the solver's arithmetic (no products, no
filtering, no factorization), so the CUDA path and the CPU oracle can both
consume its arrays without sharing any method code.

The paper's own benchmark matrices (PageRank, Mittelmann, NetworkPlan, SCUC,
MIPLIB; Table "benchmarks", Sec. 4.1) are not available, so the shapes below
stand in for them:

* ``config1``  random LP matrix A (2,000 x 5,000, 5 nonzeros per column at
  uniform random rows), normal equations, 4 equal row blocks;
* ``config2``  staircase A (200,000 x 500,000, 64 uneven diagonal blocks,
  8 nonzeros per column, 90 % inside the column's own block);
* ``config3``  block-angular A (128 blocks, 2,048 linking rows) in the
  augmented (KKT) form of Eq. (augmented);
* ``config4``  staircase A (2,000,000 x 5,000,000, 256 blocks) with a
  30-step drifting theta sequence (preconditioner reuse, Sec. 3.4);
* ``serving_requests``  a Poisson stream of staircase problems.

Every generator takes a ``scale`` so that tests can draw small instances
of the same shape.  Random draws happen in a fixed order: structure,
values, theta, right-hand side.  CSR arrays are ``int64`` row pointers,
``int32`` column indices sorted inside each row, ``float64`` values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Csr:
    """A sparse matrix in CSR form (rows sorted, no duplicates)."""

    nrows: int
    ncols: int
    rowptr: np.ndarray  # int64 [nrows+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols))
        for i in range(self.nrows):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            d[i, self.col[s:e]] = self.val[s:e]
        return d


@dataclasses.dataclass
class NormalProblem:
    """S = A diag(theta) A^T + rho I, solved by Block Jacobi PCG."""

    A: Csr
    theta: np.ndarray
    b: np.ndarray
    block_ptr: np.ndarray  # int64 [nblocks+1] row blocks of S (= of A)
    rho: float
    tau: float
    delta: float
    rtol: float = 1e-8
    maxit: int = 2000
    name: str = ""


@dataclasses.dataclass
class AugmentedProblem:
    """K = [[-diag(1/theta), A^T], [A, rho I]] in bordered block-diagonal order.

    A's rows are ordered block by block with the ``nlink`` linking rows last;
    A's columns are ordered block by block.  ``row_block_ptr`` and
    ``col_block_ptr`` delimit the diagonal blocks of A.
    """

    A: Csr
    theta: np.ndarray
    b: np.ndarray  # right-hand side in the BBD order of K
    row_block_ptr: np.ndarray
    col_block_ptr: np.ndarray
    nlink: int
    rho: float
    tau: float
    delta: float
    rtol: float = 1e-8
    maxit: int = 3000
    restart: int = 30
    name: str = ""


# ---------------------------------------------------------------------------
# small helpers (integer bookkeeping only)
# ---------------------------------------------------------------------------

def _largest_remainder(weights: np.ndarray, total: int) -> np.ndarray:
    """Integers proportional to ``weights`` that sum to ``total``."""
    w = np.asarray(weights, dtype=np.float64)
    exact = w * (total / w.sum())
    base = np.floor(exact).astype(np.int64)
    rest = int(total - base.sum())
    if rest > 0:
        frac = exact - base
        order = np.lexsort((np.arange(len(w)), -frac))  # largest first, ties by index
        base[order[:rest]] += 1
    return base


def _sizes_in_range(raw: np.ndarray, total: int, lo: int, hi: int) -> np.ndarray:
    """Scale ``raw`` to sum ``total`` while keeping every entry in [lo, hi]."""
    sizes = _largest_remainder(raw, total)
    for _ in range(1000):
        sizes = np.clip(sizes, lo, hi)
        diff = int(total - sizes.sum())
        if diff == 0:
            return sizes
        free = sizes > lo if diff < 0 else sizes < hi
        adj = _largest_remainder(np.ones(int(free.sum())), abs(diff))
        sizes[free] += np.sign(diff) * adj
    raise ValueError("cannot fit block sizes into the requested range")


def _ptr(sizes: np.ndarray) -> np.ndarray:
    p = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=p[1:])
    return p


def _draw_column_rows(rng, col_block, row_ptr, per_col, p_in):
    """Rows of every column: ``per_col`` distinct rows, each inside the
    column's own row block with probability ``p_in`` (uniform there), else
    uniform over the rows outside that block."""
    n = len(col_block)
    m = int(row_ptr[-1])
    lo = row_ptr[col_block][:, None]
    hi = row_ptr[col_block + 1][:, None]
    msize = hi - lo
    inside = rng.random((n, per_col)) < p_in
    rows = np.empty((n, per_col), dtype=np.int64)

    def fill(mask):
        k = int(mask.sum())
        u = rng.random(k)
        lo_m = np.broadcast_to(lo, mask.shape)[mask]
        ms = np.broadcast_to(msize, mask.shape)[mask]
        ins = inside[mask]
        r_in = lo_m + np.minimum((u * ms).astype(np.int64), ms - 1)
        outside = m - ms
        r_out = np.minimum((u * np.maximum(outside, 1)).astype(np.int64), np.maximum(outside - 1, 0))
        r_out = np.where(r_out >= lo_m, r_out + ms, r_out)
        rows[mask] = np.where(ins | (outside == 0), r_in, r_out)

    fill(np.ones((n, per_col), dtype=bool))
    for _ in range(10000):
        srt = np.sort(rows, axis=1)
        dup_sorted = np.zeros_like(srt, dtype=bool)
        dup_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
        if not dup_sorted.any():
            return srt
        # redraw the later copies of a duplicated row (positions in sorted order)
        order = np.argsort(rows, axis=1, kind="stable")
        redo = np.zeros_like(dup_sorted)
        np.put_along_axis(redo, order, dup_sorted, axis=1)
        fill(redo)
    raise RuntimeError("could not draw distinct rows")


def _csr_from_columns(m: int, n: int, rows_by_col: np.ndarray, vals_by_col: np.ndarray) -> Csr:
    """CSR of a matrix given, for each column j, its row indices (sorted)."""
    per_col = rows_by_col.shape[1]
    r = rows_by_col.reshape(-1)
    c = np.repeat(np.arange(n, dtype=np.int64), per_col)
    v = vals_by_col.reshape(-1)
    order = np.argsort(r, kind="stable")  # stable: columns stay ascending in a row
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=rowptr[1:])
    return Csr(m, n, rowptr, c[order].astype(np.int32), v[order].astype(np.float64))


def _log_uniform(rng, lo: float, hi: float, size) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def staircase(rng, row_sizes, col_sizes, per_col: int, p_in: float) -> Csr:
    """Staircase matrix: column block b's nonzeros fall mostly in row block b."""
    row_ptr = _ptr(np.asarray(row_sizes))
    col_ptr = _ptr(np.asarray(col_sizes))
    n = int(col_ptr[-1])
    m = int(row_ptr[-1])
    col_block = np.repeat(np.arange(len(col_sizes)), np.asarray(col_sizes))
    rows = _draw_column_rows(rng, col_block, row_ptr, per_col, p_in)
    vals = rng.standard_normal(rows.shape)
    return _csr_from_columns(m, n, rows, vals)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def config1(seed: int = 1, m: int = 2000, n: int = 5000, per_col: int = 5, nblocks: int = 4) -> NormalProblem:
    """Random LP matrix, uniform rows per column; 4 equal row blocks."""
    rng = np.random.default_rng(seed)
    A = staircase(rng, [m], [n], per_col, 1.0)
    theta = _log_uniform(rng, 1e-2, 1e2, n)
    b = rng.standard_normal(m)
    block_ptr = np.array([(k * m) // nblocks for k in range(nblocks + 1)], dtype=np.int64)
    return NormalProblem(A, theta, b, block_ptr, rho=1e-6, tau=1e-3, delta=1e-12, maxit=2000,
                         name=f"random-LP {m}x{n} {per_col}/col, {nblocks} equal blocks")


def config2(seed: int = 2, scale: float = 1.0) -> NormalProblem:
    """Staircase 200k x 500k, 64 uneven blocks in [1k, 6k] rows, 8/col, 90 % in-block."""
    rng = np.random.default_rng(seed)
    nb = 64
    m = int(round(200_000 * scale))
    lo, hi = max(1, int(round(1000 * scale))), max(1, int(round(6000 * scale)))
    raw = rng.integers(lo, hi + 1, nb)
    row_sizes = _sizes_in_range(raw, m, lo, hi)
    n = int(round(2.5 * m))
    col_sizes = _largest_remainder(row_sizes, n)
    A = staircase(rng, row_sizes, col_sizes, 8, 0.9)
    theta = _log_uniform(rng, 1e-3, 1e3, n)
    b = rng.standard_normal(m)
    return NormalProblem(A, theta, b, _ptr(row_sizes), rho=1e-6, tau=1e-3, delta=1e-4, maxit=2000,
                         name=f"staircase {m}x{n} 8/col 90% in-block, {nb} uneven blocks")


def config4_structure(seed: int = 4, scale: float = 1.0, nblocks: int = 256):
    """Staircase 2M x 5M, 6/col, equal blocks; returns (A, theta0, g, b, block_ptr)."""
    rng = np.random.default_rng(seed)
    m = int(round(2_000_000 * scale))
    n = int(round(2.5 * m))
    row_sizes = _largest_remainder(np.ones(nblocks), m)
    col_sizes = _largest_remainder(row_sizes, n)
    A = staircase(rng, row_sizes, col_sizes, 6, 0.9)
    theta0 = _log_uniform(rng, 1e-1, 1e1, n)
    g = rng.normal(0.0, 0.5, n)
    b = rng.standard_normal(m)
    return A, theta0, g, b, _ptr(row_sizes)


def drift_theta(theta0: np.ndarray, g: np.ndarray, k: int) -> np.ndarray:
    """theta_k = clamp(theta_0 * exp(k g), 1e-8, 1e8): the IPM-like drift of the scaling."""
    return np.clip(theta0 * np.exp(k * g), 1e-8, 1e8)


def config4(seed: int = 4, scale: float = 1.0, nblocks: int = 256, steps: int = 30):
    """IPM sequence: one A, ``steps`` theta vectors.  Returns (NormalProblem for
    step 0, list of theta_k)."""
    A, theta0, g, b, block_ptr = config4_structure(seed, scale, nblocks)
    thetas = [drift_theta(theta0, g, k) for k in range(steps)]
    prob = NormalProblem(A, thetas[0], b, block_ptr, rho=1e-6, tau=1e-3, delta=1e-12, maxit=2000,
                         name=f"staircase {A.nrows}x{A.ncols} 6/col, {nblocks} blocks, {steps} IPM steps")
    return prob, thetas


def config3(seed: int = 3, scale: float = 1.0, nblocks: int = 128, nlink: int = 2048,
            link_frac: float = 0.02) -> AugmentedProblem:
    """Block-angular LP in augmented form, BBD order (x_k, lambda_k per block, border last)."""
    rng = np.random.default_rng(seed)
    lo, hi = max(2, int(round(2000 * scale))), max(2, int(round(20000 * scale)))
    msz = rng.integers(lo, hi + 1, nblocks).astype(np.int64)
    nsz = np.maximum(1, np.round(1.5 * msz).astype(np.int64))
    per_col = min(6, int(msz.min()))
    # diagonal blocks: 6 distinct in-block rows per column
    blockA = staircase(rng, msz, nsz, per_col, 1.0)
    n = int(nsz.sum())
    m_int = int(msz.sum())
    # linking rows: every (link row, column) pair present with probability link_frac
    cnt = rng.binomial(nlink, link_frac, n)
    tot = int(cnt.sum())
    lcol = np.repeat(np.arange(n, dtype=np.int64), cnt)
    lrow = rng.integers(0, nlink, tot)
    for _ in range(10000):
        key = lcol * nlink + lrow
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(tot, dtype=bool)
        dup[order[1:]] = ks[1:] == ks[:-1]
        if not dup.any():
            break
        lrow[dup] = rng.integers(0, nlink, int(dup.sum()))
    key = lrow * n + lcol
    order = np.argsort(key, kind="stable")
    lrow, lcol = lrow[order], lcol[order]
    lval = rng.standard_normal(tot)
    # stack [blockA; link]
    m = m_int + nlink
    rowptr = np.zeros(m + 1, dtype=np.int64)
    rowptr[: m_int + 1] = blockA.rowptr
    rowptr[m_int + 1:] = blockA.nnz + np.cumsum(np.bincount(lrow, minlength=nlink))
    col = np.concatenate([blockA.col, lcol.astype(np.int32)])
    val = np.concatenate([blockA.val, lval])
    A = Csr(m, n, rowptr, col, val)
    theta = _log_uniform(rng, 1e-8, 1e8, n)
    b = rng.standard_normal(n + m)
    return AugmentedProblem(A, theta, b, _ptr(msz), _ptr(nsz), nlink, rho=1e-8, tau=1e-3, delta=1e-12,
                            name=f"block-angular {m}x{n}, {nblocks} blocks + {nlink} linking rows, KKT form")


@dataclasses.dataclass
class Request:
    arrival_s: float
    problem: NormalProblem
    followups: list  # list of theta vectors for the follow-up solves


def serving_request(rng, arrival_s: float, m_lo: int = 1000, m_hi: int = 500_000) -> Request:
    m = int(round(float(_log_uniform(rng, m_lo, m_hi, 1)[0])))
    n = int(round(2.5 * m))
    per_col = int(rng.integers(5, 9))
    nb = max(1, math.ceil(m / 4000))
    row_sizes = _largest_remainder(np.ones(nb), m)
    col_sizes = _largest_remainder(row_sizes, n)
    A = staircase(rng, row_sizes, col_sizes, min(per_col, m), 0.9 if nb > 1 else 1.0)
    theta = _log_uniform(rng, 1e-4, 1e4, n)
    b = rng.standard_normal(m)
    nf = int(rng.integers(1, 11))
    thetas = []
    t = theta
    for _ in range(nf):
        t = np.clip(t * np.exp(rng.normal(0.0, 0.5, n)), 1e-8, 1e8)
        thetas.append(t)
    prob = NormalProblem(A, theta, b, _ptr(row_sizes), rho=1e-6, tau=1e-3, delta=1e-12, maxit=2000,
                         name=f"request m={m}")
    return Request(arrival_s, prob, thetas)


def serving_arrivals(seed: int = 5, count: int = 2000, rate: float = 200.0) -> np.ndarray:
    """Poisson arrival times (exponential gaps) of the request stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))


def serving_requests(seed: int = 5, count: int = 2000, rate: float = 200.0, m_lo: int = 1000,
                     m_hi: int = 500_000):
    """Yield requests one by one (drawn lazily: the full stream is large)."""
    arrivals = serving_arrivals(seed, count, rate)
    rng = np.random.default_rng(seed + 1000)
    for t in arrivals:
        yield serving_request(rng, float(t), m_lo, m_hi)
