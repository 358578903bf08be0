"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
a dense numpy/scipy routine, a brute-force enumeration, a hand-worked example
(tests/golden/), a closed form or an invariant of the method.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg as sla

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_sparse(rng, m, n, per_col):
    d = np.zeros((m, n))
    for j in range(n):
        rows = rng.choice(m, size=min(per_col, m), replace=False)
        d[rows, j] = rng.standard_normal(len(rows))
    return d


# ---------------------------------------------------------------- Eq. (schur)

def test_transpose(orc):
    rng = np.random.default_rng(0)
    d = rand_sparse(rng, 9, 14, 3)
    T = orc.transpose(orc.from_dense(d))
    np.testing.assert_array_equal(T.dense(), d.T)


def test_normal_matrix_matches_dense_product(orc):
    rng = np.random.default_rng(1)
    d = rand_sparse(rng, 12, 30, 4)
    theta = np.exp(rng.uniform(-5, 5, 30))
    S = orc.normal_matrix(orc.from_dense(d), theta, 1e-6)
    ref = d @ np.diag(theta) @ d.T + 1e-6 * np.eye(12)
    np.testing.assert_allclose(S.dense(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    # structural pattern: (i, j) stored iff rows i, j share a column, plus the diagonal
    struct = ((np.abs(d) > 0).astype(int) @ (np.abs(d) > 0).T.astype(int) > 0) | np.eye(12, dtype=bool)
    assert (S.dense() != 0).sum() <= struct.sum()
    pat = np.zeros((12, 12), bool)
    for i in range(12):
        pat[i, S.col[S.rowptr[i]:S.rowptr[i + 1]]] = True
    np.testing.assert_array_equal(pat, struct)


def test_normal_matrix_exact_on_dyadic_values(orc):
    """Small integers and power-of-two theta: every product and sum is exact,
    so any dropped or duplicated term changes the result."""
    rng = np.random.default_rng(2)
    d = rng.integers(-3, 4, (8, 20)).astype(float) * (rng.random((8, 20)) < 0.4)
    theta = 2.0 ** rng.integers(-4, 5, 20)
    S = orc.normal_matrix(orc.from_dense(d), theta, 0.25)
    ref = d @ np.diag(theta) @ d.T + 0.25 * np.eye(8)
    np.testing.assert_array_equal(S.dense(), ref)


def test_normal_matrix_bitwise_symmetric(orc):
    rng = np.random.default_rng(3)
    d = rand_sparse(rng, 40, 100, 5)
    theta = np.exp(rng.uniform(-7, 7, 100))
    D = orc.normal_matrix(orc.from_dense(d), theta, 1e-6).dense()
    assert np.array_equal(D, D.T)


def test_normal_matrix_rounding_rule(orc):
    """Entry (i, j), i > j, equals fma-accumulated fl(a_ik theta_k) a_jk, k ascending."""
    rng = np.random.default_rng(4)
    d = rand_sparse(rng, 6, 40, 4)
    theta = np.exp(rng.uniform(-5, 5, 40))
    S = orc.normal_matrix(orc.from_dense(d), theta, 0.0).dense()
    from fractions import Fraction

    def fma(a, b, c):  # exact a*b+c rounded once (int/int true division rounds correctly)
        return float(Fraction(a) * Fraction(b) + Fraction(c))

    for i in range(6):
        for j in range(i + 1):
            acc = 0.0
            for k in range(40):
                if d[i, k] != 0 and d[j, k] != 0:
                    acc = fma(d[i, k] * theta[k], d[j, k], acc)
            if i == j:
                acc = acc + 0.0
            assert S[i, j] == acc and S[j, i] == acc


# ------------------------------------------------------- Eq. (augmented), BBD

def test_augmented_matches_block_form(orc):
    from paper_2604_23979_gb300 import workloads as W
    p = W.config3(scale=0.002, nblocks=3, nlink=4, link_frac=0.2)
    A = p.A
    K, pos, kbp = orc.augmented(A, p.theta, p.rho, p.row_block_ptr, p.col_block_ptr)
    Ad = orc.as_mat(A).dense()
    m, n = Ad.shape
    full = np.block([[-np.diag(1.0 / p.theta), Ad.T], [Ad, p.rho * np.eye(m)]])
    perm = np.empty(n + m, np.int64)
    perm[pos] = np.arange(n + m)
    np.testing.assert_array_equal(K.dense(), full[np.ix_(perm, perm)])
    # block k = [x_k; lambda_k] and the border (linking rows) last
    assert kbp[-1] == n + m - p.nlink
    for k in range(3):
        xs = np.arange(p.col_block_ptr[k], p.col_block_ptr[k + 1])
        ls = n + np.arange(p.row_block_ptr[k], p.row_block_ptr[k + 1])
        np.testing.assert_array_equal(pos[xs], kbp[k] + np.arange(len(xs)))
        np.testing.assert_array_equal(pos[ls], kbp[k] + len(xs) + np.arange(len(ls)))


# ------------------------------------------ Eq. (filter) and Eq. (diagcorr)

def _load_golden_filter():
    rows, kept, meta = {}, {}, {}
    with open(os.path.join(GOLDEN, "filter_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "row":
                i, vals = rest.split(":")
                rows[int(i)] = [float(x) for x in vals.split()]
            elif key == "kept":
                i, vals = rest.split(":")
                kept[int(i)] = [int(x) for x in vals.split()]
            elif key == "diag:":
                meta["diag"] = [float(x) for x in rest.split()]
            else:
                meta[key] = float(rest)
    n = int(meta["n"])
    return np.array([rows[i] for i in range(n)]), kept, meta


def test_filter_golden_hand_example(orc):
    A, kept, meta = _load_golden_filter()
    P = orc.filter_correct(orc.from_dense(A), np.array([0, len(A)]), meta["tau"], meta["delta"])
    for i in range(len(A)):
        assert list(P.col[P.rowptr[i]:P.rowptr[i + 1]]) == kept[i]
    np.testing.assert_array_equal(np.diag(P.dense()), meta["diag"])


def _brute_filter(D, bp, tau, delta):
    n = len(D)
    blk = np.searchsorted(bp, np.arange(n), side="right") - 1
    out = np.zeros_like(D)
    keep = np.zeros_like(D, dtype=bool)
    for i in range(n):
        for j in range(n):
            if blk[i] != blk[j]:
                continue
            if i == j:
                s = -1.0 if D[i, i] < 0 else 1.0
                out[i, i] = D[i, i] + delta * s
                keep[i, i] = True
            elif D[i, j] != 0:
                drop = abs(D[i, j]) < tau * abs(D[i, i]) and abs(D[i, j]) < tau * abs(D[j, j])
                if not drop:
                    out[i, j] = D[i, j]
                    keep[i, j] = True
    return out, keep


def _pattern(P):
    pat = np.zeros((P.nrows, P.ncols), bool)
    for i in range(P.nrows):
        pat[i, P.col[P.rowptr[i]:P.rowptr[i + 1]]] = True
    return pat


@pytest.mark.parametrize("seed", range(4))
def test_filter_bruteforce(orc, seed):
    rng = np.random.default_rng(10 + seed)
    n = 23
    D = rand_sparse(rng, n, n, 6) * np.exp(rng.uniform(-6, 6, (n, n)))
    D = D + D.T + np.diag(np.exp(rng.uniform(-3, 3, n)) * rng.choice([-1, 1], n))
    bp = np.array([0, 7, 15, n])
    tau, delta = 10.0 ** rng.uniform(-3, 0), 1e-3
    P = orc.filter_correct(orc.from_dense(D), bp, tau, delta)
    ref, keep = _brute_filter(D, bp, tau, delta)
    np.testing.assert_array_equal(_pattern(P), keep)
    np.testing.assert_array_equal(P.dense(), ref)


def test_filter_invariants(orc):
    rng = np.random.default_rng(20)
    n = 40
    D = rand_sparse(rng, n, n, 8) * np.exp(rng.uniform(-5, 5, (n, n)))
    D = D + D.T + np.diag(np.exp(rng.uniform(0, 3, n)))
    S = orc.from_dense(D)
    bp = np.array([0, 13, 27, n])
    pats = [_pattern(orc.filter_correct(S, bp, t, 0.0)) for t in (0.0, 1e-3, 1e-2, 1e-1, 1.0)]
    inblock = _pattern(orc.filter_correct(S, bp, 0.0, 0.0))
    blk = np.searchsorted(bp, np.arange(n), side="right") - 1
    assert np.array_equal(inblock, (D != 0) & (blk[:, None] == blk[None, :]) | np.eye(n, dtype=bool))
    for a, b in zip(pats, pats[1:]):  # larger tau keeps a subset
        assert not (b & ~a).any()
    for p in pats:  # every diagonal kept; symmetric input -> symmetric pattern
        assert p.diagonal().all()
        assert np.array_equal(p, p.T)
    # tau = 0, delta = 0 is the identity on the in-block entries
    P0 = orc.filter_correct(S, bp, 0.0, 0.0).dense()
    np.testing.assert_array_equal(P0, np.where(inblock, D, 0.0))
    # invariant under scaling by a power of two (exact)
    p1 = _pattern(orc.filter_correct(orc.from_dense(8.0 * D), bp, 1e-2, 0.0))
    assert np.array_equal(p1, pats[2])
    # filtering commutes with block extraction
    whole = orc.filter_correct(S, bp, 1e-2, 0.0, whole=True)
    assert np.array_equal(_pattern(whole) & (blk[:, None] == blk[None, :]), pats[2])


def test_diag_correction(orc):
    D = np.diag([2.0, -4.0, 0.0, 1.0]) + np.diag([0.5, 0.5, 0.5], 1) + np.diag([0.5, 0.5, 0.5], -1)
    S = orc.from_dense(D)
    S.col = S.col.astype(np.int32)
    # an explicitly stored zero diagonal
    Sz = orc.from_dense(D + np.diag([0, 0, 1.0, 0]))
    Sz.val[Sz.rowptr[2] + 1] = 0.0
    bp = np.array([0, 4])
    P = orc.filter_correct(Sz, bp, 0.0, 0.5)
    np.testing.assert_array_equal(np.diag(P.dense()), [2.5, -4.5, 0.5, 1.5])
    P0 = orc.filter_correct(Sz, bp, 0.0, 0.0)
    np.testing.assert_array_equal(P0.dense(), Sz.dense())
    # off-diagonals never corrected
    np.testing.assert_array_equal(P.dense() - np.diag(np.diag(P.dense())), D - np.diag(np.diag(D)))


# ------------------------------------------------------------ level sets

def _brute_levels(pat, bp):
    n = len(pat)
    lo = -np.ones(n, int)
    up = -np.ones(n, int)
    for b in range(len(bp) - 1):
        s, e = bp[b], bp[b + 1]

        def lev_lo(i, memo={}):
            deps = [j for j in range(s, i) if pat[i, j]]
            return 0 if not deps else 1 + max(lev_lo(j) for j in deps)

        def lev_up(i):
            deps = [j for j in range(i + 1, e) if pat[i, j]]
            return 0 if not deps else 1 + max(lev_up(j) for j in deps)

        for i in range(s, e):
            lo[i] = lev_lo(i)
            up[i] = lev_up(i)
    return lo, up


@pytest.mark.parametrize("seed", range(3))
def test_levels_bruteforce(orc, seed):
    rng = np.random.default_rng(30 + seed)
    n = 18
    pat = rng.random((n, n)) < 0.2
    pat = pat | pat.T | np.eye(n, dtype=bool)
    D = np.where(pat, 1.0, 0.0)
    bp = np.array([0, 8, n])
    lo, up = orc.levels(orc.from_dense(D), bp)
    blo, bup = _brute_levels(pat, bp)
    np.testing.assert_array_equal(lo, blo)
    np.testing.assert_array_equal(up, bup)
    nlev, lptr, rows = orc.level_lists(bp, lo)
    assert list(nlev) == [blo[:8].max() + 1, blo[8:].max() + 1]
    at = 0
    for b in range(2):
        for L in range(nlev[b]):
            seg = rows[lptr[at]:lptr[at + 1]]
            assert list(seg) == sorted(i for i in range(bp[b], bp[b + 1]) if blo[i] == L)
            at += 1


def test_levels_special_cases(orc):
    n = 12
    tri = np.eye(n) * 4 + np.eye(n, k=1) + np.eye(n, k=-1)
    lo, up = orc.levels(orc.from_dense(tri), np.array([0, n]))
    np.testing.assert_array_equal(lo, np.arange(n))
    np.testing.assert_array_equal(up, np.arange(n)[::-1])
    lo, up = orc.levels(orc.from_dense(np.eye(n)), np.array([0, n]))
    assert (lo == 0).all() and (up == 0).all()
    # two blocks of the tridiagonal: the coupling entry is ignored
    lo, _ = orc.levels(orc.from_dense(tri), np.array([0, 5, n]))
    np.testing.assert_array_equal(lo, np.r_[np.arange(5), np.arange(n - 5)])


# ------------------------------------------------------------ IC(0), ILU(0)

def spd(rng, n, density=0.3):
    M = rand_sparse(rng, n, n, max(1, int(density * n)))
    return M @ M.T + n * np.eye(n)


def test_ic0_tridiagonal_equals_cholesky(orc):
    n = 30
    T = 4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    P = orc.from_dense(T)
    F, alpha, st = orc.ic0(P, np.array([0, n]))
    assert st == 0 and alpha[0] == 0.0
    L = np.tril(orc.Mat(n, n, P.rowptr, P.col, F).dense())
    np.testing.assert_allclose(L, np.linalg.cholesky(T), rtol=1e-14, atol=1e-15)


def test_ic0_dense_block_equals_cholesky(orc):
    rng = np.random.default_rng(40)
    n = 16
    D = spd(rng, n, 1.0)
    D = D + 0.0 * np.ones((n, n))  # fully dense pattern
    D[D == 0] = 1e-30
    P = orc.from_dense(D)
    F, _, st = orc.ic0(P, np.array([0, n]))
    L = np.tril(orc.Mat(n, n, P.rowptr, P.col, F).dense())
    np.testing.assert_allclose(L, np.linalg.cholesky(D), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_ic0_reproduces_pattern_entries(orc, seed):
    """(L L^T)_ij = p_ij for every (i, j) in the pattern (IC(0) property)."""
    rng = np.random.default_rng(50 + seed)
    n = 40
    D = spd(rng, n, 0.08)
    bp = np.array([0, 17, n])
    P = orc.filter_correct(orc.from_dense(D), bp, 0.0, 0.0)
    F, alpha, st = orc.ic0(P, bp)
    assert st == 0 and (alpha == 0).all()
    L = np.tril(orc.Mat(n, n, P.rowptr, P.col, F).dense())
    LLt = L @ L.T
    pat = _pattern(P)
    np.testing.assert_allclose(LLt[pat], P.dense()[pat], rtol=1e-12, atol=1e-12)
    assert np.all(L[np.tril(~pat)] == 0)


def test_ic0_tau0_one_block_is_unfiltered(orc):
    """Invariant: drop tolerance 0 and one block reproduce the plain IC(0) of S."""
    from paper_2604_23979_gb300 import workloads as W
    p = W.config1(m=300, n=750)
    S = orc.normal_matrix(p.A, p.theta, p.rho)
    bp = np.array([0, S.nrows])
    P = orc.filter_correct(S, bp, 0.0, 0.0)
    assert np.array_equal(P.rowptr, S.rowptr) and np.array_equal(P.col, S.col)
    assert np.array_equal(P.val, S.val)


def test_ic0_shift_retry_and_breakdown(orc):
    # tridiagonal (fill-closed) with eigenvalues 1 +- 0.9*sqrt(2): indefinite.
    # By hand: alpha = 0, 1e-3, 1e-2, 1e-1 leave the last pivot negative
    # (e.g. alpha = 0.1: d_2 = 1.1 - (0.9/sqrt(1.1 - 0.81/1.1))^2 < 0); alpha = 1
    # gives pivots 2, 2 - 0.405, 2 - 0.508 > 0.
    A = np.array([[1.0, 0.9, 0.0], [0.9, 1.0, 0.9], [0.0, 0.9, 1.0]])
    F, alpha, st = orc.ic0(orc.from_dense(A), np.array([0, 3]))
    assert st == 0 and alpha[0] == 1.0
    # with the shift the factor reproduces A + alpha diag(A) on the pattern
    Ash = A + alpha[0] * np.diag(np.diag(A))
    P = orc.from_dense(A)
    L = np.tril(orc.Mat(3, 3, P.rowptr, P.col, F).dense())
    np.testing.assert_allclose((L @ L.T)[A != 0], Ash[A != 0], rtol=1e-14)
    # a negative diagonal defeats every shift
    F, alpha, st = orc.ic0(orc.from_dense(-np.eye(3)), np.array([0, 3]))
    assert st == orc.BREAKDOWN and alpha[0] == -1


def test_ilu0_shift_retry_and_breakdown(orc):
    """The ILU(0) shift ladder (the breakdown rule for the BBD block factors).

    By hand, in exact dyadic arithmetic: A = [[1,1,0],[1,2,1],[0,1,1]] is
    tridiagonal (fill-closed, so ILU(0) = LU without pivoting) with u11 = 1,
    l21 = 1, u22 = 2 - 1 = 1, l32 = 1, u33 = 1 - 1 = 0: the unshifted factor
    has a zero last pivot.  With alpha = 1e-3 the diagonal becomes 1.001,
    2.002, 1.001 and u33 = 1.001 - 1/(2.002 - 1/1.001) ~ 0.004 != 0, so the
    ladder stops at its second rung."""
    A = np.array([[1.0, 1.0, 0.0], [1.0, 2.0, 1.0], [0.0, 1.0, 1.0]])
    P = orc.from_dense(A)
    # the unshifted rung alone breaks down (zero pivot, not a non-finite one)
    F0, alpha0, st0 = orc.ilu0(P, np.array([0, 3]), shifts=[0.0])
    assert st0 == orc.BREAKDOWN and alpha0[0] == -1
    F, alpha, st = orc.ilu0(P, np.array([0, 3]))
    assert st == 0 and alpha[0] == 1e-3
    # the factor reproduces the shifted matrix A + alpha diag(A) on the pattern
    Ash = A + 1e-3 * np.diag(np.diag(A))
    Fm = orc.Mat(3, 3, P.rowptr, P.col, F).dense()
    L = np.tril(Fm, -1) + np.eye(3)
    U = np.triu(Fm)
    np.testing.assert_allclose((L @ U)[A != 0], Ash[A != 0], rtol=1e-13)
    u33 = 1.001 - 1.0 / (2.002 - 1.0 / 1.001)
    np.testing.assert_allclose(U[2, 2], u33, rtol=1e-10)
    # a second block that needs no shift keeps alpha = 0 (the rule is per block)
    B = np.zeros((5, 5))
    B[:3, :3] = A
    B[3:, 3:] = [[4.0, 1.0], [1.0, 4.0]]
    F2, alpha2, st2 = orc.ilu0(orc.from_dense(B), np.array([0, 3, 5]))
    assert st2 == 0 and list(alpha2) == [1e-3, 0.0]
    # a zero diagonal defeats every shift (alpha p_ii = 0): breakdown
    F, alpha, st = orc.ilu0(orc.from_dense(np.array([[0.0, 1.0], [1.0, 0.0]])), np.array([0, 2]))
    assert st == orc.BREAKDOWN and alpha[0] == -1
    # a non-finite pivot is a breakdown too (l21 overflows for every shift)
    F, alpha, st = orc.ilu0(orc.from_dense(np.array([[1e-300, 1e300], [1e300, 1.0]])), np.array([0, 2]))
    assert st == orc.BREAKDOWN and alpha[0] == -1


def test_ilu0_dense_equals_lu(orc):
    rng = np.random.default_rng(60)
    n = 14
    D = rng.standard_normal((n, n)) + 3 * n * np.eye(n)  # no pivoting needed
    P = orc.from_dense(D)
    F, alpha, st = orc.ilu0(P, np.array([0, n]))
    assert st == 0
    Fm = orc.Mat(n, n, P.rowptr, P.col, F).dense()
    L = np.tril(Fm, -1) + np.eye(n)
    U = np.triu(Fm)
    perm, Lr, Ur = sla.lu(D)
    assert np.array_equal(perm, np.eye(n))
    np.testing.assert_allclose(L, Lr, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(U, Ur, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_ilu0_reproduces_pattern_entries(orc, seed):
    rng = np.random.default_rng(70 + seed)
    n = 35
    D = rand_sparse(rng, n, n, 4) + 6 * np.eye(n)
    D = D + (D.T != 0) * 1e-3  # symmetric pattern, nonsymmetric values
    bp = np.array([0, 20, n])
    P = orc.filter_correct(orc.from_dense(D), bp, 0.0, 0.0)
    F, alpha, st = orc.ilu0(P, bp)
    assert st == 0
    Fm = orc.Mat(n, n, P.rowptr, P.col, F).dense()
    LU = (np.tril(Fm, -1) + np.eye(n)) @ np.triu(Fm)
    pat = _pattern(P)
    np.testing.assert_allclose(LU[pat], P.dense()[pat], rtol=1e-12, atol=1e-12)


def test_ic0_apply_is_block_triangular_solve(orc):
    rng = np.random.default_rng(80)
    n = 30
    D = spd(rng, n, 0.1)
    bp = np.array([0, 11, n])
    P = orc.filter_correct(orc.from_dense(D), bp, 0.0, 0.0)
    F, _, _ = orc.ic0(P, bp)
    L = np.tril(orc.Mat(n, n, P.rowptr, P.col, F).dense())
    r = rng.standard_normal(n)
    z = orc.ic0_apply(P, F, bp, r)
    np.testing.assert_allclose(z, np.linalg.solve(L @ L.T, r), rtol=1e-11)
    # block-diagonal: no coupling between blocks
    assert np.all((L @ L.T)[:11, 11:] == 0)


# ------------------------------------------------------------ PCG, GMRES

def test_pcg_diagonal_converges_in_one_iteration(orc):
    n = 25
    rng = np.random.default_rng(90)
    S = orc.from_dense(np.diag(np.exp(rng.uniform(-5, 5, n))))
    bp = np.array([0, 10, n])
    P = orc.filter_correct(S, bp, 1e-3, 0.0)
    F, _, _ = orc.ic0(P, bp)
    b = rng.standard_normal(n)
    res = orc.pcg_bj(S, P, F, bp, b)
    assert res.status == 0 and res.iters == 1
    np.testing.assert_allclose(res.x, b / np.diag(S.dense()), rtol=1e-14)


def test_pcg_exact_ic0_one_iteration(orc):
    """Tridiagonal S, one block, tau = 0: IC(0) is the exact Cholesky factor."""
    n = 50
    T = 3 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    S = orc.from_dense(T)
    bp = np.array([0, n])
    P = orc.filter_correct(S, bp, 0.0, 0.0)
    F, _, _ = orc.ic0(P, bp)
    b = np.random.default_rng(91).standard_normal(n)
    res = orc.pcg_bj(S, P, F, bp, b)
    assert res.status == 0 and res.iters == 1 and res.relres_true <= 1e-8


def test_pcg_matches_dense_solve(orc):
    from paper_2604_23979_gb300 import workloads as W
    p = W.config1(m=200, n=500)
    st, res = orc.bj_solve(p)
    Sd = st.S.dense()
    ref = np.linalg.solve(Sd, p.b)
    assert res.status == 0 and res.relres_true <= 1e-8
    assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) <= 1e-6
    assert np.linalg.norm(p.b - Sd @ res.x) / np.linalg.norm(p.b) == pytest.approx(res.relres_true, rel=1e-6)


def test_pcg_without_preconditioner_is_cg_bound(orc):
    """Identity blocks (1x1 blocks => Jacobi): CG on n=30 converges within n steps."""
    rng = np.random.default_rng(92)
    n = 30
    D = spd(rng, n, 0.2)
    S = orc.from_dense(D)
    bp = np.arange(n + 1)
    P = orc.filter_correct(S, bp, 0.0, 0.0)
    F, _, _ = orc.ic0(P, bp)
    res = orc.pcg_bj(S, P, F, bp, rng.standard_normal(n), rtol=1e-10)
    assert res.status == 0 and res.iters <= n + 2
    np.testing.assert_allclose(D @ res.x, orc.spmv(S, res.x), rtol=1e-13)


def test_pcg_edge_cases(orc):
    n = 10
    S = orc.from_dense(2 * np.eye(n))
    bp = np.array([0, n])
    P = orc.filter_correct(S, bp, 0.0, 0.0)
    F, _, _ = orc.ic0(P, bp)
    res = orc.pcg_bj(S, P, F, bp, np.zeros(n))
    assert res.status == 0 and res.iters == 0 and not res.x.any()
    b = np.ones(n)
    res = orc.pcg_bj(S, P, F, bp, b, x0=b / 2)  # exact initial guess
    assert res.status == 0 and res.iters == 0


def test_gmres_small_without_restart(orc):
    rng = np.random.default_rng(100)
    n = 25
    D = rng.standard_normal((n, n)) + 8 * np.eye(n)
    K = orc.from_dense(D)
    b = rng.standard_normal(n)
    res = orc.gmres(K, b, rtol=1e-12, restart=30)
    assert res.status == 0 and res.iters <= n
    np.testing.assert_allclose(res.x, np.linalg.solve(D, b), rtol=1e-9)


def test_gmres_exact_preconditioner_one_iteration(orc):
    rng = np.random.default_rng(101)
    n = 20
    D = rng.standard_normal((n, n)) + 8 * np.eye(n)
    K = orc.from_dense(D)
    bp = np.array([0, n])
    F, _, _ = orc.ilu0(K, bp)  # full pattern: ILU(0) = LU
    res = orc.gmres(K, rng.standard_normal(n), orc.PRE_BJ_ILU0, K, F, bp)
    assert res.status == 0 and res.iters == 1


def test_gmres_minimal_residual(orc):
    """GMRES property: after k steps of one cycle the iterate minimises
    ||b - K x|| over the Krylov space span{b, Kb, ..., K^(k-1) b}, and the
    Givens estimate |g_(k+1)| equals that residual."""
    rng = np.random.default_rng(103)
    n = 20
    D = rng.standard_normal((n, n)) + 3 * np.eye(n)
    K = orc.from_dense(D)
    b = rng.standard_normal(n)
    prev = np.inf
    for k in range(1, 9):
        res = orc.gmres(K, b, rtol=1e-300, maxit=k, restart=30)
        Kry = np.empty((n, k))
        v = b.copy()
        for j in range(k):
            Kry[:, j] = v
            v = D @ v
        Q, _ = np.linalg.qr(Kry)
        y, *_ = np.linalg.lstsq(D @ Q, b, rcond=None)
        best = np.linalg.norm(b - D @ Q @ y) / np.linalg.norm(b)
        assert res.iters == k
        assert res.relres_true == pytest.approx(best, rel=1e-7)
        assert res.relres_rec == pytest.approx(best, rel=1e-7)
        assert res.relres_true <= prev * (1 + 1e-12)
        prev = res.relres_true


def test_gmres_restarts(orc):
    rng = np.random.default_rng(102)
    n = 60
    D = rng.standard_normal((n, n)) + 4 * np.sqrt(n) * np.eye(n)
    K = orc.from_dense(D)
    b = rng.standard_normal(n)
    res = orc.gmres(K, b, rtol=1e-10, restart=5)
    assert res.status == 0 and res.iters > 5
    assert np.linalg.norm(b - D @ res.x) / np.linalg.norm(b) <= 1e-10


# ------------------------------------------- BiCGSTAB (Block Jacobi, Sec. 4.3)

def _distinct_eigen(rng, n, lams):
    """Non-symmetric, diagonalisable n x n matrix whose eigenvalues are the
    values of lams repeated (V diag V^-1 with a well-conditioned V)."""
    V = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    d = np.array([lams[i % len(lams)] for i in range(n)], float)
    return V @ np.diag(d) @ np.linalg.inv(V)


def test_bicgstab_identity_one_half_pass(orc):
    n = 12
    b = np.random.default_rng(110).standard_normal(n)
    res = orc.bicgstab(orc.from_dense(np.eye(n)), b)
    assert res.status == 0 and res.iters == 1
    np.testing.assert_array_equal(res.x, b)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_bicgstab_terminates_after_k_passes(orc, k):
    """k distinct eigenvalues: the BiCG residual polynomial of degree k
    annihilates r0, so the k-th pass ends at its first half with s = 0 (and
    not earlier for a generic right-hand side)."""
    rng = np.random.default_rng(111 + k)
    n = 24
    D = _distinct_eigen(rng, n, [1.0, 2.5, 4.0, 7.0][:k])
    b = rng.standard_normal(n)
    res = orc.bicgstab(orc.from_dense(D), b, rtol=1e-9)
    assert res.status == 0 and res.iters == k
    np.testing.assert_allclose(res.x, np.linalg.solve(D, b), rtol=1e-8, atol=1e-10)


def test_bicgstab_first_pass_is_galerkin_then_minimal_residual(orc):
    """After one pass from x0 = 0: s = b - alpha A b is the vector of that form
    orthogonal to the shadow b, and omega minimises ||s - omega A s||."""
    rng = np.random.default_rng(115)
    n = 30
    D = rng.standard_normal((n, n)) + 6 * np.eye(n)
    b = rng.standard_normal(n)
    res = orc.bicgstab(orc.from_dense(D), b, rtol=1e-300, maxit=1)
    assert res.status == 5 and res.iters == 1
    Ab = D @ b
    # the alpha with b^T (b - alpha A b) = 0 (the 1 x 1 Galerkin system)
    alpha = np.linalg.solve([[b @ Ab]], [b @ b])[0]
    s = b - alpha * Ab
    assert abs(b @ s) <= 1e-12 * np.linalg.norm(b) * np.linalg.norm(s)
    As = D @ s
    omega = np.linalg.lstsq(As[:, None], s, rcond=None)[0][0]
    r1 = s - omega * As
    assert res.relres_rec == pytest.approx(np.linalg.norm(r1) / np.linalg.norm(b), rel=1e-9)
    np.testing.assert_allclose(res.x, alpha * b + omega * s, rtol=1e-10, atol=1e-13)


def test_bicgstab_exact_preconditioner_one_pass(orc):
    """ILU(0) on the full pattern is the exact LU: M^-1 S = I, one half pass."""
    rng = np.random.default_rng(116)
    n = 20
    D = rng.standard_normal((n, n)) + 8 * np.eye(n)
    K = orc.from_dense(D)
    bp = np.array([0, n])
    F, _, _ = orc.ilu0(K, bp)
    b = rng.standard_normal(n)
    res = orc.bicgstab(K, b, orc.PRE_BJ_ILU0, K, F, bp)
    assert res.status == 0 and res.iters == 1
    np.testing.assert_allclose(res.x, np.linalg.solve(D, b), rtol=1e-10)


def test_bicgstab_recurrence_tracks_true_residual(orc):
    """With a Block-Jacobi IC(0) preconditioner, after k passes the recurrence
    residual equals ||b - S x|| (x and r are updated with the same steps)."""
    from paper_2604_23979_gb300 import workloads as W
    p = W.config1(m=200, n=500)
    st = orc.bj_setup_factor(p.A, p.theta, p.rho, p.block_ptr, p.tau, p.delta)
    Sd = st.S.dense()
    for k in (1, 3, 6):
        res = orc.bicgstab(st.S, p.b, orc.PRE_BJ_IC0, st.P, st.F, p.block_ptr, rtol=1e-300, maxit=k)
        assert res.iters == k
        true = np.linalg.norm(p.b - Sd @ res.x) / np.linalg.norm(p.b)
        assert res.relres_true == pytest.approx(true, rel=1e-9)
        assert res.relres_rec == pytest.approx(true, rel=1e-6, abs=1e-14)


def test_bicgstab_bj_matches_dense_solve(orc):
    from paper_2604_23979_gb300 import workloads as W
    p = W.config1(m=200, n=500)
    st = orc.bj_setup_factor(p.A, p.theta, p.rho, p.block_ptr, p.tau, p.delta)
    res = orc.bicgstab(st.S, p.b, orc.PRE_BJ_IC0, st.P, st.F, p.block_ptr, rtol=1e-8, maxit=2000)
    ref = np.linalg.solve(st.S.dense(), p.b)
    assert res.status == 0 and res.relres_true <= 1e-8
    assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) <= 1e-6
    # right preconditioning: no more passes than PCG needs products, twice over
    pcg = orc.pcg_bj(st.S, st.P, st.F, p.block_ptr, p.b)
    assert res.iters <= pcg.iters


def test_bicgstab_nonsymmetric_matches_dense_solve(orc):
    rng = np.random.default_rng(117)
    n = 40
    D = rng.standard_normal((n, n)) + 10 * np.eye(n)
    b = rng.standard_normal(n)
    res = orc.bicgstab(orc.from_dense(D), b, rtol=1e-12)
    assert res.status == 0
    np.testing.assert_allclose(res.x, np.linalg.solve(D, b), rtol=1e-9, atol=1e-12)


def test_bicgstab_edge_cases(orc):
    n = 10
    S = orc.from_dense(2 * np.eye(n))
    res = orc.bicgstab(S, np.zeros(n))
    assert res.status == 0 and res.iters == 0 and not res.x.any()
    b = np.ones(n)
    res = orc.bicgstab(S, b, x0=b / 2)
    assert res.status == 0 and res.iters == 0
    res = orc.bicgstab(S, b, maxit=0)
    assert res.status == 5 and res.iters == 0


# ------------------------------------------------------------ BBD (Sec. 2.4)

def _small_bbd(orc, seed=3):
    from paper_2604_23979_gb300 import workloads as W
    p = W.config3(seed=seed, scale=0.002, nblocks=3, nlink=5, link_frac=0.3)
    K, pos, kbp = orc.augmented(p.A, p.theta, p.rho, p.row_block_ptr, p.col_block_ptr)
    return p, K, kbp


def test_dense_lu_matches_scipy(orc):
    rng = np.random.default_rng(110)
    a = rng.standard_normal((33, 33))
    lu, ipiv, st = orc.dense_lu(a)
    ref_lu, ref_piv = sla.lu_factor(a)
    assert st == 0
    np.testing.assert_array_equal(ipiv, ref_piv)
    np.testing.assert_allclose(lu, ref_lu, rtol=1e-11, atol=1e-12)
    b = rng.standard_normal(33)
    np.testing.assert_allclose(orc.dense_lu_solve(lu, ipiv, b), np.linalg.solve(a, b), rtol=1e-10)


def test_bbd_schur_and_apply_match_dense(orc):
    p, K, kbp = _small_bbd(orc)
    N = K.nrows
    P = orc.filter_correct(K, kbp, p.tau, p.delta, whole=True)
    F, alpha, st = orc.ilu0(P, kbp)
    assert st == 0
    Pd = P.dense()
    Fd = orc.Mat(N, N, P.rowptr, P.col, F).dense()
    b0 = int(kbp[-1])
    # M = blockdiag(L_k U_k) on the interior, P elsewhere
    Mi = np.zeros((b0, b0))
    for k in range(len(kbp) - 1):
        s, e = kbp[k], kbp[k + 1]
        blk = Fd[s:e, s:e]
        Mi[s:e, s:e] = (np.tril(blk, -1) + np.eye(e - s)) @ np.triu(blk)
    E, Fb, Cb = Pd[:b0, b0:], Pd[b0:, :b0], Pd[b0:, b0:]
    ref = Cb - Fb @ np.linalg.solve(Mi, E)
    SB = orc.bbd_schur(P, F, kbp)
    np.testing.assert_allclose(SB, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    lu, ipiv, st = orc.dense_lu(SB)
    M = np.block([[Mi, E], [Fb, Cb]])
    r = np.random.default_rng(111).standard_normal(N)
    z = orc.bbd_apply(P, F, kbp, lu, ipiv, r)
    # backward error of the block solve (the KKT blocks span theta in [1e-8, 1e8])
    berr = np.abs(M @ z - r).max() / (np.abs(M).sum(axis=1).max() * np.abs(z).max() + np.abs(r).max())
    assert berr <= 1e-13


def test_bbd_exact_blocks_gmres_one_iteration(orc):
    """Blocks whose pattern is closed under elimination and tau = 0, delta = 0:
    the block LU is exact, so M = K and right-preconditioned GMRES stops after
    one step."""
    rng = np.random.default_rng(112)
    nb, bs, border = 3, 6, 4
    n = nb * bs + border
    D = np.zeros((n, n))
    for k in range(nb):
        s = k * bs
        D[s:s + bs, s:s + bs] = rng.standard_normal((bs, bs)) + 8 * np.eye(bs)  # dense blocks
    D[: nb * bs, nb * bs:] = rng.standard_normal((nb * bs, border)) * (rng.random((nb * bs, border)) < 0.5)
    D[nb * bs:, : nb * bs] = rng.standard_normal((border, nb * bs)) * (rng.random((border, nb * bs)) < 0.5)
    D[nb * bs:, nb * bs:] = rng.standard_normal((border, border)) + 8 * np.eye(border)
    K = orc.from_dense(D)
    kbp = np.arange(0, nb * bs + 1, bs)
    P = orc.filter_correct(K, kbp, 0.0, 0.0, whole=True)
    F, _, _ = orc.ilu0(P, kbp)
    lu, ipiv, _ = orc.dense_lu(orc.bbd_schur(P, F, kbp))
    b = rng.standard_normal(n)
    res = orc.gmres(K, b, orc.PRE_BBD, P, F, kbp, lu, ipiv)
    assert res.status == 0 and res.iters == 1
    np.testing.assert_allclose(res.x, np.linalg.solve(D, b), rtol=1e-9)


def test_bbd_gmres_small_kkt(orc):
    """A small KKT system of the block-angular shape with a mild scaling
    (theta in [1e-2, 1e2], rho = 1e-2): right-preconditioned GMRES(30) with the
    BBD preconditioner reaches the 1e-8 true residual."""
    from paper_2604_23979_gb300 import workloads as W
    p = W.config3(seed=5, scale=0.002, nblocks=3, nlink=5, link_frac=0.3)
    rng = np.random.default_rng(0)
    p.theta = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), len(p.theta)))
    p.rho = 1e-2
    K, pos, kbp = orc.augmented(p.A, p.theta, p.rho, p.row_block_ptr, p.col_block_ptr)
    P = orc.filter_correct(K, kbp, p.tau, p.delta, whole=True)
    F, alpha, st = orc.ilu0(P, kbp)
    lu, ipiv, _ = orc.dense_lu(orc.bbd_schur(P, F, kbp))
    res = orc.gmres(K, p.b, orc.PRE_BBD, P, F, kbp, lu, ipiv, maxit=3000)
    assert res.status == 0
    assert np.linalg.norm(p.b - K.dense() @ res.x) / np.linalg.norm(p.b) <= 1e-8


# ------------------------------------------------ GCR(m), "IGCR(m)" (Sec. 4.3)

def _krylov_min_residual(D, Minv, b, k):
    """min ||b - D Minv V y|| over the k-dimensional Krylov space of D Minv
    from b (right preconditioning), by a dense least-squares solve."""
    n = len(b)
    Kry = np.empty((n, k))
    v = b.copy()
    for j in range(k):
        Kry[:, j] = v
        v = D @ (Minv @ v)
    Q, _ = np.linalg.qr(Kry)
    y, *_ = np.linalg.lstsq(D @ Minv @ Q, b, rcond=None)
    return np.linalg.norm(b - D @ Minv @ Q @ y) / np.linalg.norm(b), Minv @ Q @ y


def test_gcr_minimal_residual(orc):
    """Each step of a cycle minimises ||b - K x|| over the Krylov space (the
    GMRES property); the recurrence residual is the same value."""
    rng = np.random.default_rng(120)
    n = 20
    D = rng.standard_normal((n, n)) + 3 * np.eye(n)
    K = orc.from_dense(D)
    b = rng.standard_normal(n)
    for k in range(1, 9):
        res = orc.gcr(K, b, rtol=1e-300, maxit=k, restart=30)
        best, xbest = _krylov_min_residual(D, np.eye(n), b, k)
        assert res.iters == k and res.status == 5
        assert res.relres_true == pytest.approx(best, rel=1e-7)
        assert res.relres_rec == pytest.approx(best, rel=1e-7)
        np.testing.assert_allclose(res.x, xbest, rtol=1e-7, atol=1e-10)


def test_gcr_right_preconditioned_minimal_residual(orc):
    """With a Block-Jacobi ILU(0) preconditioner (three blocks, not exact),
    the iterate is M^-1 times the minimiser over the Krylov space of K M^-1."""
    rng = np.random.default_rng(121)
    n = 24
    D = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.3) + 5 * np.eye(n)
    K = orc.from_dense(D)
    bp = np.array([0, 8, 15, n])
    F, _, _ = orc.ilu0(K, bp)
    Minv = np.column_stack([orc.precond_apply(orc.PRE_BJ_ILU0, K, F, bp, e) for e in np.eye(n)])
    b = rng.standard_normal(n)
    for k in (1, 3, 6):
        res = orc.gcr(K, b, orc.PRE_BJ_ILU0, K, F, bp, rtol=1e-300, maxit=k, restart=30)
        best, xbest = _krylov_min_residual(D, Minv, b, k)
        assert res.relres_true == pytest.approx(best, rel=1e-7)
        np.testing.assert_allclose(res.x, xbest, rtol=1e-7, atol=1e-10)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_gcr_terminates_after_k_steps(orc, k):
    rng = np.random.default_rng(122 + k)
    n = 24
    D = _distinct_eigen(rng, n, [1.0, 2.5, 4.0, 7.0][:k])
    b = rng.standard_normal(n)
    res = orc.gcr(orc.from_dense(D), b, rtol=1e-9)
    assert res.status == 0 and res.iters == k
    np.testing.assert_allclose(res.x, np.linalg.solve(D, b), rtol=1e-8, atol=1e-10)


def test_gcr_exact_preconditioner_one_step(orc):
    rng = np.random.default_rng(126)
    n = 20
    D = rng.standard_normal((n, n)) + 8 * np.eye(n)
    K = orc.from_dense(D)
    bp = np.array([0, n])
    F, _, _ = orc.ilu0(K, bp)
    res = orc.gcr(K, rng.standard_normal(n), orc.PRE_BJ_ILU0, K, F, bp)
    assert res.status == 0 and res.iters == 1


def test_gcr_restarts(orc):
    rng = np.random.default_rng(127)
    n = 60
    D = rng.standard_normal((n, n)) + 4 * np.sqrt(n) * np.eye(n)
    b = rng.standard_normal(n)
    res = orc.gcr(orc.from_dense(D), b, rtol=1e-10, restart=5)
    assert res.status == 0 and res.iters > 5
    assert np.linalg.norm(b - D @ res.x) / np.linalg.norm(b) <= 1e-10


def test_gcr_bbd_small_kkt(orc):
    """The BBD preconditioner on a small, mildly scaled KKT system: GCR(30)
    reaches the 1e-8 true residual and the dense solution."""
    from paper_2604_23979_gb300 import workloads as W
    p = W.config3(seed=5, scale=0.002, nblocks=3, nlink=5, link_frac=0.3)
    rng = np.random.default_rng(0)
    p.theta = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), len(p.theta)))
    p.rho = 1e-2
    K, pos, kbp = orc.augmented(p.A, p.theta, p.rho, p.row_block_ptr, p.col_block_ptr)
    P = orc.filter_correct(K, kbp, p.tau, p.delta, whole=True)
    F, alpha, st = orc.ilu0(P, kbp)
    lu, ipiv, _ = orc.dense_lu(orc.bbd_schur(P, F, kbp))
    res = orc.gcr(K, p.b, orc.PRE_BBD, P, F, kbp, lu, ipiv, maxit=3000)
    Kd = K.dense()
    assert res.status == 0
    assert np.linalg.norm(p.b - Kd @ res.x) / np.linalg.norm(p.b) <= 1e-8
    ref = np.linalg.solve(Kd, p.b)
    assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) <= 1e-5


def test_gcr_edge_cases(orc):
    n = 10
    S = orc.from_dense(2 * np.eye(n))
    res = orc.gcr(S, np.zeros(n))
    assert res.status == 0 and res.iters == 0 and not res.x.any()
    b = np.ones(n)
    res = orc.gcr(S, b, x0=b / 2)
    assert res.status == 0 and res.iters == 0
    res = orc.gcr(S, b, maxit=0)
    assert res.status == 5 and res.iters == 0
