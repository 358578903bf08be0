"""The seeded input generators produce the stated workloads: shapes, densities,
block structure, value and scaling ranges, and determinism (CPU only)."""
import numpy as np

from paper_2604_23979_gb300 import workloads as W


def col_counts(A):
    return np.bincount(A.col, minlength=A.ncols)


def rows_of_columns(A):
    """(row, col) pairs of A."""
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    return rows, A.col


def test_csr_is_well_formed():
    for A in (W.config1().A, W.config2(scale=0.05).A, W.config3(scale=0.01).A):
        assert A.rowptr[0] == 0 and np.all(np.diff(A.rowptr) >= 0) and A.rowptr[-1] == len(A.col)
        for i in range(0, A.nrows, max(1, A.nrows // 50)):
            c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
            assert np.all(np.diff(c) > 0), "columns sorted, no duplicates"
        assert A.col.min() >= 0 and A.col.max() < A.ncols


def test_config1_random_lp():
    p = W.config1()
    A = p.A
    assert (A.nrows, A.ncols) == (2000, 5000)
    assert np.all(col_counts(A) == 5)
    assert np.array_equal(p.block_ptr, [0, 500, 1000, 1500, 2000])
    assert 1e-2 <= p.theta.min() and p.theta.max() <= 1e2
    assert (p.rho, p.tau, p.delta, p.rtol, p.maxit) == (1e-6, 1e-3, 1e-12, 1e-8, 2000)


def test_config2_staircase():
    p = W.config2(scale=0.25)
    A = p.A
    assert (A.nrows, A.ncols) == (50000, 125000)
    sizes = np.diff(p.block_ptr)
    assert len(sizes) == 64 and sizes.sum() == 50000
    assert sizes.min() >= 250 and sizes.max() <= 1500
    assert np.all(col_counts(A) == 8)
    # about 90 % of a column's entries fall in the column's own row block
    col_sizes = W._largest_remainder(sizes, A.ncols)  # column blocks as the generator draws them
    assert col_sizes.sum() == A.ncols
    col_block = np.repeat(np.arange(64), col_sizes)
    rows, cols = rows_of_columns(A)
    row_block = np.searchsorted(p.block_ptr, rows, side="right") - 1
    frac = np.mean(row_block == col_block[cols])
    assert 0.88 <= frac <= 0.92, frac
    assert 1e-3 <= p.theta.min() and p.theta.max() <= 1e3
    assert p.delta == 1e-4


def test_config3_block_angular_kkt():
    p = W.config3(scale=0.02)
    A = p.A
    msz = np.diff(p.row_block_ptr)
    nsz = np.diff(p.col_block_ptr)
    assert len(msz) == 128 and np.all(nsz == np.maximum(1, np.round(1.5 * msz)))
    assert msz.min() >= 40 and msz.max() <= 400
    assert A.nrows == msz.sum() + p.nlink and A.ncols == nsz.sum()
    # every column: 6 in-block entries plus its linking-row entries
    rows, cols = rows_of_columns(A)
    inb = rows < msz.sum()
    assert np.all(np.bincount(cols[inb], minlength=A.ncols) == 6)
    links = np.bincount(cols[~inb], minlength=A.ncols)
    assert abs(links.mean() - 0.02 * p.nlink) < 0.1 * 0.02 * p.nlink
    assert 1e-8 <= p.theta.min() and p.theta.max() <= 1e8
    assert p.rho == 1e-8 and p.restart == 30


def test_config4_drift_is_clamped():
    A, theta0, g, b, bp = W.config4_structure(scale=0.01)
    assert np.all(col_counts(A) == 6) and len(bp) == 257
    assert 1e-1 <= theta0.min() and theta0.max() <= 1e1
    assert abs(g.std() - 0.5) < 0.05
    for k in (0, 5, 29):
        t = W.drift_theta(theta0, g, k)
        assert t.min() >= 1e-8 and t.max() <= 1e8
    assert np.array_equal(W.drift_theta(theta0, g, 0), np.clip(theta0, 1e-8, 1e8))


def test_serving_stream():
    arr = W.serving_arrivals(count=4000, rate=200.0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 1 / 200.0) < 0.05 / 200.0
    rng = np.random.default_rng(0)
    for _ in range(20):
        r = W.serving_request(rng, 0.0, 1000, 20000)
        A = r.problem.A
        assert 1000 <= A.nrows <= 20000 and A.ncols == round(2.5 * A.nrows)
        cc = col_counts(A)
        assert cc.min() == cc.max() and 5 <= cc[0] <= 8
        assert len(r.problem.block_ptr) - 1 == int(np.ceil(A.nrows / 4000))
        assert 1 <= len(r.followups) <= 10
        assert all(t.min() >= 1e-8 and t.max() <= 1e8 for t in r.followups)


def test_generators_are_deterministic():
    a, b = W.config2(scale=0.02), W.config2(scale=0.02)
    assert np.array_equal(a.A.col, b.A.col) and np.array_equal(a.A.val, b.A.val)
    assert np.array_equal(a.theta, b.theta) and np.array_equal(a.b, b.b)
