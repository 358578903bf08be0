"""The allocation-free normal-equation product, through the C ABI, against the
handle API's sdsl_spmv and against the oracle's product with its own S =
A diag(theta) A^T + rho I.  It exists for callers that cannot allocate
device memory (a host program whose own pool holds the HBM, or a serving
loop where an allocation would synchronise the device), so the test also
checks that calls leave the device's free memory unchanged.  Collected last
on purpose: it must also pass after every other test has used the library
(and, run alone, in a fresh process)."""
import numpy as np
import pytest

import oracle
from paper_2604_23979_gb300 import sdsl
from paper_2604_23979_gb300 import workloads as W
from tests.gpu_util import rel, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_23979_gb300 import build

    build.build()
    sdsl.load()


def csr_transpose(A):
    """A^T in CSR by a stable sort of the entries on their column."""
    rows = np.repeat(np.arange(A.nrows, dtype=np.int64), np.diff(A.rowptr))
    order = np.argsort(A.col, kind="stable")
    trp = np.zeros(A.ncols + 1, np.int64)
    np.cumsum(np.bincount(A.col, minlength=A.ncols), out=trp[1:])
    return trp, rows[order].astype(np.int32), A.val[order]


def csr_mv(rp, ci, v, x, nrows):
    rows = np.repeat(np.arange(nrows), np.diff(rp))
    return np.bincount(rows, weights=v * x[ci], minlength=nrows)


def test_noalloc_matches_spmv_two_calls():
    import torch

    prob = W.config1()
    A = prob.A
    m, n, nnz = A.nrows, A.ncols, A.nnz
    trp, tci, tv = csr_transpose(A)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    d = [dev(a) for a in (A.rowptr, A.col, A.val, trp, tci, tv, prob.theta)]
    S = oracle.normal_matrix(A, prob.theta, prob.rho)  # the oracle's own S
    h, keep = setup(prob)
    try:
        rng = np.random.default_rng(11)
        for call in range(2):
            xh = rng.standard_normal(m) * (10.0 ** call)
            x = dev(xh)
            y = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
            r = torch.empty(m, dtype=torch.float64, device="cuda")
            sdsl.sdsl_normal_spmv_noalloc(m, n, nnz, *d, prob.rho, x, y)
            sdsl.sdsl_spmv(h, x, r)
            torch.cuda.synchronize()
            yh, rh = y.cpu().numpy(), r.cpu().numpy()
            assert np.all(np.isfinite(yh)), f"call {call}: unwritten outputs"
            # Same operator, different rounding order: within 1e-12 of the
            # componentwise magnitude |A| theta |A^T| |x| + rho |x|.
            mag = csr_mv(A.rowptr, A.col, np.abs(A.val),
                         prob.theta * csr_mv(trp, tci, np.abs(tv), np.abs(xh), n), m) + prob.rho * np.abs(xh)
            assert np.all(np.abs(yh - rh) <= 1e-12 * mag), f"call {call}"
            assert rel(yh, rh) <= 1e-12, f"call {call}"
            # and the oracle's product with its explicit S
            oh = oracle.spmv(S, xh)
            assert np.all(np.abs(yh - oh) <= 1e-12 * mag), f"call {call} vs oracle"
    finally:
        sdsl.sdsl_free(h)


def test_noalloc_calls_allocate_nothing():
    """After a first call (which may load the module and look up the scratch
    address), further calls leave the device's free memory unchanged."""
    import torch

    prob = W.config1()
    A = prob.A
    m, n, nnz = A.nrows, A.ncols, A.nnz
    trp, tci, tv = csr_transpose(A)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    d = [dev(a) for a in (A.rowptr, A.col, A.val, trp, tci, tv, prob.theta)]
    x = dev(np.random.default_rng(12).standard_normal(m))
    y = torch.empty(m, dtype=torch.float64, device="cuda")
    sdsl.sdsl_normal_spmv_noalloc(m, n, nnz, *d, prob.rho, x, y)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        sdsl.sdsl_normal_spmv_noalloc(m, n, nnz, *d, prob.rho, x, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_oversize():
    import torch

    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    n = sdsl.NOALLOC_MAX_COLS + 1
    with pytest.raises(sdsl.SdslError, match="scratch limit"):
        sdsl.sdsl_normal_spmv_noalloc(1, n, 1, z, z, z, z, z, z, z, 0.0, z, z)
