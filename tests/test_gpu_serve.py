"""Serving loop on the GPU: a stream of independent requests served with
continuous batching (overlapping streams, admission by memory) gives, for
every solve of every request, the same result as serving that request alone;
converged solves reach the FP64 true residual 1e-8 recomputed with the
oracle's system matrix."""
import numpy as np
import pytest

import oracle
from paper_2604_23979_gb300 import sdsl
from paper_2604_23979_gb300 import serve
from paper_2604_23979_gb300 import workloads as W
from tests.gpu_util import relres

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_23979_gb300 import build

    build.build()
    sdsl.load()


def stream(count=10, seed=7):
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(0.002, count))
    return [W.serving_request(rng, float(t), 1000, 20000) for t in arrivals]


def xs(results):
    return [[s.x for s in r.solves] for r in results]


def test_mix_equals_alone_and_meets_tolerance():
    reqs = stream()
    alone, _ = serve.GpuServer(slots=1, factor_prec=32, keep_x=True).serve(reqs)
    mixed, summ = serve.GpuServer(slots=4, factor_prec=32, keep_x=True).serve(reqs)
    assert summ["max_concurrency"] > 1, "the mix never overlapped"
    for ra, rm in zip(alone, mixed):
        assert len(ra.solves) == len(rm.solves) == 1 + len(reqs[ra.index].followups)
        for sa, sm in zip(ra.solves, rm.solves):
            assert sa.iters == sm.iters and sa.status == sm.status
            assert np.array_equal(sa.x, sm.x), f"request {ra.index}: result differs in the mix"
    # the first solve of every request against the oracle's S (FP64 true residual)
    for r in mixed:
        p = reqs[r.index].problem
        S = oracle.normal_matrix(p.A, p.theta, p.rho)
        s0 = r.solves[0]
        if s0.status == 0:
            assert relres(S, s0.x, p.b) <= p.rtol


def test_memory_budget_limits_the_mix():
    reqs = stream(count=6, seed=11)
    costs = [serve.footprint_bytes(r.problem.A, 32) for r in reqs]
    budget = 2 * max(costs)  # at most two of the largest at once
    alone, _ = serve.GpuServer(slots=1, factor_prec=32, keep_x=True).serve(reqs)
    srv = serve.GpuServer(slots=6, factor_prec=32, keep_x=True, budget_bytes=budget)
    mixed, summ = srv.serve(reqs, costs=costs)
    assert summ["requests"] == 6
    for ra, rm in zip(alone, mixed):
        for sa, sm in zip(ra.solves, rm.solves):
            assert np.array_equal(sa.x, sm.x)
    # the scheduler never charged more than the budget (its record after
    # every admission), and the measured charges that replaced the
    # estimates are smaller than them
    sched = srv.scheduler
    assert sched.charged and max(u for _, u in sched.charged) <= budget
    assert all(0 < c < e for c, e in zip(sched._costs, costs))


def test_measured_footprint_below_the_admission_estimate():
    """The handle's reported device memory: positive after setup, growing
    with the factorization, its peak at least its current holding, and below
    the column-count estimate the server admits a request on (so that the
    measured charge, which replaces the estimate, frees budget)."""
    rng = np.random.default_rng(5)
    for m_hi in (5000, 40000):
        req = W.serving_request(rng, 0.0, m_hi // 2, m_hi)
        prob = req.problem
        o, keep = sdsl.options_for(prob, factor_prec=32)
        h = sdsl.sdsl_setup(o, prob.A.nrows, prob.A.ncols, prob.A.rowptr, prob.A.col, prob.A.val, prob.theta)
        try:
            i0 = sdsl.sdsl_get_info(h)
            sdsl.sdsl_factor(h)
            i1 = sdsl.sdsl_get_info(h)
        finally:
            sdsl.sdsl_free(h)
        assert i0.device_bytes > 0 and i0.peak_device_bytes >= i0.device_bytes
        assert i1.device_bytes > i0.device_bytes and i1.peak_device_bytes >= i1.device_bytes
        est = serve.footprint_bytes(prob.A, 32)
        assert i1.peak_device_bytes < est, (i1.peak_device_bytes, est)
