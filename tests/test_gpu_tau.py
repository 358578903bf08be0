"""Filter threshold schedules (Sec. 4.2-4.3) through the C ABI: the
threshold set for the next build, the two-phase switch after a number of IPM
steps, and the relaxation of a filter under which a fresh preconditioner
fails -- each build's filtered pattern bit-exact against the oracle's filter
at that threshold, and the solves against the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2604_23979_gb300 import sdsl
from paper_2604_23979_gb300 import workloads as W
from tests.gpu_util import iters_close, relres, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_23979_gb300 import build

    build.build()
    sdsl.load()


def pattern_matches(h, prob, theta, tau):
    S = oracle.normal_matrix(prob.A, theta, prob.rho)
    P = oracle.filter_correct(S, prob.block_ptr, tau, prob.delta)
    prp, pci, pv, fv, alpha = sdsl.sdsl_export_precond(h)
    return np.array_equal(prp, P.rowptr) and np.array_equal(pci, P.col)


def test_set_tau_applies_to_the_next_build():
    prob = W.config1(m=600, n=1500)
    h, keep = setup(prob, 64)
    try:
        sdsl.sdsl_factor(h)
        assert pattern_matches(h, prob, prob.theta, prob.tau)
        sdsl.sdsl_set_tau(h, 0.05)
        assert pattern_matches(h, prob, prob.theta, prob.tau)  # kept until the next build
        sdsl.sdsl_factor(h)
        assert pattern_matches(h, prob, prob.theta, 0.05)
        x = np.zeros(len(prob.b))
        st = sdsl.sdsl_solve(h, prob.b, x)
        assert st.tau_used == 0.05 and st.status == 0
        ref = oracle.bj_setup_factor(prob.A, prob.theta, prob.rho, prob.block_ptr, 0.05, prob.delta)
        r = oracle.pcg_bj(ref.S, ref.P, ref.F, prob.block_ptr, prob.b, rtol=prob.rtol, maxit=prob.maxit)
        assert iters_close(st.iters, r.iters) and relres(ref.S, x, prob.b) <= 1e-8
        with pytest.raises(sdsl.SdslError):
            sdsl.sdsl_set_tau(h, -1.0)
    finally:
        sdsl.sdsl_free(h)


def test_two_phase_threshold_switch():
    """tau_switch_step = 2, tau_after = 1e-2: builds before the second IPM
    step filter at tau, builds from it on at 1e-2."""
    prob, thetas = W.config4(scale=0.002, nblocks=8, steps=4)
    h, keep = setup(prob, 64, tau_switch_step=2, tau_after=1e-2, refactor_ratio=0.0)
    try:
        sdsl.sdsl_factor(h)
        used = []
        for k, th in enumerate(thetas):
            if k:
                sdsl.sdsl_update_diag(h, th)
                sdsl.sdsl_factor(h)
            tau = prob.tau if k < 2 else 1e-2
            assert pattern_matches(h, prob, th, tau), k
            x = np.zeros(len(prob.b))
            st = sdsl.sdsl_solve(h, prob.b, x, allow=(sdsl.ERR_NOT_CONVERGED,))
            used.append(st.tau_used)
        assert used == [prob.tau, prob.tau, 1e-2, 1e-2]
    finally:
        sdsl.sdsl_free(h)


def test_relaxed_filter_after_a_failed_fresh_solve():
    """tau = 0.1 on the 5 % staircase: the oracle needs 1,184 iterations; with
    a cap of 1,000 the fresh preconditioner fails, and tau_relax = 0.1 rebuilds
    it at 0.01 (813 oracle iterations) and repeats the solve, which converges;
    the next build is back at 0.1."""
    prob = W.config2(scale=0.05)
    h, keep = setup(prob, 64, tau=0.1, tau_relax=0.1, maxit=1000, refactor_ratio=0.0)
    try:
        sdsl.sdsl_factor(h)
        x = np.zeros(len(prob.b))
        st = sdsl.sdsl_solve(h, prob.b, x)
        assert st.status == 0 and st.rebuilt == 1 and st.iters_discarded == 1000
        assert abs(st.tau_used - 0.01) <= 1e-15
        assert pattern_matches(h, prob, prob.theta, 0.1 * 0.1)
        ref = oracle.bj_setup_factor(prob.A, prob.theta, prob.rho, prob.block_ptr, 0.1 * 0.1, prob.delta)
        r = oracle.pcg_bj(ref.S, ref.P, ref.F, prob.block_ptr, prob.b, rtol=prob.rtol, maxit=3000)
        assert iters_close(st.iters, r.iters), (st.iters, r.iters)
        assert relres(ref.S, x, prob.b) <= 1e-8
        sdsl.sdsl_factor(h)  # the scheduled threshold again
        assert pattern_matches(h, prob, prob.theta, 0.1)
    finally:
        sdsl.sdsl_free(h)
