"""GPU parity of the Block-Jacobi path against the FP64 oracle, through the C ABI.

Bars: bit-exact system matrix, filtered pattern, corrected values, level sets
and shift decisions; factor values within a rounding tolerance; solutions with
a true relative residual <= 1e-8 (recomputed by the oracle's SpMV), within
1e-6 of the oracle's solution, and iteration counts within max(1, 5 %).
"""
import numpy as np
import pytest

import oracle
from paper_2604_23979_gb300 import sdsl
from paper_2604_23979_gb300 import workloads as W
from tests.gpu_util import iters_close, rel, relres, replay_reuse, run_bj, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_23979_gb300 import build

    build.build()
    sdsl.load()


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def check_structures(prob, ref, g):
    rp, ci, v = g["S"]
    assert np.array_equal(rp, ref.S.rowptr) and np.array_equal(ci, ref.S.col)
    assert np.array_equal(bits(v), bits(ref.S.val)), "S values differ bitwise"
    prp, pci, pv, fv, alpha = g["P"]
    assert np.array_equal(prp, ref.P.rowptr), "filtered row pointers differ"
    assert np.array_equal(pci, ref.P.col), "filtered pattern differs"
    assert np.array_equal(bits(pv), bits(ref.P.val)), "corrected values differ bitwise"
    assert np.array_equal(alpha, ref.alpha), "shift decisions differ"
    for which, lev in ((0, ref.lev_lo), (1, ref.lev_up)):
        nlev, lptr, rows = g["lev_lo"] if which == 0 else g["lev_up"]
        rn, rp_, rr = oracle.level_lists(prob.block_ptr, lev)
        assert np.array_equal(nlev, rn), f"level counts differ ({which})"
        assert np.array_equal(lptr, rp_), f"level pointers differ ({which})"
        assert np.array_equal(rows, rr), f"level rows differ ({which})"
    return fv


def check_factor(prob, ref, fv, tol):
    P = ref.P
    row = np.repeat(np.arange(P.nrows), np.diff(P.rowptr))
    low = P.col <= row
    for b in range(len(prob.block_ptr) - 1):
        s, e = prob.block_ptr[b], prob.block_ptr[b + 1]
        m = low & (row >= s) & (row < e)
        if m.any():
            assert rel(fv[m], ref.F[m]) <= tol, f"factor of block {b} off"


def check_solution(prob, ref_state, ref_res, g, iters_exact=True):
    st = g["stats"]
    assert st["status"] == 0, st
    x = g["x"]
    true_rel = relres(ref_state.S, x, prob.b)
    assert true_rel <= prob.rtol, true_rel
    assert rel(x, ref_res.x) <= 1e-6
    if iters_exact:
        assert iters_close(st["iters"], ref_res.iters), (st["iters"], ref_res.iters)


CASES = {
    "c1": lambda: W.config1(),
    "c1-small": lambda: W.config1(m=300, n=750),
    "c2-5pct": lambda: W.config2(scale=0.05),
}


@pytest.mark.parametrize("case", list(CASES))
def test_bj_parity_fp64(case):
    prob = CASES[case]()
    ref_state, ref = oracle.bj_solve(prob)
    assert ref.status == 0
    g = run_bj(prob, 64)
    fv = check_structures(prob, ref_state, g)
    check_factor(prob, ref_state, fv, 1e-10)
    check_solution(prob, ref_state, ref, g)


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("case", ["c1", "c2-5pct"])
def test_both_solve_kernels_fp64(case, kernel):
    """Level-synchronous, flag-synchronised and staged (cp.async) block solves give
    the same parity (FP64 factors, FP64 apply)."""
    prob = CASES[case]()
    ref_state, ref = oracle.bj_solve(prob)
    g = run_bj(prob, 64, solve_kernel=kernel)
    check_structures(prob, ref_state, g)
    check_solution(prob, ref_state, ref, g)


def test_block_beyond_staged_limit():
    """A single 70,000-row block: more rows than the staged sweeps' 16-bit
    block-local indices allow, so the solve falls back to the
    level-synchronous sweeps (in global memory) and still meets the oracle's
    bars; forcing the staged kernel is refused with an argument error."""
    prob = W.config1(m=70000, n=175000, nblocks=1)
    ref_state, ref = oracle.bj_solve(prob)
    assert ref.status == 0
    g = run_bj(prob, 64)
    check_solution(prob, ref_state, ref, g)
    with pytest.raises(sdsl.SdslError):
        run_bj(prob, 32, solve_kernel=3)


@pytest.mark.parametrize("prec", [64, 32])
def test_staged_readiness_modes_agree(prec):
    """The staged sweeps with per-value readiness and with per-level counters
    compute every row in the same order: bit-identical solutions and counts,
    and the FP64 form meets the oracle's bars (the autotuner is off: it would
    time each option set on its own and may pick another product form)."""
    prob = CASES["c2-5pct"]()
    shape = dict(solve_kernel=3, sweep_lane_entries=16, sweep_far_gap=3, tune=0)
    g1 = run_bj(prob, prec, sweep_wait=1, **shape)
    g2 = run_bj(prob, prec, sweep_wait=2, **shape)
    assert g1["stats"]["iters"] == g2["stats"]["iters"]
    assert np.array_equal(g1["x"], g2["x"])
    if prec == 64:
        ref_state, ref = oracle.bj_solve(prob)
        check_solution(prob, ref_state, ref, g2)


@pytest.mark.parametrize("prec,E", [(64, 8), (32, 4), (32, 16)])
def test_level_synchronous_sweep_agrees(prec, E):
    """The level-synchronous sweep (one named barrier per level, every entry
    of a tile summed as far) computes each row in the order of the per-value
    protocol on the same tiles (far gap 1): bit-identical solutions and
    counts; the solve meets the oracle's bars (FP64 factors, and FP32
    factors under the float-float apply)."""
    prob = CASES["c2-5pct"]()
    g1 = run_bj(prob, prec, solve_kernel=3, sweep_wait=1, sweep_far_gap=1, sweep_lane_entries=E, tune=0)
    g3 = run_bj(prob, prec, solve_kernel=3, sweep_wait=3, sweep_lane_entries=E, tune=0)
    assert g3["stats"]["sweep_shape"] == [E, 1]
    assert g1["stats"]["iters"] == g3["stats"]["iters"]
    assert np.array_equal(g1["x"], g3["x"])
    ref_state, ref = oracle.bj_solve(prob)
    check_solution(prob, ref_state, ref, g3)


def test_level_synchronous_sweep_edge_blocks():
    """Level-synchronous sweeps on single-row, empty-level-free ragged blocks
    and one block holding every row: same solution as the per-value protocol."""
    for bp in ([0, 1, 2, 50, 51, 300], [0, 300]):
        prob = W.config1(m=300, n=750)
        prob.block_ptr = np.asarray(bp, dtype=np.int64)
        g1 = run_bj(prob, 64, solve_kernel=3, sweep_wait=1, sweep_far_gap=1, sweep_lane_entries=2, tune=0)
        g3 = run_bj(prob, 64, solve_kernel=3, sweep_wait=3, sweep_lane_entries=2, tune=0)
        assert g1["stats"]["status"] == 0 and g3["stats"]["status"] == 0
        assert np.array_equal(g1["x"], g3["x"])


@pytest.mark.parametrize("form", [1, 2, 3])
def test_explicit_and_factored_products(form):
    """The PCG product with the explicit CSR of S and in the factored form
    A (theta o (A^T p)) + rho p are the same operator: both reach the oracle's
    solution and iteration count."""
    prob = CASES["c2-5pct"]()
    ref_state, ref = oracle.bj_solve(prob)
    g = run_bj(prob, 64, spmv_form=form)
    check_solution(prob, ref_state, ref, g)


@pytest.mark.parametrize("apply", [64, 48])
def test_fp32_storage_exact_apply(apply):
    """FP32-stored factors applied in FP64 or in float-float arithmetic: one
    fixed linear preconditioner (to ~1e-14), so the iteration count stays
    within 5 % of the oracle's, and the two applies agree to ~1e-12."""
    prob = CASES["c2-5pct"]()
    ref_state, ref = oracle.bj_solve(prob)
    g = run_bj(prob, 32, apply_prec=apply)
    check_solution(prob, ref_state, ref, g)


def test_float_float_apply_matches_fp64_apply():
    """z = M^{-1} r with the FP32-stored factors: the float-float apply equals
    the FP64-arithmetic apply of the same stored numbers to ~1e-13, and both
    equal the oracle's triangular solves on those FP32-rounded factors."""
    prob = CASES["c2-5pct"]()
    ref_state = oracle.bj_setup_factor(prob.A, prob.theta, prob.rho, prob.block_ptr, prob.tau, prob.delta)
    import torch

    rng = np.random.default_rng(17)
    r = rng.standard_normal(prob.A.nrows)
    r_d = torch.from_numpy(r).cuda()
    out = {}
    for apply in (64, 48, 32):
        h, keep = setup(prob, 32, apply_prec=apply)
        try:
            sdsl.sdsl_factor(h)
            z_d = torch.zeros_like(r_d)
            sdsl.sdsl_precond_apply(h, r_d, z_d)
            torch.cuda.synchronize()
            out[apply] = z_d.cpu().numpy()
        finally:
            sdsl.sdsl_free(h)
    # The operator both exact applies realise: the oracle's factor rounded to
    # FP32, each diagonal entry used through its stored FP32 reciprocal
    # float(1 / l_ii).  Model it on the oracle's values: off-diagonal entries
    # float(l_ij), diagonal entries 1 / float(1 / l_ii) (dividing by it is
    # multiplying by the stored reciprocal, to one FP64 rounding).
    P = ref_state.P
    row = np.repeat(np.arange(P.nrows), np.diff(P.rowptr))
    diag = P.col == row
    F32 = ref_state.F.astype(np.float32).astype(np.float64)
    F32[diag] = 1.0 / (1.0 / ref_state.F[diag]).astype(np.float32).astype(np.float64)
    z_ref = oracle.ic0_apply(P, F32, prob.block_ptr, r)
    # the two exact applies of the same stored numbers agree to rounding
    assert rel(out[48], out[64]) <= 1e-12
    # against the model: factor values that agree to 1e-10 before rounding
    # can round to neighbouring FP32 numbers in rare entries
    assert rel(out[64], z_ref) <= 1e-9
    assert rel(out[48], z_ref) <= 1e-9
    assert rel(out[32], out[64]) > 1e-10  # the FP32-arithmetic apply is not that operator


@pytest.mark.parametrize("case", ["c1", "c2-5pct"])
def test_bj_parity_fp32_factors(case):
    """FP32 factors under the FP64 loop (default apply: float-float): same
    structures, factor values within FP32 rounding, FP64 true residual <= 1e-8,
    x within 1e-6 of the oracle's and the iteration count within 5 %."""
    prob = CASES[case]()
    ref_state, ref = oracle.bj_solve(prob)
    g = run_bj(prob, 32)
    fv = check_structures(prob, ref_state, g)
    check_factor(prob, ref_state, fv, 1e-6)
    check_solution(prob, ref_state, ref, g)


def test_fp32_arithmetic_apply_converges():
    """The FP32-arithmetic apply (not a fixed linear operator) still reaches
    1e-8 under the flexible beta; its count is reported, bounded loosely."""
    prob = CASES["c2-5pct"]()
    ref_state, ref = oracle.bj_solve(prob)
    g = run_bj(prob, 32, apply_prec=32)
    check_solution(prob, ref_state, ref, g, iters_exact=False)
    assert g["stats"]["iters"] <= 1.5 * ref.iters + 5


def test_bounded_wait_gives_up_with_timeout_status():
    """Triangular-solve waits that run out (wait_test: every per-level wait
    waits for a tile count that is never reached; wait_limit: give up after
    64 polls) make the solve return SDSL_ERR_TIMEOUT instead of hanging; the
    context stays usable and the next handle solves normally."""
    n = 2000
    main = np.full(n, 4.0)
    off = np.full(n - 1, -1.0)
    D = np.diag(main) + np.diag(off, 1) + np.diag(off, -1)
    S = oracle.from_dense(D)
    b = np.ones(n)
    for test, expect in ((1, sdsl.ERR_TIMEOUT), (0, sdsl.OK)):
        o = sdsl.sdsl_default_options()
        o.form, o.nblocks, o.tau, o.delta = sdsl.FORM_CSR, 1, 0.0, 0.0
        o.solve_kernel, o.sweep_wait, o.graph_iters = 3, 2, 0
        o.wait_test, o.wait_limit = test, 64 if test else 0
        o.mem_space = sdsl.MEM_HOST
        h = sdsl.sdsl_setup(o, n, n, S.rowptr, S.col, S.val, None)
        try:
            sdsl.sdsl_factor(h)
            x = np.zeros(n)
            st = sdsl.sdsl_solve(h, b, x, allow=(sdsl.ERR_TIMEOUT,))
            assert st.status == expect, (test, st.status)
            if expect == sdsl.OK:
                assert relres(S, x, b) <= 1e-8
        finally:
            sdsl.sdsl_free(h)


def test_graph_and_plain_launches_agree():
    prob = W.config1(m=400, n=1000)
    a = run_bj(prob, 64, graph_iters=0)
    b = run_bj(prob, 64, graph_iters=16)
    assert a["stats"]["iters"] == b["stats"]["iters"]
    assert np.array_equal(bits(a["x"]), bits(b["x"]))


def test_deterministic_bits():
    prob = W.config2(scale=0.02)
    a = run_bj(prob, 32)
    b = run_bj(prob, 32)
    assert np.array_equal(bits(a["x"]), bits(b["x"]))


def test_device_and_host_pointers_agree():
    import torch

    prob = W.config1(m=500, n=1250)
    host = run_bj(prob, 64)
    h, keep = setup(prob, 64, device=True)
    try:
        sdsl.sdsl_factor(h)
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b)
        st = sdsl.sdsl_solve(h, b, x)
        torch.cuda.synchronize()
        assert st.status == 0
        assert np.array_equal(bits(x.cpu().numpy()), bits(host["x"]))
    finally:
        sdsl.sdsl_free(h)


def test_zero_rhs_and_exact_guess():
    prob = W.config1(m=200, n=500)
    ref_state, ref = oracle.bj_solve(prob)
    g = run_bj(prob, 64, b=np.zeros(200))
    assert g["stats"]["iters"] == 0 and not g["x"].any()
    g = run_bj(prob, 64, x0=ref.x)
    r0 = oracle.pcg_bj(ref_state.S, ref_state.P, ref_state.F, prob.block_ptr, prob.b, x0=ref.x)
    assert g["stats"]["iters"] == r0.iters == 0


def test_block_shapes_single_jacobi_empty_ragged():
    base = W.config1(m=257, n=640)
    for bp in ([0, 257], list(range(258)), [0, 10, 10, 100, 101, 257], [0, 1, 2, 3, 257]):
        prob = W.config1(m=257, n=640)
        prob.block_ptr = np.array(bp, dtype=np.int64)
        ref_state, ref = oracle.bj_solve(prob)
        g = run_bj(prob, 64)
        check_structures(prob, ref_state, g)
        check_solution(prob, ref_state, ref, g)
    del base


def test_empty_rows_of_A():
    prob = W.config1(m=120, n=300)
    A = prob.A
    # drop every entry of rows 5 and 77: S_55 = S_77 = rho
    keep = np.ones(A.nnz, bool)
    for r in (5, 77):
        keep[A.rowptr[r]:A.rowptr[r + 1]] = False
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))[keep]
    A.col, A.val = A.col[keep], A.val[keep]
    A.rowptr = np.zeros(A.nrows + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=A.nrows), out=A.rowptr[1:])
    ref_state, ref = oracle.bj_solve(prob)
    g = run_bj(prob, 64)
    check_structures(prob, ref_state, g)
    check_solution(prob, ref_state, ref, g)


def test_maxit_reached():
    prob = W.config1(m=300, n=750)
    prob.maxit = 5
    ref_state, ref = oracle.bj_solve(prob)
    assert ref.status == oracle.NOT_CONVERGED and ref.iters == 5
    g = run_bj(prob, 64)
    assert g["stats"]["status"] == sdsl.ERR_NOT_CONVERGED and g["stats"]["iters"] == 5
    assert rel(g["x"], ref.x) <= 1e-9


def test_argument_errors():
    prob = W.config1(m=50, n=120)
    o, keep = sdsl.options_for(prob)
    A = prob.A
    bad = A.col.copy()
    bad[A.rowptr[3]], bad[A.rowptr[3] + 1] = bad[A.rowptr[3] + 1], bad[A.rowptr[3]]  # unsorted row
    with pytest.raises(sdsl.SdslError) as e:
        sdsl.sdsl_setup(o, A.nrows, A.ncols, A.rowptr, bad, A.val, prob.theta)
    assert e.value.status == sdsl.ERR_ARG
    bp = np.array([0, 10, 5, 50], np.int64)
    o.block_ptr, o.nblocks = bp.ctypes.data, 3
    with pytest.raises(sdsl.SdslError) as e:
        sdsl.sdsl_setup(o, A.nrows, A.ncols, A.rowptr, A.col, A.val, prob.theta)
    assert e.value.status == sdsl.ERR_ARG
    h, keep2 = setup(prob)
    try:
        x = np.zeros(50)
        with pytest.raises(sdsl.SdslError) as e:
            sdsl.sdsl_solve(h, prob.b, x)
        assert e.value.status == sdsl.ERR_STATE
    finally:
        sdsl.sdsl_free(h)


def test_update_diag_values_and_reuse():
    prob = W.config2(scale=0.02)
    h, keep = setup(prob, 64)
    try:
        sdsl.sdsl_factor(h)
        x1 = np.zeros(len(prob.b))
        st1 = sdsl.sdsl_solve(h, prob.b, x1)
        # unchanged theta: bit-identical solve
        sdsl.sdsl_update_diag(h, prob.theta)
        x2 = np.zeros(len(prob.b))
        st2 = sdsl.sdsl_solve(h, prob.b, x2)
        assert st1.iters == st2.iters and np.array_equal(bits(x1), bits(x2))
        # new theta: S recomputed on the fixed pattern, bit-exact; factors kept
        rng = np.random.default_rng(9)
        theta2 = np.clip(prob.theta * np.exp(rng.normal(0, 0.5, len(prob.theta))), 1e-8, 1e8)
        sdsl.sdsl_update_diag(h, theta2)
        rp, ci, v = sdsl.sdsl_export_system(h)
        S2 = oracle.normal_matrix(prob.A, theta2, prob.rho)
        assert np.array_equal(ci, S2.col) and np.array_equal(bits(v), bits(S2.val))
        x3 = np.zeros(len(prob.b))
        st3 = sdsl.sdsl_solve(h, prob.b, x3)
        # oracle: same stale preconditioner (built from theta), new S
        ref = oracle.bj_setup_factor(prob.A, prob.theta, prob.rho, prob.block_ptr, prob.tau, prob.delta)
        r3 = oracle.pcg_bj(S2, ref.P, ref.F, prob.block_ptr, prob.b, rtol=prob.rtol, maxit=prob.maxit)
        assert st3.status == 0 and r3.status == 0
        assert iters_close(st3.iters, r3.iters), (st3.iters, r3.iters)
        assert relres(S2, x3, prob.b) <= 1e-8
    finally:
        sdsl.sdsl_free(h)


def test_reuse_rule_sequence():
    """Preconditioner reuse across an IPM-like theta sequence (Sec. 3.4): the
    rebuild decisions of the library equal those of the rule replayed on the
    oracle, and so do the iteration counts."""
    prob, thetas = W.config4(scale=0.002, nblocks=8, steps=8)
    h, keep = setup(prob, 64)
    gpu = []
    try:
        sdsl.sdsl_factor(h)
        for k, th in enumerate(thetas):
            if k:
                sdsl.sdsl_update_diag(h, th)
            x = np.zeros(len(prob.b))
            st = sdsl.sdsl_solve(h, prob.b, x, allow=(sdsl.ERR_NOT_CONVERGED,))
            gpu.append((st.iters, st.rebuilt, st.status, st.iters_discarded))
    finally:
        sdsl.sdsl_free(h)
    ora = [(r["iters"], r["rebuilt"], r["status"], r["discarded"]) for r in replay_reuse(prob, thetas)]
    for (gi, gr, gs, gd), (oi, orb, os_, od) in zip(gpu, ora):
        assert gs == os_ and gr == orb, (gpu, ora)
        if gs == 0:
            assert iters_close(gi, oi), (gpu, ora)


def _fresh_and_stale(prob, th0, th1):
    """Oracle PCG counts on S(th1) with a preconditioner built from th1 (fresh)
    and from th0 (stale)."""
    S1 = oracle.normal_matrix(prob.A, th1, prob.rho)
    out = []
    for th in (th1, th0):
        st = oracle.bj_setup_factor(prob.A, th, prob.rho, prob.block_ptr, prob.tau, prob.delta)
        out.append(oracle.pcg_bj(S1, st.P, st.F, prob.block_ptr, prob.b, rtol=prob.rtol, maxit=prob.maxit).iters)
    return out


def test_reuse_rule_capped_post_build_solve_still_rebuilds():
    """A first solve after a build that hits maxit is not a baseline: the next
    system is solved with a rebuilt preconditioner."""
    prob, thetas = W.config4(scale=0.002, nblocks=8, steps=2)
    fresh0 = replay_reuse(prob, thetas[:1])[0]["iters"]
    cap = max(2, fresh0 // 2)
    h, keep = setup(prob, 64, maxit=cap)
    try:
        sdsl.sdsl_factor(h)
        x = np.zeros(len(prob.b))
        st0 = sdsl.sdsl_solve(h, prob.b, x, allow=(sdsl.ERR_NOT_CONVERGED,))
        assert st0.status == sdsl.ERR_NOT_CONVERGED and st0.iters == cap and st0.rebuilt == 0
        sdsl.sdsl_update_diag(h, thetas[1])
        st1 = sdsl.sdsl_solve(h, prob.b, x, allow=(sdsl.ERR_NOT_CONVERGED,))
        assert st1.rebuilt == 1 and st1.iters_discarded == 0  # rebuilt before the solve
        assert st1.builds == 2
    finally:
        sdsl.sdsl_free(h)


def test_reuse_rule_stale_failure_rebuilds_and_resolves():
    """A solve that does not converge under a reused preconditioner is rebuilt
    and repeated in the same call; the repeated solve equals a fresh one."""
    prob, thetas = W.config4(scale=0.002, nblocks=8, steps=5)
    th1 = thetas[4]  # four drift steps on: fresh 699, stale 1,093 oracle iterations
    fresh, stale = _fresh_and_stale(prob, thetas[0], th1)
    fresh0 = replay_reuse(prob, thetas[:1])[0]["iters"]
    assert stale > fresh + 4 and fresh0 < stale, (fresh0, fresh, stale)
    cap = max(fresh0, fresh) + 2 + (stale - max(fresh0, fresh)) // 4   # fresh solves fit, the stale one not
    assert cap < stale
    h, keep = setup(prob, 64, maxit=cap)
    try:
        sdsl.sdsl_factor(h)
        x = np.zeros(len(prob.b))
        st0 = sdsl.sdsl_solve(h, prob.b, x)
        assert st0.status == 0 and st0.rebuilt == 0
        sdsl.sdsl_update_diag(h, th1)
        st1 = sdsl.sdsl_solve(h, prob.b, x)
        assert st1.status == 0 and st1.rebuilt == 1 and st1.iters_discarded == cap
        assert iters_close(st1.iters, fresh), (st1.iters, fresh)
        assert relres(oracle.normal_matrix(prob.A, th1, prob.rho), x, prob.b) <= 1e-8
    finally:
        sdsl.sdsl_free(h)


@pytest.fixture(scope="module")
def full_c2():
    """The full 200k x 500k staircase and the oracle's own solve of it (FP64,
    its block loops on every host core; the same bits as a serial run)."""
    prob = W.config2()
    ref_state, ref = oracle.bj_solve(prob)
    assert ref.status == 0
    return prob, ref_state, ref


@pytest.mark.parametrize("prec", [64, 32])
def test_full_size_config2(prec, full_c2):
    """Full 200k x 500k staircase in the benchmark's launch configuration
    (FP64 factors, and FP32 factors with the default float-float apply): S,
    the filtered pattern, corrected values, level sets and shifts compared in
    full (bit-exact); factor values on every fourth block; the solution
    checked by the oracle's FP64 true residual, against the oracle's x
    (1e-6) and the oracle's iteration count (within 5 %)."""
    prob, ref, res = full_c2
    g = run_bj(prob, prec)
    fv = check_structures(prob, ref, g)
    P = ref.P
    row = np.repeat(np.arange(P.nrows), np.diff(P.rowptr))
    low = P.col <= row
    for b in range(0, len(prob.block_ptr) - 1, 4):
        s, e = prob.block_ptr[b], prob.block_ptr[b + 1]
        m = low & (row >= s) & (row < e)
        assert rel(fv[m], ref.F[m]) <= (1e-10 if prec == 64 else 1e-6)
    check_solution(prob, ref, res, g)
