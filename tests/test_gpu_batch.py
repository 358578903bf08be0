"""Batched solves (several requests in the same launches) through the C ABI:
each request's iterates are those of its solve alone, bit for bit; the
launches of the batch carry every request's blocks (far fewer launches than
the requests' solves one after another); the results meet the oracle."""
import numpy as np
import pytest

import oracle
from paper_2604_23979_gb300 import sdsl
from paper_2604_23979_gb300 import workloads as W
from tests.gpu_util import iters_close, rel, relres, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_23979_gb300 import build

    build.build()
    sdsl.load()


BATCH_OPTS = dict(sweep_slots=2, spmv_form=3, graph_iters=16)


def problems():
    rng = np.random.default_rng(31)
    ps = [W.config2(scale=0.02), W.config2(scale=0.05), W.config1(m=1200, n=3000, nblocks=3)]
    ps += [W.serving_request(rng, 0.0, 1000, 20000).problem for _ in range(3)]
    return ps


def solve_alone(ps, prec):
    out = []
    for p in ps:
        h, keep = setup(p, prec, **BATCH_OPTS)
        try:
            sdsl.sdsl_factor(h)
            x = np.zeros(len(p.b))
            n0 = sdsl.sdsl_kernel_launches()
            st = sdsl.sdsl_solve(h, p.b, x)
            out.append((x, int(st.iters), int(st.status), sdsl.sdsl_kernel_launches() - n0))
        finally:
            sdsl.sdsl_free(h)
    return out


@pytest.mark.parametrize("prec", [32, 64, 16])
def test_batch_equals_alone_bit_for_bit(prec):
    ps = problems()
    alone = solve_alone(ps, prec)
    hs, keeps = [], []
    try:
        for p in ps:
            h, keep = setup(p, prec, **BATCH_OPTS)
            sdsl.sdsl_factor(h)
            hs.append(h)
            keeps.append(keep)
        xs = [np.zeros(len(p.b)) for p in ps]
        n0 = sdsl.sdsl_kernel_launches()
        sts = sdsl.sdsl_batch_solve(hs, [p.b for p in ps], xs)
        batch_launches = sdsl.sdsl_kernel_launches() - n0
    finally:
        for h in hs:
            sdsl.sdsl_free(h)
    for i, (p, (xa, ia, sa, _)) in enumerate(zip(ps, alone)):
        assert sts[i].status == sa and sts[i].iters == ia, (i, sts[i].iters, ia)
        assert np.array_equal(xs[i].view(np.int64), xa.view(np.int64)), f"request {i} differs in the batch"
    # one launch carries the blocks of every request: the batch needs about
    # as many iteration launches as its longest solve, not their sum
    alone_launches = sum(a[3] for a in alone)
    assert batch_launches < 0.5 * alone_launches, (batch_launches, alone_launches)


def test_batch_meets_oracle():
    ps = problems()[:4]
    hs, keeps = [], []
    try:
        for p in ps:
            h, keep = setup(p, 32, **BATCH_OPTS)
            sdsl.sdsl_factor(h)
            hs.append(h)
            keeps.append(keep)
        xs = [np.zeros(len(p.b)) for p in ps]
        sts = sdsl.sdsl_batch_solve(hs, [p.b for p in ps], xs)
    finally:
        for h in hs:
            sdsl.sdsl_free(h)
    for p, x, st in zip(ps, xs, sts):
        ref_state, ref = oracle.bj_solve(p)
        assert st.status == 0 and ref.status == 0
        assert relres(ref_state.S, x, p.b) <= p.rtol
        assert rel(x, ref.x) <= 1e-6
        assert iters_close(st.iters, ref.iters), (st.iters, ref.iters)


def test_batch_with_unbatchable_handles_solves_each():
    """Handles of different kernel shapes (FP64 and FP32 factors) are solved
    one after another by the same call, with the same results."""
    ps = problems()[:2]
    alone = [solve_alone([ps[0]], 64)[0], solve_alone([ps[1]], 32)[0]]
    hs, keeps = [], []
    try:
        for p, prec in zip(ps, (64, 32)):
            h, keep = setup(p, prec, **BATCH_OPTS)
            sdsl.sdsl_factor(h)
            hs.append(h)
            keeps.append(keep)
        xs = [np.zeros(len(p.b)) for p in ps]
        sts = sdsl.sdsl_batch_solve(hs, [p.b for p in ps], xs)
    finally:
        for h in hs:
            sdsl.sdsl_free(h)
    for i in range(2):
        assert sts[i].iters == alone[i][1]
        assert np.array_equal(xs[i], alone[i][0])


def test_continuous_batch_join_and_leave():
    """Requests join a running batch between graph launches and leave as soon
    as their own solve ends; every result equals the solve alone, bit for
    bit, and a request that finishes early is handed back before the others."""
    ps = problems()
    alone = solve_alone(ps, 32)
    hs, keeps = [], []
    B = sdsl.sdsl_batch_create(16)
    try:
        for p in ps:
            h, keep = setup(p, 32, **BATCH_OPTS)
            sdsl.sdsl_factor(h)
            hs.append(h)
            keeps.append(keep)
        xs = [np.zeros(len(p.b)) for p in ps]
        order, steps = [], 0
        for i in range(3):  # three start together
            sdsl.sdsl_batch_add(B, hs[i], ps[i].b, xs[i])
        pending = list(range(3, len(ps)))
        while sdsl.sdsl_batch_size(B) > 0 or pending:
            if pending and steps % 2 == 1:  # the others join while the batch runs
                i = pending.pop(0)
                sdsl.sdsl_batch_add(B, hs[i], ps[i].b, xs[i])
            out = sdsl.sdsl_batch_step(B, max_graphs=1, cap=8)
            steps += 1
            for hv, st in out:
                i = [h.value for h in hs].index(hv)
                order.append(i)
                assert st.status == alone[i][2] and st.iters == alone[i][1], (i, st.iters, alone[i][1])
            assert steps < 10000
    finally:
        sdsl.sdsl_batch_free(B)
        for h in hs:
            sdsl.sdsl_free(h)
    assert sorted(order) == list(range(len(ps)))
    for i in range(len(ps)):
        assert np.array_equal(xs[i].view(np.int64), alone[i][0].view(np.int64)), f"request {i} differs"
    # the request with the fewest iterations among the first three leaves first
    first3 = sorted(range(3), key=lambda i: alone[i][1])
    assert order.index(first3[0]) < order.index(first3[2])
