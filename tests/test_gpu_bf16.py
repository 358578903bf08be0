"""BF16 factor storage (factor_prec 16): the staged sweeps read 2-byte factor
values and apply them in float-float (default) or FP32 arithmetic under the
FP64 Krylov loop.

Bars: the apply equals the FP64 triangular solves of the same stored numbers
(the exported FP64 factor rounded FP64 -> FP32 -> BF16, each diagonal used
through its stored reciprocal) to float-float rounding; solves reach a true
relative residual <= 1e-8 and agree with the oracle's solution to 1e-6.  The
iteration count is a different preconditioner's (BF16 keeps 8 significand
bits) and is recorded, bounded loosely, not held to the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2604_23979_gb300 import sdsl
from paper_2604_23979_gb300 import workloads as W
from tests.gpu_util import rel, relres, run_bj, setup

CASES = {
    "c1": lambda: W.config1(),
    "c2-5pct": lambda: W.config2(scale=0.05),
}


@pytest.fixture(scope="module")
def built():
    from paper_2604_23979_gb300 import build

    build.build()
    sdsl.load()


def to_bf16(a):
    """FP64 -> FP32 (round to nearest) -> BF16 (round to nearest even), as FP64."""
    u = np.ascontiguousarray(a, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_model():
    """The host model of the rounding: exact on BF16 numbers, ties to even,
    relative error at most 2^-8, the unit roundoff of 8 significand bits."""
    x = np.array([1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-30])
    y = to_bf16(x)
    assert y[0] == 1.0 and y[1] == 1.0 + 2.0 ** -7
    assert y[2] == 1.0  # tie, to the even neighbour
    assert y[3] == 1.0 + 2.0 ** -6  # tie, to the even neighbour
    assert y[4] == -2.5
    r = np.random.default_rng(3).standard_normal(10000) * 10.0 ** np.random.default_rng(4).uniform(-20, 20, 10000)
    assert np.all(np.abs(to_bf16(r) - r) <= 2.0 ** -8 * np.abs(r) * (1 + 1e-6))


@pytest.mark.gpu
@pytest.mark.parametrize("apply", [48, 32])
def test_bf16_apply_matches_rounded_factor(built, apply):
    """z = M^{-1} r with BF16-stored factors equals the oracle's FP64
    triangular solves on the same rounded numbers: to ~1e-12 under the
    float-float apply, to FP32 accumulation error under the FP32 apply.
    The exported factor is the stored one (BF16 values), equal to the
    oracle's factor rounded FP64 -> FP32 -> BF16."""
    import torch

    prob = CASES["c2-5pct"]()
    ref_state = oracle.bj_setup_factor(prob.A, prob.theta, prob.rho, prob.block_ptr, prob.tau, prob.delta)
    rng = np.random.default_rng(19)
    r = rng.standard_normal(prob.A.nrows)
    r_d = torch.from_numpy(r).cuda()
    h, keep = setup(prob, 16, apply_prec=apply)
    try:
        sdsl.sdsl_factor(h)
        z_d = torch.zeros_like(r_d)
        sdsl.sdsl_precond_apply(h, r_d, z_d)
        torch.cuda.synchronize()
        z = z_d.cpu().numpy()
        prp, pci, pv, fv, alpha = sdsl.sdsl_export_precond(h)
    finally:
        sdsl.sdsl_free(h)
    P = ref_state.P
    assert np.array_equal(prp, P.rowptr) and np.array_equal(pci, P.col)
    row = np.repeat(np.arange(P.nrows), np.diff(P.rowptr))
    low = P.col < row
    diag = P.col == row
    # the stored values are BF16 numbers: the oracle's factor rounded (a
    # value within rounding of a BF16 midpoint may land on its neighbour)
    Fo = ref_state.F
    assert np.array_equal(to_bf16(fv[low | diag]), fv[low | diag])
    assert np.mean(fv[low] == to_bf16(Fo[low])) > 0.9999
    # model: the stored off-diagonal values, each diagonal entry used through
    # its stored reciprocal bf16(float(1 / l_ii))
    Fb = np.zeros_like(Fo)
    Fb[low] = fv[low]
    Fb[diag] = 1.0 / to_bf16(1.0 / Fo[diag])
    z_ref = oracle.ic0_apply(P, Fb, prob.block_ptr, r)
    assert rel(z, z_ref) <= (1e-11 if apply == 48 else 1e-4)
    # BF16 storage is a different operator from FP32 storage
    F32 = Fo.astype(np.float32).astype(np.float64)
    F32[diag] = 1.0 / (1.0 / Fo[diag]).astype(np.float32).astype(np.float64)
    assert rel(oracle.ic0_apply(P, F32, prob.block_ptr, r), z_ref) > 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("case", list(CASES))
def test_bf16_factors_solve(built, case, record_property):
    """BF16 factors under the FP64 loop: true residual <= 1e-8, x within 1e-6
    of the oracle's; iterations recorded against the oracle's."""
    prob = CASES[case]()
    ref_state, ref = oracle.bj_solve(prob)
    g = run_bj(prob, 16)
    st = g["stats"]
    assert st["status"] == 0, st
    assert relres(ref_state.S, g["x"], prob.b) <= prob.rtol
    assert rel(g["x"], ref.x) <= 1e-6
    record_property("iters_bf16", int(st["iters"]))
    record_property("iters_oracle", int(ref.iters))
    print(f"\n{case}: BF16 factors {st['iters']} iterations, oracle (FP64 factors) {ref.iters}")
    assert st["iters"] <= 3 * ref.iters + 10


@pytest.mark.gpu
def test_bf16_rejects_unsupported_forms(built):
    """BF16 storage exists for Block Jacobi with float-float or FP32 apply."""
    prob = W.config1(m=300, n=750)
    with pytest.raises(sdsl.SdslError):
        setup(prob, 16, apply_prec=64)
    with pytest.raises(sdsl.SdslError):
        setup(prob, 16, method=sdsl.BBD_GMRES)
