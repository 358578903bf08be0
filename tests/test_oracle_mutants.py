"""Plant mistakes in a copy of the oracle (on the CPU) and check that the pins
catch each one: a dropped term, a wrong sign, a wrong index or operand."""
import os
import subprocess

import pytest

import oracle
from oracle import build as obuild
import tests.test_oracle_pins as pins

SRC = open(obuild.SRC).read()

# (name, original text, planted text, pins expected to fail)
MUTANTS = [
    ("filter-or", "if (a < ti && a < tj) continue;", "if (a < ti || a < tj) continue;",
     [pins.test_filter_golden_hand_example]),
    ("filter-nonstrict", "if (a < ti && a < tj) continue;", "if (a <= ti && a <= tj) continue;",
     [pins.test_filter_golden_hand_example]),
    ("schur-operand", "acc = fma(t, v[pl], acc);", "acc = fma(t, v[ph], acc);",
     [pins.test_normal_matrix_exact_on_dyadic_values]),
    ("schur-no-rho", "if (i == j) acc = acc + rho;", "if (i == j) acc = acc + 0.0;",
     [pins.test_normal_matrix_exact_on_dyadic_values]),
    ("schur-theta-index", "double t = v[ph] * theta[ci[ph]];", "double t = v[ph] * theta[ci[pl] ^ 1];",
     [pins.test_normal_matrix_matches_dense_product]),
    ("diagcorr-sign", "double sg = v[p] < 0.0 ? -1.0 : 1.0;", "double sg = 1.0;",
     [pins.test_filter_golden_hand_example]),
    ("levels-off-by-one", "lev_lo[i] = best + 1;", "lev_lo[i] = best + 2;",
     [pins.test_levels_special_cases]),
    ("levels-lower-scope", "if (j >= s && j < i && lev_lo[j] > best) best = lev_lo[j];",
     "if (j < i && lev_lo[j] > best) best = lev_lo[j];", [pins.test_levels_special_cases]),
    ("ic0-sign", "if (kq >= 0) acc = acc - F[q] * F[kq];", "if (kq >= 0) acc = acc + F[q] * F[kq];",
     [pins.test_ic0_dense_block_equals_cholesky]),
    ("ic0-diag-term", "dsum = dsum - F[q] * F[q];", "dsum = dsum - F[q] * F[q] * 0.5;",
     [pins.test_ic0_tridiagonal_equals_cholesky]),
    ("ilu0-divide", "F[p] = F[p] / F[kd];", "F[p] = F[p] * F[kd];", [pins.test_ilu0_dense_equals_lu]),
    ("ilu0-no-shift", "F[p] = (j == i) ? shifted(pv[p], alpha) : pv[p];", "F[p] = pv[p];",
     [pins.test_ilu0_shift_retry_and_breakdown]),
    ("ilu0-zero-pivot-accepted", "if (F[dpos] == 0.0 || !isfinite(F[dpos])) return 1;",
     "if (!isfinite(F[dpos])) return 1;", [pins.test_ilu0_shift_retry_and_breakdown]),
    ("ilu0-shift-sign", "return alpha == 0.0 ? pii : pii + alpha * pii;", "return alpha == 0.0 ? pii : pii - alpha * pii;",
     [pins.test_ilu0_shift_retry_and_breakdown]),
    ("pcg-beta", "double beta = rho_new / rho;", "double beta = rho / rho_new;",
     [pins.test_pcg_matches_dense_solve]),
    ("pcg-alpha", "double alpha = rho / pq;", "double alpha = pq / rho;", [pins.test_pcg_matches_dense_solve]),
    ("gmres-givens", "H[i * m + j] = cs[i] * a + sn[i] * c;", "H[i * m + j] = cs[i] * a - sn[i] * c;",
     [pins.test_gmres_minimal_residual]),
    ("schur-bbd-sign", "SB[r * nb + c] = SB[r * nb + c] - acc;", "SB[r * nb + c] = SB[r * nb + c] + acc;",
     [pins.test_bbd_schur_and_apply_match_dense]),
    ("lu-pivot", "if (fabs(a[i * nb + k]) > best)", "if (fabs(a[i * nb + k]) < best)",
     [pins.test_dense_lu_matches_scipy]),
    ("bicgstab-beta", "beta = (rho_new / rho) * (alpha / omega);", "beta = (rho_new / rho) * (omega / alpha);",
     [lambda o: pins.test_bicgstab_terminates_after_k_passes(o, 3)]),
    ("bicgstab-omega", "omega = ts / tt;", "omega = tt / ts;",
     [pins.test_bicgstab_first_pass_is_galerkin_then_minimal_residual]),
    ("bicgstab-x-operand", "x[i] = x[i] + alpha * ph[i];", "x[i] = x[i] + alpha * p[i];",
     [pins.test_bicgstab_exact_preconditioner_one_pass, pins.test_bicgstab_recurrence_tracks_true_residual]),
    ("bicgstab-shadow", "double rv = dot(n, rt, vv);", "double rv = dot(n, r, vv);",
     [lambda o: pins.test_bicgstab_terminates_after_k_passes(o, 3)]),
    ("bicgstab-s-sign", "r[i] = r[i] - alpha * vv[i];", "r[i] = r[i] + alpha * vv[i];",
     [pins.test_bicgstab_identity_one_half_pass]),
    ("gcr-direction-sign", "pj[l] = pj[l] - c * P[i * n + l];", "pj[l] = pj[l] + c * P[i * n + l];",
     [pins.test_gcr_minimal_residual]),
    ("gcr-no-preconditioner", "precond_apply(M, r, pj);", "memcpy(pj, r, sz);",
     [pins.test_gcr_right_preconditioned_minimal_residual]),
    ("gcr-step-operand", "double a = dot(n, qj, r);", "double a = dot(n, pj, r);",
     [pins.test_gcr_minimal_residual]),
    ("gcr-normalise", "pj[l] = pj[l] / d;", "pj[l] = pj[l] * d;", [pins.test_gcr_minimal_residual]),
]


@pytest.mark.parametrize("name,orig,planted,tests", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, orig, planted, tests):
    assert SRC.count(orig) == 1, f"mutation anchor for {name} not unique"
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(orig, planted))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", str(src), "-o", str(so),
                    "-lm"], check=True)
    caught = 0
    with oracle.oracle.use_library(str(so)):
        for t in tests:
            try:
                t(oracle)
            except (AssertionError, Exception):
                caught += 1
    assert caught == len(tests), f"planted mistake {name} was not caught"
