"""Helpers shared by the GPU parity tests (call the library through its C ABI)."""
import numpy as np

from paper_2604_23979_gb300 import sdsl


def setup(prob, prec=64, graph_iters=16, device=False, **over):
    o, keep = sdsl.options_for(prob, factor_prec=prec, graph_iters=graph_iters)
    for k, v in over.items():
        setattr(o, k, v)
    A = prob.A
    arrs = [A.rowptr, A.col, A.val, prob.theta]
    if device:
        import torch

        arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    h = sdsl.sdsl_setup(o, A.nrows, A.ncols, *arrs)
    return h, (o, keep, arrs)


def run_bj(prob, prec=64, graph_iters=16, b=None, x0=None, **over):
    h, keep = setup(prob, prec, graph_iters, **over)
    try:
        sdsl.sdsl_factor(h)
        b = prob.b if b is None else b
        x = np.zeros(len(b)) if x0 is None else x0.copy()
        st = sdsl.sdsl_solve(h, np.ascontiguousarray(b), x, x0_zero=x0 is None)
        out = dict(x=x, stats=st.as_dict(), S=sdsl.sdsl_export_system(h), P=sdsl.sdsl_export_precond(h),
                   lev_lo=sdsl.sdsl_export_levels(h, 0), lev_up=sdsl.sdsl_export_levels(h, 1))
    finally:
        sdsl.sdsl_free(h)
    return out


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def relres(S, x, b):
    """||b - S x|| / ||b|| with the oracle's FP64 SpMV."""
    import oracle

    return float(np.linalg.norm(b - oracle.spmv(S, x)) / np.linalg.norm(b))


def iters_close(gpu, ref):
    """Iteration counts within max(1, 5 %) of the oracle's."""
    return abs(gpu - ref) <= max(1, int(np.ceil(0.05 * ref)))


def replay_reuse(prob, thetas, ratio=1.5, maxit=None, keep_x=None):
    """The preconditioner-reuse rule (Sec. 3.4) replayed on the oracle over a
    theta sequence: factor at step 0; the first converged solve after a build
    is the baseline; a converged solve needing more than ratio x the baseline,
    or a solve that does not converge, requests a rebuild before the next
    step; a solve that does not converge under a reused preconditioner is
    rebuilt and repeated at once (from x0 = 0).  Returns one dict per step."""
    import oracle

    maxit = prob.maxit if maxit is None else maxit
    out = []
    state, base, need, since = None, -1, True, 0
    for k, th in enumerate(thetas):
        S = oracle.normal_matrix(prob.A, th, prob.rho)
        rebuilt = 0
        if need:
            state = oracle.bj_setup_factor(prob.A, th, prob.rho, prob.block_ptr, prob.tau, prob.delta)
            base, need, since, rebuilt = -1, False, 0, int(k > 0)
        r = oracle.pcg_bj(S, state.P, state.F, prob.block_ptr, prob.b, rtol=prob.rtol, maxit=maxit)
        discarded = 0
        if r.status != 0 and since > 0:
            discarded = r.iters
            state = oracle.bj_setup_factor(prob.A, th, prob.rho, prob.block_ptr, prob.tau, prob.delta)
            base, since, rebuilt = -1, 0, 1
            r = oracle.pcg_bj(S, state.P, state.F, prob.block_ptr, prob.b, rtol=prob.rtol, maxit=maxit)
        since += 1
        margin = None  # how close this solve came to the ratio threshold (relative)
        if r.status == 0:
            if base < 0:
                base = r.iters
            else:
                margin = abs(r.iters / (ratio * base) - 1.0)
                if r.iters > ratio * base:
                    need = True
        else:
            need = True
        out.append(dict(k=k, iters=r.iters, status=r.status, rebuilt=rebuilt, discarded=discarded, margin=margin,
                        relres=float(np.linalg.norm(prob.b - oracle.spmv(S, r.x)) / np.linalg.norm(prob.b)),
                        x=r.x if keep_x is None or k in keep_x else None))
    return out
