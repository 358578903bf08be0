"""Write oracle/reference_counts.json: the oracle's PCG iteration count on the
full 200k x 500k staircase workload, and its run time, for the record.

The count comes from running the oracle itself (FP64, IEEE-deterministic with
-ffp-contract=off, the same bits with or without threads), never from the
CUDA path.  The tests and bench.py run their own oracle solves.
Run:  python -m oracle.reference_counts
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

OUT = os.path.join(HERE, "reference_counts.json")


def main():
    import oracle
    from paper_2604_23979_gb300 import workloads as W

    prob = W.config2()
    t0 = time.perf_counter()
    st, res = oracle.bj_solve(prob)
    t1 = time.perf_counter()
    data = {"config2": {"iters": res.iters, "status": res.status, "relres_true": res.relres_true,
                        "restarts_note": "count of products S p, true-residual checks excluded",
                        "oracle_seconds": round(t1 - t0, 1), "nnz_S": st.S.nnz, "nnz_P": st.P.nnz}}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps(data))


if __name__ == "__main__":
    main()
