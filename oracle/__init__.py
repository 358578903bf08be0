"""FP64 CPU oracle of the SDSL-Solver hot path (arXiv 2604.23979).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the library never does.  It shares
no code with the CUDA path.  See ``oracle/sdsl_oracle.c`` for the algorithms
and the passages of the paper each one follows.

Pinning: every routine is checked in ``tests/test_oracle_pins.py`` against
values the mathematics fixes (dense numpy/scipy factorizations, brute-force
enumeration, closed forms, one-iteration convergence with exact
preconditioners).  Nothing here is "parity unpinned" except the at-scale
iteration counts of the synthetic workloads, which the paper cannot fix.
"""
from .oracle import *  # noqa: F401,F403
