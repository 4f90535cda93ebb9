"""FP64 CPU oracle for ROR-BK (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  It shares no code with the CUDA solver; the C source
``rorbk_oracle.c`` is compiled with gcc into ``_build/liboracle.so``.

Python wrappers here only marshal numpy arrays into the C functions; every
step of the method runs in the C file, which cites the paper passage each
function follows (Algorithm 1, Section 2, Section 3.1).
"""
from .oracle import (  # noqa: F401
    build, lib, OracleMatrix, philox4x64_10, partition, orthogonality,
    proposal, sample, residual, topk, block_gram, cholesky, chol_solve,
    spd_inverse, static_operator, update_with_inverse, update_with_cholesky,
    solve, SolveResult, initial_solution, fabgmres, block_norms, weighted_cdf, PAPER, RESIDUAL_WEIGHTED,
    column_gram, column_operator, update_woodbury, update_woodbury_cholesky, thread_count,
)
