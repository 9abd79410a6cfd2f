"""CPU oracle for the steady-state solver (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, deliberately unoptimised restatement of what
the solver computes, written from the paper (Nation, "Steady-state solution
methods for open quantum optical systems", arXiv:1504.06768) in float64
NumPy/SciPy. It exists to check the CUDA library: only the test-suite, the
smoke check and the CPU-baseline leg of the benchmark may import it. The
product library never imports, links or calls anything here, and nothing
here imports the product library.

Modules
-------
liouvillian  Eq. (lindblad)/(eigval): dense and sparse L, matrix-free apply,
             element-wise rows; the trace-row and shifted forms (Eq. linear,
             Eq. inverse).
steady       Dense FP64 LU of L with one row replaced by the trace condition;
             null vector by SVD as an independent cross-check.
ordering     Cuthill-McKee / reverse Cuthill-McKee (Sec. "Direct
             factorization"), bandwidth and profile.
ilu          iLU(0) and ILUT (Sec. "Iterative solvers"), triangular solves,
             condition estimate.
krylov       Right-preconditioned BiCGSTAB and restarted GMRES(m); the
             doubly-iterative inverse-power method; the plain CPU sparse
             iterative steady-state pipeline.
metrics      Trace distance, Hermiticity, positivity, residual norm.
rng          The counter-based generator (SplitMix64) for the inverse-power
             start vector.

Parity status: every function is pinned by tests under tests/ to closed
forms, printed values of the paper, invariants or brute force.
"""
