"""Dense FP64 steady state (oracle; test infrastructure only).

The steady state is the null vector of L (Eq. eigval) normalised to unit
trace. Because the trace is conserved (sum of the diagonal-element rows of L
vanishes), one such row is redundant; replacing row 0 by the trace condition
sum_i rho_ii = 1 gives a nonsingular system whenever the steady state is
unique. This is the linear-system form of the section "Direct factorization",
solved here by LAPACK's dense LU with partial pivoting.
"""
from __future__ import annotations

import numpy as np

from .liouvillian import liouvillian_dense, trace_columns


def trace_row_system(L: np.ndarray, d: int):
    """Return (A, b): L with row 0 replaced by the trace condition, b = e_0."""
    A = np.array(L, dtype=np.complex128, copy=True)
    A[0, :] = 0.0
    A[0, trace_columns(d)] = 1.0
    b = np.zeros(A.shape[0], dtype=np.complex128)
    b[0] = 1.0
    return A, b


def unvec(x: np.ndarray, d: int) -> np.ndarray:
    """Column-stacked vector -> d x d matrix (inverse of vec, Eq. eigval)."""
    return np.asarray(x).reshape((d, d), order="F")


def steady_state_dense(H, c_ops) -> np.ndarray:
    """rho_ss by dense LU of the trace-row system; returns rho (d x d), Tr rho = 1."""
    d = H.shape[0]
    L = liouvillian_dense(H, c_ops)
    A, b = trace_row_system(L, d)
    x = np.linalg.solve(A, b)
    rho = unvec(x, d).copy()
    return rho / np.trace(rho)


def steady_state_svd(H, c_ops) -> np.ndarray:
    """Independent check: right singular vector of L for its smallest singular
    value, unstacked and trace-normalised."""
    d = H.shape[0]
    L = liouvillian_dense(H, c_ops)
    _, _, vh = np.linalg.svd(L)
    x = vh[-1].conj()
    rho = unvec(x, d).copy()
    return rho / np.trace(rho)
