"""Incomplete LU preconditioners and triangular solves (oracle; test
infrastructure only).

Section "Iterative solvers": the iLU class builds an incomplete LU of the
modified Liouvillian by discarding fill-in.
  * iLU(0): the factorisation is restricted to the pattern of A (no fill),
    computed with the row-wise IKJ elimination.
  * ILUT(d, p): dual-threshold incomplete LU. Read here as: in row i, an
    entry is dropped when its modulus is below d * ||a_i||_inf (the infinity
    norm of the original row); after elimination each of the strict-lower and
    strict-upper parts of row i keeps at most ceil(p * nnz(a_i) / 2) entries of
    largest modulus (ties: lower column first); the diagonal is always kept;
    no pivoting.
  * The condition estimate is ||M^{-1} e||_inf with e the all-ones vector
    (the section's estimate of the approximate inverse's stability).

Factors are returned as one CSR matrix: the strict lower part is L (unit
diagonal implied), the diagonal and upper part are U.
"""
from __future__ import annotations

import heapq
import math
from typing import Dict

import numpy as np
import scipy.sparse as sp


class ZeroPivot(ArithmeticError):
    pass


def _rows(A) -> list:
    A = sp.csr_matrix(A)
    A.sort_indices()
    out = []
    for i in range(A.shape[0]):
        s, e = A.indptr[i], A.indptr[i + 1]
        out.append({int(j): complex(v) for j, v in zip(A.indices[s:e], A.data[s:e])})
    return out


def _to_csr(rows: list, n: int) -> sp.csr_matrix:
    indptr = [0]
    idx, val = [], []
    for r in rows:
        for j in sorted(r):
            idx.append(j)
            val.append(r[j])
        indptr.append(len(idx))
    return sp.csr_matrix((np.array(val, dtype=np.complex128), np.array(idx, dtype=np.int64),
                          np.array(indptr, dtype=np.int64)), shape=(n, n))


def ilu0(A, pivot_floor: float = 0.0) -> sp.csr_matrix:
    """iLU(0) by IKJ elimination on the pattern of A.

    for i: for each stored k < i in increasing order:
        a_ik <- a_ik / a_kk;  for each stored j > k in row k with (i, j) stored:
        a_ij <- a_ij - a_ik a_kj.
    Raises ZeroPivot if a diagonal entry is missing or |a_kk| <= pivot_floor.
    """
    n = A.shape[0]
    rows = _rows(A)
    for k in range(n):
        if k not in rows[k] or abs(rows[k][k]) <= pivot_floor:
            raise ZeroPivot(k)
    for i in range(n):
        ri = rows[i]
        for k in sorted(c for c in ri if c < i):
            rk = rows[k]
            ri[k] = ri[k] / rk[k]
            f = ri[k]
            for j, ukj in rk.items():
                if j > k and j in ri:
                    ri[j] = ri[j] - f * ukj
        if abs(ri[i]) <= pivot_floor:
            raise ZeroPivot(i)
    return _to_csr(rows, n)


def ilut(A, drop_tol: float = 1e-4, fill_factor: float = 10.0,
         pivot_floor: float = 0.0) -> sp.csr_matrix:
    """ILUT with the dual threshold read as in the module docstring (no pivoting)."""
    n = A.shape[0]
    rows = _rows(A)
    U: list = [None] * n                         # upper rows (diag first-class)
    out = []
    for i in range(n):
        ai = rows[i]
        tau = drop_tol * (max(abs(v) for v in ai.values()) if ai else 0.0)
        lfil = int(math.ceil(fill_factor * len(ai) / 2.0))
        w: Dict[int, complex] = dict(ai)
        pending = [c for c in w if c < i]
        heapq.heapify(pending)
        while pending:
            k = heapq.heappop(pending)
            uk = U[k]
            wk = w[k] / uk[k]
            if abs(wk) < tau:
                del w[k]
                continue
            w[k] = wk
            for j, ukj in uk.items():
                if j > k:
                    if j in w:
                        w[j] = w[j] - wk * ukj
                    else:
                        w[j] = -(wk * ukj)
                        if j < i:
                            heapq.heappush(pending, j)
        if i not in w or abs(w[i]) <= pivot_floor:
            raise ZeroPivot(i)
        lower = [(j, v) for j, v in w.items() if j < i and abs(v) >= tau and v != 0]
        upper = [(j, v) for j, v in w.items() if j > i and abs(v) >= tau and v != 0]
        lower.sort(key=lambda t: (-abs(t[1]), t[0]))
        upper.sort(key=lambda t: (-abs(t[1]), t[0]))
        row = dict(lower[:lfil])
        row.update(dict(upper[:lfil]))
        row[i] = w[i]
        U[i] = {j: v for j, v in row.items() if j >= i}
        out.append(row)
    return _to_csr(out, n)


def lower_solve(F: sp.csr_matrix, b: np.ndarray) -> np.ndarray:
    """y with (I + strict_lower(F)) y = b, by forward substitution row by row."""
    F = sp.csr_matrix(F)
    n = F.shape[0]
    y = np.array(b, dtype=np.complex128, copy=True)
    for i in range(n):
        s, e = F.indptr[i], F.indptr[i + 1]
        acc = y[i]
        for t in range(s, e):
            j = F.indices[t]
            if j < i:
                acc -= F.data[t] * y[j]
        y[i] = acc
    return y


def upper_solve(F: sp.csr_matrix, y: np.ndarray) -> np.ndarray:
    """z with upper(F) z = y (diagonal included), by backward substitution."""
    F = sp.csr_matrix(F)
    n = F.shape[0]
    z = np.array(y, dtype=np.complex128, copy=True)
    for i in range(n - 1, -1, -1):
        s, e = F.indptr[i], F.indptr[i + 1]
        acc = z[i]
        diag = None
        for t in range(s, e):
            j = F.indices[t]
            if j > i:
                acc -= F.data[t] * z[j]
            elif j == i:
                diag = F.data[t]
        z[i] = acc / diag
    return z


def split_factors(F: sp.csr_matrix):
    """(L, U) as separate sparse matrices: unit lower and upper with diagonal."""
    F = sp.csr_matrix(F)
    n = F.shape[0]
    L = sp.tril(F, k=-1, format="csr") + sp.identity(n, dtype=np.complex128, format="csr")
    U = sp.triu(F, k=0, format="csr")
    return sp.csr_matrix(L), sp.csr_matrix(U)


def precond_apply_fast(F: sp.csr_matrix, r: np.ndarray) -> np.ndarray:
    """M^{-1} r = U^{-1} L^{-1} r using SciPy's sparse triangular solve as the
    primitive (same arithmetic as lower_solve/upper_solve, different order of
    summation within a row)."""
    from scipy.sparse.linalg import spsolve_triangular
    L, U = split_factors(F)
    y = spsolve_triangular(L, r, lower=True, unit_diagonal=True)
    return spsolve_triangular(U, y, lower=False)


def condition_estimate(F: sp.csr_matrix) -> float:
    """||M^{-1} e||_inf with e = (1, 1, ..., 1)."""
    e = np.ones(F.shape[0], dtype=np.complex128)
    return float(np.max(np.abs(upper_solve(F, lower_solve(F, e)))))
