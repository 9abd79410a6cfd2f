"""Pins for the derived triangular-solve tolerance (tests/error_bounds.py):
the bound must hold for substitutions actually carried out in complex FP32
and FP64, must not be vacuous, and must be broken by a plausible mistake
(a dropped term, a wrong diagonal)."""
import numpy as np
import pytest
import scipy.sparse as sp

from error_bounds import U_FP32, U_FP64, precond_error_bound, split


def _factors(n, seed, per_row=6, band=40):
    """Random combined factors shaped like an iLU(0) of a banded matrix."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in rng.choice(np.arange(max(0, i - band), min(n, i + band + 1)), size=per_row, replace=False):
            if j == i:
                continue
            rows.append(i)
            cols.append(j)
            vals.append((rng.standard_normal() + 1j * rng.standard_normal()) * 0.3)
        rows.append(i)
        cols.append(i)
        vals.append(1.5 + rng.random() + 1j * rng.standard_normal())
    F = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    F.sum_duplicates()
    F.sort_indices()
    return F


def _substitute(F, r, dtype, drop=None, acc_dtype=None):
    """Row-by-row forward then back substitution in `dtype` (the products
    and sums of each row in that precision); drop = (row, k) leaves out the
    k-th term of that lower-solve row."""
    acc_dtype = acc_dtype or dtype
    L, U = split(F.astype(dtype))
    n = F.shape[0]
    y = np.zeros(n, dtype=acc_dtype)
    rr = r.astype(dtype).astype(acc_dtype)
    for i in range(n):
        s = rr[i]
        cols = L.indices[L.indptr[i]:L.indptr[i + 1]]
        vals = L.data[L.indptr[i]:L.indptr[i + 1]].astype(acc_dtype)
        for k, (j, v) in enumerate(zip(cols, vals)):
            if j == i or (drop is not None and drop == (i, k)):
                continue
            s = s - v * y[j]
        y[i] = s
    z = np.zeros(n, dtype=acc_dtype)
    for i in range(n - 1, -1, -1):
        cols = U.indices[U.indptr[i]:U.indptr[i + 1]]
        vals = U.data[U.indptr[i]:U.indptr[i + 1]].astype(acc_dtype)
        s, dg = y[i], None
        for j, v in zip(cols, vals):
            if j == i:
                dg = v
            else:
                s = s - v * z[j]
        z[i] = s * (acc_dtype(1) / dg)
    return y, z


def _exact(F, r, dtype):
    """The same solve in extended precision (long double) on the factors and
    right-hand side rounded to `dtype`: the reference the bound speaks of."""
    Fd = F.astype(dtype).astype(np.clongdouble)
    return _substitute(Fd.tocsr(), r.astype(dtype).astype(np.clongdouble), np.clongdouble)


@pytest.mark.parametrize("dtype,u", [(np.complex64, U_FP32), (np.complex128, U_FP64)])
def test_bound_holds_and_is_not_vacuous(dtype, u):
    F = _factors(160, seed=1)
    r = np.random.default_rng(2).standard_normal(160) + 1j * np.random.default_rng(3).standard_normal(160)
    _, zh = _substitute(F, r, dtype)
    ye, ze = _exact(F, r, dtype)
    Fr = F.astype(dtype).astype(np.complex128)
    bound = precond_error_bound(Fr, ye.astype(np.complex128), ze.astype(np.complex128), u)
    err = np.abs(zh.astype(np.clongdouble) - ze).astype(np.float64)
    assert np.all(err <= bound)
    # informative: the bound is within a few orders of magnitude of the error
    scale = np.abs(ze).astype(np.float64)
    assert np.median(bound / scale) < 1e4 * u
    assert np.max(err) > 0


def test_dropped_term_breaks_bound():
    F = _factors(160, seed=4)
    r = np.random.default_rng(5).standard_normal(160) + 1j * np.random.default_rng(6).standard_normal(160)
    _, zh = _substitute(F, r, np.complex64, drop=(40, 0))
    ye, ze = _exact(F, r, np.complex64)
    Fr = F.astype(np.complex64).astype(np.complex128)
    bound = precond_error_bound(Fr, ye.astype(np.complex128), ze.astype(np.complex128), U_FP32)
    err = np.abs(zh.astype(np.clongdouble) - ze).astype(np.float64)
    assert np.any(err > bound)


def test_wrong_diagonal_breaks_bound():
    F = _factors(120, seed=7)
    G = F.tolil()
    G[30, 30] = G[30, 30] * (1 + 1e-4)          # a slightly wrong pivot in the solver's factors
    r = np.random.default_rng(8).standard_normal(120) + 0j
    _, zh = _substitute(G.tocsr(), r, np.complex64)
    ye, ze = _exact(F, r, np.complex64)
    Fr = F.astype(np.complex64).astype(np.complex128)
    bound = precond_error_bound(Fr, ye.astype(np.complex128), ze.astype(np.complex128), U_FP32)
    err = np.abs(zh.astype(np.clongdouble) - ze).astype(np.float64)
    assert np.any(err > bound)
