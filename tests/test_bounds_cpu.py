"""Pins for the derived triangular-solve tolerance (tests/error_bounds.py):
the backward-error bound must hold for substitutions actually carried out in
complex FP32 and FP64 (rows summed in order, as a plain loop does), must be
tight enough to matter, and must be broken by a plausible mistake (a dropped
term, a wrong pivot, a transposed factor)."""
import numpy as np
import pytest
import scipy.sparse as sp

from error_bounds import U_FP32, U_FP64, precond_backward_check, split


def _factors(n, seed, per_row=6, band=40, offdiag=0.3):
    """Random combined factors shaped like an iLU(0) of a banded matrix."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in rng.choice(np.arange(max(0, i - band), min(n, i + band + 1)), size=per_row, replace=False):
            if j == i:
                continue
            rows.append(i)
            cols.append(j)
            vals.append((rng.standard_normal() + 1j * rng.standard_normal()) * offdiag)
        rows.append(i)
        cols.append(i)
        vals.append(1.5 + rng.random() + 1j * rng.standard_normal())
    F = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    F.sum_duplicates()
    F.sort_indices()
    return F


def _substitute(F, r, dtype, drop=None, transpose_upper=False):
    """Row-by-row forward then back substitution in `dtype` (the products
    and sums of each row in that precision); drop = (row, k) leaves out the
    k-th term of that lower-solve row."""
    L, U = split(F.astype(dtype))
    if transpose_upper:             # the strict lower part transposed in place of U's strict part
        U = (sp.triu(F.astype(dtype).T, k=1) + sp.diags(F.astype(dtype).diagonal())).tocsr()
    n = F.shape[0]
    y = np.zeros(n, dtype=dtype)
    rr = r.astype(dtype)
    for i in range(n):
        s = rr[i]
        for k, t in enumerate(range(L.indptr[i], L.indptr[i + 1])):
            j = L.indices[t]
            if j == i or (drop is not None and drop == (i, k)):
                continue
            s = s - L.data[t] * y[j]
        y[i] = s
    z = np.zeros(n, dtype=dtype)
    for i in range(n - 1, -1, -1):
        s, dg = y[i], None
        for t in range(U.indptr[i], U.indptr[i + 1]):
            j = U.indices[t]
            if j == i:
                dg = U.data[t]
            else:
                s = s - U.data[t] * z[j]
        z[i] = s * (dtype(1) / dg)
    return z


def _rhs(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("offdiag", [0.3, 3.0])          # mild and strongly non-dominant factors
@pytest.mark.parametrize("dtype,u", [(np.complex64, U_FP32), (np.complex128, U_FP64)])
def test_bound_holds_and_is_tight(dtype, u, offdiag):
    F = _factors(160, seed=1, offdiag=offdiag)
    r = _rhs(160, 2).astype(dtype)
    z = _substitute(F, r, dtype)
    Fr = F.astype(dtype).astype(np.complex128)
    resid, bound = precond_backward_check(Fr, r, z, u)
    assert np.all(resid <= bound)
    # tight: the bound is within two orders of magnitude of the largest residual
    assert np.max(resid / bound) > 1e-2 or dtype is np.complex128
    # and a few hundred roundoffs of the row scale at most
    L, U = split(Fr)
    scale = abs(L) @ (abs(U) @ np.abs(z.astype(np.complex128)))
    assert np.max(bound / scale) < 200 * u


@pytest.mark.parametrize("dtype,u", [(np.complex64, U_FP32), (np.complex128, U_FP64)])
def test_dropped_term_breaks_bound(dtype, u):
    F = _factors(160, seed=4)
    r = _rhs(160, 5).astype(dtype)
    z = _substitute(F, r, dtype, drop=(40, 0))
    resid, bound = precond_backward_check(F.astype(dtype).astype(np.complex128), r, z, u)
    assert np.any(resid > bound)


def test_wrong_pivot_breaks_bound():
    F = _factors(120, seed=7)
    G = F.tolil()
    G[30, 30] = G[30, 30] * (1 + 1e-4)          # a slightly wrong pivot in the solver's factors
    r = _rhs(120, 8).astype(np.complex64)
    z = _substitute(G.tocsr(), r, np.complex64)
    resid, bound = precond_backward_check(F.astype(np.complex64).astype(np.complex128), r, z, U_FP32)
    assert np.any(resid > bound)


def test_transposed_upper_factor_breaks_bound():
    F = _factors(120, seed=9)
    r = _rhs(120, 10)
    z = _substitute(F, r, np.complex128, transpose_upper=True)
    resid, bound = precond_backward_check(F, r, z, U_FP64)
    assert np.any(resid > bound)
