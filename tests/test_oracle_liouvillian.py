"""Pins for the oracle's Liouvillian (Eq. lindblad, Eq. eigval, Eq. linear,
Eq. inverse) against mathematics that does not go through numpy.kron."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.liouvillian import (default_weight, liouvillian_apply, liouvillian_dense,
                                liouvillian_row, liouvillian_sparse, modified_liouvillian,
                                shifted_liouvillian, trace_columns)
from oracle.steady import steady_state_dense
from workloads import driven_cavity, jaynes_cummings_rwa, random_system, sigma_minus

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_matrix(d, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))


def _lindblad_action(H, c_ops, X):
    """-i[H, X] + sum C X C^+ - (X C^+C + C^+C X)/2 by plain matrix products."""
    H = H.toarray()
    Y = -1j * (H @ X - X @ H)
    for C in c_ops:
        C = C.toarray()
        Cd = C.conj().T
        Y = Y + C @ X @ Cd - 0.5 * (X @ Cd @ C + Cd @ C @ X)
    return Y


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_vectorised_matrix_equals_superoperator_action(seed):
    s = random_system(5, n_c=2, seed=seed)
    L = liouvillian_dense(s.H, s.c_ops)
    X = _rand_matrix(5, seed + 10)
    lhs = L @ X.reshape(-1, order="F")
    rhs = _lindblad_action(s.H, s.c_ops, X).reshape(-1, order="F")
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_row_stacking_would_fail():
    """A transposed stacking convention must not pass the action test."""
    s = random_system(4, n_c=1, seed=3)
    L = liouvillian_dense(s.H, s.c_ops)
    X = _rand_matrix(4, 5)
    lhs = L @ X.reshape(-1, order="C")
    rhs = _lindblad_action(s.H, s.c_ops, X).reshape(-1, order="C")
    assert np.max(np.abs(lhs - rhs)) > 1e-3


@pytest.mark.parametrize("seed", [0, 4])
def test_all_forms_agree(seed):
    s = random_system(6, n_c=3, seed=seed)
    Ld = liouvillian_dense(s.H, s.c_ops)
    Ls = liouvillian_sparse(s.H, s.c_ops)
    np.testing.assert_allclose(Ls.toarray(), Ld, atol=1e-13, rtol=0)
    x = np.random.default_rng(seed).standard_normal(36) + 0j
    np.testing.assert_allclose(liouvillian_apply(s.H, s.c_ops, x), Ld @ x, atol=1e-12, rtol=0)
    for p in (0, 7, 35):
        np.testing.assert_allclose(liouvillian_row(s.H, s.c_ops, p), Ld[p], atol=1e-13, rtol=0)


@pytest.mark.parametrize("seed", [0, 1])
def test_trace_preservation(seed):
    """Tr L[X] = 0 for every X: the diagonal-element rows of L sum to zero."""
    s = random_system(5, n_c=2, seed=seed)
    L = liouvillian_dense(s.H, s.c_ops)
    np.testing.assert_allclose(L[trace_columns(5), :].sum(axis=0), 0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_hermiticity_preservation(seed):
    """L[X^+] = L[X]^+ for every X."""
    s = random_system(5, n_c=2, seed=seed)
    L = liouvillian_dense(s.H, s.c_ops)
    X = _rand_matrix(5, 99)
    Y1 = (L @ X.conj().T.reshape(-1, order="F")).reshape((5, 5), order="F")
    Y2 = (L @ X.reshape(-1, order="F")).reshape((5, 5), order="F").conj().T
    np.testing.assert_allclose(Y1, Y2, atol=1e-12)


def test_two_level_decay_textbook_rates():
    g = json.load(open(os.path.join(GOLD, "hand_examples.json")))["two_level_decay"]
    gamma = g["gamma"]
    L = liouvillian_dense(sp.csr_matrix((2, 2), dtype=complex), [np.sqrt(gamma) * sigma_minus()])
    d = 2
    idx = lambda i, j: i + d * j                      # noqa: E731  (rho_ij position)
    gnd, exc = 0, 1
    assert L[idx(exc, exc), idx(exc, exc)] == pytest.approx(-gamma)
    assert L[idx(gnd, gnd), idx(exc, exc)] == pytest.approx(gamma)
    assert L[idx(exc, gnd), idx(exc, gnd)] == pytest.approx(-gamma / 2)
    assert L[idx(gnd, exc), idx(gnd, exc)] == pytest.approx(-gamma / 2)
    assert abs(L[idx(gnd, gnd), idx(gnd, gnd)]) == 0


def test_modified_liouvillian_row_and_rhs():
    s = driven_cavity(N=6)
    L = liouvillian_sparse(s.H, s.c_ops)
    w = default_weight(L)
    Lt, b = modified_liouvillian(L, 6, w)
    diff = (Lt - L).toarray()
    expect = np.zeros_like(diff)
    expect[0, trace_columns(6)] = w
    np.testing.assert_allclose(diff, expect, atol=1e-14)
    assert b[0] == w and np.all(b[1:] == 0)
    rho = steady_state_dense(s.H, s.c_ops)
    np.testing.assert_allclose(Lt @ rho.reshape(-1, order="F"), b, atol=1e-12)


def test_shifted_liouvillian_full_diagonal():
    s = jaynes_cummings_rwa(N=4)
    L = liouvillian_sparse(s.H, s.c_ops)
    assert np.count_nonzero(L.diagonal()) < L.shape[0]   # RWA JC: vacuum population row
    S = shifted_liouvillian(L, 1e-15)
    D = S.tocoo()
    assert np.count_nonzero(D.row == D.col) == L.shape[0]
    dl, ds = L.diagonal(), S.diagonal()
    zero = dl == 0
    assert np.all(ds[zero] == -1e-15)
    assert np.all(np.abs(ds[~zero] - dl[~zero] + 1e-15) <= 4e-16 * np.abs(dl[~zero]))


def test_sparse_pattern_drops_exact_zeros():
    s = driven_cavity(N=5)
    L = liouvillian_sparse(s.H, s.c_ops)
    Ld = liouvillian_dense(s.H, s.c_ops)
    assert L.nnz == np.count_nonzero(Ld)
