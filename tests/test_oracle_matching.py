"""The oracle's weighted bipartite matching (section "Direct factorization")
against what fixes it: hand-traced cases, SciPy's maximum matching
cardinality, and the zero-free diagonal it exists to produce."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import maximum_bipartite_matching

from oracle.liouvillian import default_weight, liouvillian_sparse, modified_liouvillian
from oracle.matching import weighted_mbm
from workloads import driven_cavity, jaynes_cummings_rwa, paper_spin_chain


def test_hand_traced_without_augmentation():
    """Column maxima 25 (col 1, row 0), 16 (col 0, row 1), 9 (col 2, row 2):
    every column gets its heaviest row."""
    A = sp.csr_matrix(np.array([[1, 5, 0], [4, 0, 0], [0, 2, 3]], dtype=complex))
    match, k = weighted_mbm(A)
    assert match.tolist() == [1, 0, 2] and k == 3


def test_hand_traced_augmenting_path():
    """Column 0 first takes row 0 (weight 25); column 1 has only row 0, so the
    search goes through column 0 to its next row (row 1) and flips the path."""
    A = sp.csr_matrix(np.array([[5, 1], [4, 0]], dtype=complex))
    match, k = weighted_mbm(A)
    assert match.tolist() == [1, 0] and k == 2


def test_weights_choose_the_larger_diagonal():
    A = sp.csr_matrix(np.array([[1, 3j], [2, 1]], dtype=complex))
    match, _ = weighted_mbm(A)
    assert match.tolist() == [1, 0]                     # diagonal 2, 3j instead of 1, 1


def test_dominant_diagonal_is_kept():
    rng = np.random.default_rng(0)
    A = sp.random(40, 40, density=0.15, random_state=rng) * (1 + 1j) + sp.diags(10 + rng.random(40))
    match, k = weighted_mbm(A)
    assert k == 40 and match.tolist() == list(range(40))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("density", [0.03, 0.08])
def test_cardinality_is_maximum(seed, density):
    """Structurally singular cases included: the matched count equals the
    maximum matching size SciPy finds."""
    rng = np.random.default_rng(seed)
    A = sp.random(60, 60, density=density, random_state=rng, format="csr")
    A.data = A.data + 1j * rng.random(A.nnz)
    match, k = weighted_mbm(A)
    ref = maximum_bipartite_matching(sp.csr_matrix((np.ones(A.nnz), A.indices, A.indptr), shape=A.shape),
                                     perm_type="row")
    assert k == int(np.sum(ref >= 0))
    used = match[match >= 0]
    assert len(set(used.tolist())) == len(used)          # a matching: rows used once
    for j in np.flatnonzero(match >= 0):
        assert A[match[j], j] != 0


@pytest.mark.parametrize("seed", range(4))
def test_zero_free_diagonal_of_a_scrambled_matrix(seed):
    """Rows of a matrix with a full diagonal shuffled: a perfect matching
    exists and A[match, :] has no zero on its diagonal."""
    rng = np.random.default_rng(seed)
    n = 50
    A = sp.random(n, n, density=0.05, random_state=rng) + sp.diags(1 + rng.random(n))
    A = sp.csr_matrix(A)[rng.permutation(n), :]
    match, k = weighted_mbm(A)
    assert k == n
    assert np.all(sp.csr_matrix(A)[match, :].diagonal() != 0)


@pytest.mark.parametrize("maker", [lambda: driven_cavity(n_th=0.2), lambda: jaynes_cummings_rwa(seed=1, N=6),
                                   lambda: paper_spin_chain()], ids=["cavity", "jc6", "spin5"])
def test_trace_row_liouvillian_gets_a_zero_free_diagonal(maker):
    s = maker()
    L = liouvillian_sparse(s.H, s.c_ops)
    A = sp.csr_matrix(modified_liouvillian(L, s.d, default_weight(L))[0])
    match, k = weighted_mbm(A)
    assert k == A.shape[0]
    assert np.all(A[match, :].diagonal() != 0)
