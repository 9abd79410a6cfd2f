"""Pins for the oracle's reverse Cuthill-McKee ordering, bandwidth and profile
(section "Direct factorization")."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.liouvillian import (default_weight, liouvillian_sparse, modified_liouvillian,
                                shifted_liouvillian)
from oracle.ordering import bandwidth_profile, permute_symmetric, rcm_order
from workloads import paper_jc_nonrwa, paper_optomechanics, paper_spin_chain

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pattern(n, entries, sym=False, diag=False):
    r = [e[0] for e in entries]
    c = [e[1] for e in entries]
    if sym:
        r, c = r + c, c + r
    if diag:
        r, c = r + list(range(n)), c + list(range(n))
    A = sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))
    A.data[:] = 1.0
    return A


def test_bandwidth_profile_hand_example():
    g = json.load(open(os.path.join(GOLD, "hand_examples.json")))["bandwidth_profile"]
    A = _pattern(g["n"], g["entries"])
    B, P, ub, lb, up, lp = bandwidth_profile(A)
    assert (B, P, ub, lb, up, lp) == (g["B"], g["P"], g["ub"], g["lb"], g["up"], g["lp"])


def test_rcm_hand_example():
    g = json.load(open(os.path.join(GOLD, "hand_examples.json")))["rcm"]
    A = _pattern(g["n"], g["edges"], sym=True, diag=True)
    assert rcm_order(A).tolist() == g["rcm"]
    assert rcm_order(A)[::-1].tolist() == g["cm"]


@pytest.mark.parametrize("n", [7, 50, 333])
def test_rcm_recovers_scrambled_path(n):
    """A path graph under a random relabelling: RCM must return bandwidth 3."""
    perm = np.random.default_rng(n).permutation(n)
    edges = [(int(perm[i]), int(perm[i + 1])) for i in range(n - 1)]
    A = _pattern(n, edges, sym=True, diag=True)
    assert bandwidth_profile(A)[0] > 3
    p = rcm_order(A)
    assert sorted(p.tolist()) == list(range(n))
    assert bandwidth_profile(permute_symmetric(A, p))[0] == 3


def test_rcm_scrambled_grid_bandwidth():
    """k x k grid graph, scrambled: the BFS ordering has half-bandwidth <= k."""
    k = 9
    idx = np.arange(k * k).reshape(k, k)
    edges = [(idx[i, j], idx[i, j + 1]) for i in range(k) for j in range(k - 1)]
    edges += [(idx[i, j], idx[i + 1, j]) for i in range(k - 1) for j in range(k)]
    perm = np.random.default_rng(0).permutation(k * k)
    edges = [(int(perm[a]), int(perm[b])) for a, b in edges]
    A = _pattern(k * k, edges, sym=True, diag=True)
    _, _, ub, lb, _, _ = bandwidth_profile(permute_symmetric(A, rcm_order(A)))
    assert ub <= k and lb <= k


def test_rcm_level_structure():
    """Cuthill-McKee order is a BFS order: along the CM sequence the BFS level
    (distance from the start within the component) never decreases."""
    s = paper_optomechanics(Nc=3, Nm=4)
    L = liouvillian_sparse(s.H, s.c_ops)
    cm = rcm_order(L)[::-1]
    S = (abs(L) + abs(L.T)).tocsr()
    dist = sp.csgraph.shortest_path(S, unweighted=True, indices=[int(cm[0])])[0]
    seq = dist[cm]
    assert np.all(np.diff(seq) >= 0)


def _paper_matrix(system, matrix):
    s = {"jc": paper_jc_nonrwa, "spin": paper_spin_chain, "opto": paper_optomechanics}[system]()
    L = liouvillian_sparse(s.H, s.c_ops)
    if matrix == "shifted":
        return shifted_liouvillian(L, 1e-15)
    return modified_liouvillian(L, s.d, default_weight(L))[0]


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "paper_rcm_bandwidth_profile.json")))["cases"],
                         ids=lambda c: f"{c['system']}-{c['matrix']}")
def test_paper_printed_bandwidth_profile(case):
    A = _paper_matrix(case["system"], case["matrix"])
    assert A.shape == (1024, 1024)
    B, P = bandwidth_profile(permute_symmetric(A, rcm_order(A)))[:2]
    assert B == case["B"]
    if case["profile_exact"]:
        assert P == case["P"]
    else:
        assert abs(P - case["P"]) / case["P"] < 1e-3
