"""The library's host-side steps (RCM ordering, level sets, ILUT), called
through their C entry points on the CPU, against the oracle and the paper's
printed bandwidths."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ilu as oilu
from oracle.liouvillian import default_weight, liouvillian_sparse, modified_liouvillian, shifted_liouvillian
from oracle.ordering import bandwidth_profile, permute_symmetric, rcm_order
from workloads import (driven_cavity, jaynes_cummings_rwa, kerr_oscillator, paper_jc_nonrwa, paper_optomechanics,
                       paper_spin_chain, random_system)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ss():
    import __graft_entry__ as g
    g.build()
    import paper_1504_06768_gb300 as lib
    return lib


def _modified(s):
    L = liouvillian_sparse(s.H, s.c_ops)
    A = sp.csr_matrix(modified_liouvillian(L, s.d, default_weight(L))[0])
    A.sort_indices()
    return A


SYSTEMS = {"cavity": lambda: driven_cavity(n_th=0.2), "jc8": lambda: jaynes_cummings_rwa(seed=3, N=8),
           "kerr12": lambda: kerr_oscillator(12, -0.7, 0.3, 1.1), "random7": lambda: random_system(7, n_c=3, seed=5)}


@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_rcm_host_is_the_oracles_order(ss, name):
    A = _modified(SYSTEMS[name]())
    assert np.array_equal(ss.rcm_order_host(A), rcm_order(A))


def test_rcm_host_disconnected_components(ss):
    """Two components and an isolated node: one pass per component."""
    blocks = [sp.random(9, 9, density=0.3, random_state=np.random.default_rng(1)), sp.identity(1),
              sp.random(6, 6, density=0.4, random_state=np.random.default_rng(2))]
    A = sp.csr_matrix(sp.block_diag(blocks) + sp.identity(16))
    A.sort_indices()
    p = ss.rcm_order_host(A)
    assert sorted(p.tolist()) == list(range(16))
    assert np.array_equal(p, rcm_order(A))


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "paper_rcm_bandwidth_profile.json")))["cases"],
                         ids=lambda c: f"{c['system']}-{c['matrix']}")
def test_rcm_host_reproduces_printed_bandwidth(ss, case):
    """Fig. 1 and Fig. 3 print the RCM bandwidth of each matrix."""
    s = {"jc": paper_jc_nonrwa, "spin": paper_spin_chain, "opto": paper_optomechanics}[case["system"]]()
    L = liouvillian_sparse(s.H, s.c_ops)
    A = shifted_liouvillian(L, 1e-15) if case["matrix"] == "shifted" else modified_liouvillian(L, s.d,
                                                                                               default_weight(L))[0]
    A = sp.csr_matrix(A)
    A.sort_indices()
    assert bandwidth_profile(permute_symmetric(A, ss.rcm_order_host(A)))[0] == case["B"]


@pytest.mark.parametrize("lower", [True, False])
def test_level_sets_host(ss, lower):
    A = _modified(SYSTEMS["jc8"]())
    A = permute_symmetric(A, rcm_order(A))
    order, ptr = ss.level_sets_host(A, lower)
    n = A.shape[0]
    assert sorted(order.tolist()) == list(range(n)) and ptr[0] == 0 and ptr[-1] == n
    level = np.empty(n, dtype=np.int64)
    for lv in range(len(ptr) - 1):
        rows = order[ptr[lv]:ptr[lv + 1]]
        assert np.all(np.diff(rows) > 0)                         # ascending inside a level
        level[rows] = lv
    for i in range(n):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        deps = cols[cols < i] if lower else cols[cols > i]
        # every dependency sits in an earlier level, and one in the level just before
        assert np.all(level[deps] < level[i])
        assert (level[i] == 0) == (len(deps) == 0)
        if len(deps):
            assert level[deps].max() == level[i] - 1


@pytest.mark.parametrize("name", ["cavity", "jc8", "kerr12"])
@pytest.mark.parametrize("drop,fill", [(1e-4, 10.0), (1e-2, 2.0), (0.0, 50.0)])
def test_ilut_host_matches_oracle(ss, name, drop, fill):
    A = _modified(SYSTEMS[name]())
    A = sp.csr_matrix(permute_symmetric(A, rcm_order(A)))
    A.sort_indices()
    got = ss.ilut_host(A, drop, fill)
    ref = sp.csr_matrix(oilu.ilut(A, drop_tol=drop, fill_factor=fill))
    ref.sort_indices()
    assert np.array_equal(got.indptr, ref.indptr) and np.array_equal(got.indices, ref.indices)
    assert np.max(np.abs(got.data - ref.data)) <= 1e-12 * np.max(np.abs(ref.data))


@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_ilu0_schedule_reproduces_the_oracles_ilu0(ss, name):
    """The batched solver factors each system from its pattern's elimination
    schedule.  Eliminating with the schedule alone (for each row, each pivot
    in ascending order: l = a_it / u_kk, then a_ij -= l u_kj for the listed
    pairs) gives the oracle's iLU(0) of the RCM-ordered trace-row system."""
    A = _modified(SYSTEMS[name]())
    Ap = sp.csr_matrix(permute_symmetric(A, rcm_order(A)))
    Ap.sort_indices()
    ptr, tgt, src = ss.ilu0_schedule_host(Ap)
    rp, col = Ap.indptr, Ap.indices
    n = Ap.shape[0]
    dpos = np.array([rp[i] + int(np.searchsorted(col[rp[i]:rp[i + 1]], i)) for i in range(n)])
    a = [complex(v) for v in Ap.data]
    for i in range(n):
        for t in range(rp[i], dpos[i]):
            k = col[t]
            a[t] = a[t] / a[dpos[k]]
            for p in range(ptr[t], ptr[t + 1]):
                j = rp[i] + tgt[p]
                assert t < j < rp[i + 1] and dpos[k] < src[p] < rp[k + 1] and col[j] == col[src[p]]
                a[j] = a[j] - a[t] * a[src[p]]
    ref = oilu.ilu0(Ap)
    ref.sort_indices()
    assert np.array_equal(ref.indptr, rp) and np.array_equal(ref.indices, col)
    got = np.array(a)
    assert np.max(np.abs(got - ref.data)) <= 1e-13 * np.max(np.abs(ref.data))
    # positions that are not pivots have empty ranges
    pivots = np.zeros(rp[-1], dtype=bool)
    for i in range(n):
        pivots[rp[i]:dpos[i]] = True
    assert np.all(np.diff(ptr)[~pivots] == 0)


def test_ilu0_schedule_host_rejects_missing_diagonal(ss):
    A = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 1.0]], dtype=complex))
    A.eliminate_zeros()
    with pytest.raises(ss.SolverError) as e:
        ss.ilu0_schedule_host(A)
    assert e.value.status == 5


def test_ilut_host_zero_pivot(ss):
    A = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 1.0]], dtype=complex))
    with pytest.raises(ss.SolverError) as e:
        ss.ilut_host(A)
    assert e.value.status == 5


def test_host_entry_points_reject_malformed_csr(ss):
    import ctypes as C
    from paper_1504_06768_gb300 import _binding as B
    rp = np.array([0, 2, 3], dtype=np.int32)
    col = np.array([1, 0, 1], dtype=np.int32)                     # row 0 not ascending
    perm = np.empty(2, dtype=np.int32)
    assert B.load().ss_rcm_order_host(2, rp.ctypes.data, col.ctypes.data, perm.ctypes.data) == B.SS_ERR_INVALID
    col = np.array([0, 2, 1], dtype=np.int32)                     # column out of range
    assert B.load().ss_rcm_order_host(2, rp.ctypes.data, col.ctypes.data, perm.ctypes.data) == B.SS_ERR_INVALID
    nl = C.c_int32()
    order = np.empty(2, dtype=np.int32)
    ptr = np.empty(3, dtype=np.int32)
    assert B.load().ss_level_sets_host(2, rp.ctypes.data, col.ctypes.data, 1, order.ctypes.data, ptr.ctypes.data,
                                       C.byref(nl)) == B.SS_ERR_INVALID


# ---------------------------------------------------------- bipartite matching

def _random_complex(n, density, seed):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=rng, format="csr")
    A.data = A.data + 1j * rng.random(A.nnz)
    A.data[rng.random(A.nnz) < 0.2] = 1.0                          # ties of equal weight
    A.sort_indices()
    return A


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("density", [0.03, 0.1])
def test_mbm_host_is_the_oracles_matching(ss, seed, density):
    from oracle.matching import weighted_mbm
    A = _random_complex(80, density, seed)
    match, k = ss.mbm_host(A)
    ref, kr = weighted_mbm(A)
    assert k == kr and np.array_equal(match, ref)


@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_mbm_host_on_trace_row_liouvillians(ss, name):
    from oracle.matching import weighted_mbm
    A = _modified(SYSTEMS[name]())
    match, k = ss.mbm_host(A)
    ref, kr = weighted_mbm(A)
    assert k == kr == A.shape[0] and np.array_equal(match, ref)
    assert np.all(A[match, :].diagonal() != 0)


# ------------------------------------------------------------- autotuner

def _table(fn):
    t = np.empty((4, 4, 4, 2))
    for lo in range(4):
        for up in range(4):
            for a in range(4):
                for st in range(2):
                    t[lo, up, a, st] = fn(lo - 1, up - 1, a - 1, st)
    return t


def test_tune_search_finds_minimum_of_a_separable_bowl():
    """Coordinate descent reaches the minimum of a separable cost (the rule
    choice is (0, 0, 0, 0); the best is (1, -1, 2, 1))."""
    import paper_1504_06768_gb300 as ss
    t = _table(lambda lo, up, a, st: 10 + (lo - 1) ** 2 + 2 * (up + 1) ** 2 + 0.5 * (a - 2) ** 2 + (0 if st else 1))
    best, probes = ss.tune_search_host(t)
    assert best == (1, -1, 2, 1)
    assert probes <= 4 * 4 * 4 * 2 and probes < 20           # memoised: far fewer than the whole table


def test_tune_search_keeps_rule_choice_when_nothing_is_better_by_one_percent():
    import paper_1504_06768_gb300 as ss
    t = _table(lambda lo, up, a, st: 1.0 + 0.001 * (lo + up + a + st) ** 2)    # < 1 % apart everywhere
    best, probes = ss.tune_search_host(t)
    assert best == (0, 0, 0, 0)
    assert probes == 1 + 2 + 2 + 2 + 1                        # the start and each coordinate's neighbours once


def test_tune_search_stops_at_local_minimum_and_respects_probe_cap():
    import paper_1504_06768_gb300 as ss
    # an isolated global minimum that no single-coordinate move approaches
    t = _table(lambda lo, up, a, st: 0.1 if (lo, up, a, st) == (2, 2, 2, 1) else
               5 + abs(lo) + abs(up) + abs(a) + st)
    best, probes = ss.tune_search_host(t)
    assert best == (0, 0, 0, 0)
    _, capped = ss.tune_search_host(_table(lambda lo, up, a, st: 10 - lo - up - a - st), max_probes=3)
    assert capped == 3
