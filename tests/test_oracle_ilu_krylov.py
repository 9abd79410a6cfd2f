"""Pins for the oracle's incomplete factorisations, triangular solves, Krylov
solvers and sparse steady-state drivers (section "Iterative solvers")."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp

from oracle import ilu
from oracle.krylov import BREAKDOWN, NOT_CONVERGED, OK, bicgstab, gmres, lgmres, select_method, steady_state_iterative
from oracle.metrics import trace_distance
from oracle.rng import splitmix64, start_vector
from oracle.steady import steady_state_dense
from workloads import driven_cavity, jaynes_cummings_rwa, kerr_oscillator, thermal_cavity

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_sparse(n, density, seed, dominance=4.0):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=rng, format="csr") \
        + 1j * sp.random(n, n, density=density, random_state=rng, format="csr")
    A = A + sp.diags(dominance * (1 + rng.random(n)) + 0.5j)
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A


def _tridiag(n, seed):
    rng = np.random.default_rng(seed)
    lo = rng.standard_normal(n - 1) + 1j * rng.standard_normal(n - 1)
    up = rng.standard_normal(n - 1) + 1j * rng.standard_normal(n - 1)
    dg = 6 + rng.random(n) + 1j * rng.random(n)
    return sp.csr_matrix(sp.diags([lo, dg, up], [-1, 0, 1]))


def _lu_nopivot(A):
    P, Lw, Uw = la.lu(A)
    assert np.allclose(P, np.eye(A.shape[0]))        # diagonally dominant: no row swaps
    return Lw, Uw


def test_ilu0_is_exact_lu_without_fill():
    A = _tridiag(40, 0)
    F = ilu.ilu0(A)
    Lw, Uw = _lu_nopivot(A.toarray())
    Lf, Uf = ilu.split_factors(F)
    np.testing.assert_allclose(Lf.toarray(), Lw, atol=1e-13)
    np.testing.assert_allclose(Uf.toarray(), Uw, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1])
def test_ilu0_matches_a_on_its_pattern(seed):
    """(L U)_ij = a_ij for every (i, j) in the pattern of A, and F has A's pattern."""
    A = _rand_sparse(60, 0.08, seed)
    F = ilu.ilu0(A)
    assert (F != 0).nnz <= A.nnz and np.array_equal(F.indptr, A.indptr) and np.array_equal(F.indices, A.indices)
    Lf, Uf = ilu.split_factors(F)
    LU = (Lf @ Uf).toarray()
    rows, cols = A.nonzero()
    np.testing.assert_allclose(LU[rows, cols], A.toarray()[rows, cols], atol=1e-12)


def test_ilu0_zero_pivot():
    A = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, 0.0]], dtype=complex))
    A.eliminate_zeros()
    with pytest.raises(ilu.ZeroPivot):
        ilu.ilu0(A)


def test_ilut_without_dropping_is_full_lu():
    A = _rand_sparse(50, 0.06, 2)
    F = ilu.ilut(A, drop_tol=0.0, fill_factor=1e6)
    Lw, Uw = _lu_nopivot(A.toarray())
    Lf, Uf = ilu.split_factors(F)
    np.testing.assert_allclose(Lf.toarray(), Lw, atol=1e-12)
    np.testing.assert_allclose(Uf.toarray(), Uw, atol=1e-12)


def test_ilut_respects_drop_and_fill_rules():
    A = _rand_sparse(80, 0.08, 3)
    drop, fill = 1e-2, 1.0
    F = ilu.ilut(A, drop_tol=drop, fill_factor=fill)
    for i in range(80):
        s, e = A.indptr[i], A.indptr[i + 1]
        tau = drop * np.max(np.abs(A.data[s:e]))
        cap = int(np.ceil(fill * (e - s) / 2))
        fs, fe = F.indptr[i], F.indptr[i + 1]
        cols, vals = F.indices[fs:fe], F.data[fs:fe]
        assert i in cols
        off = cols != i
        assert np.all(np.abs(vals[off]) >= tau)
        assert np.count_nonzero(cols < i) <= cap and np.count_nonzero(cols > i) <= cap


def test_ilut_large_drop_keeps_diagonal_only():
    A = _rand_sparse(30, 0.1, 4, dominance=100.0)
    F = ilu.ilut(A, drop_tol=0.5, fill_factor=10)
    assert np.array_equal(F.indices, np.arange(30))


def test_triangular_solves_match_dense():
    A = _rand_sparse(70, 0.07, 5)
    F = ilu.ilut(A, drop_tol=1e-3, fill_factor=3)
    Lf, Uf = ilu.split_factors(F)
    b = np.random.default_rng(0).standard_normal(70) + 1j
    y = ilu.lower_solve(F, b)
    np.testing.assert_allclose(y, la.solve_triangular(Lf.toarray(), b, lower=True), atol=1e-12)
    z = ilu.upper_solve(F, y)
    np.testing.assert_allclose(z, la.solve_triangular(Uf.toarray(), y, lower=False), atol=1e-12)
    np.testing.assert_allclose(ilu.precond_apply_fast(F, b), z, atol=1e-12)
    e = np.ones(70)
    M = Lf.toarray() @ Uf.toarray()
    assert ilu.condition_estimate(F) == pytest.approx(np.max(np.abs(np.linalg.solve(M, e))), rel=1e-10)


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
@pytest.mark.parametrize("seed", [0, 1])
def test_krylov_solves_random_system(solver, seed):
    A = _rand_sparse(120, 0.05, seed)
    b = np.random.default_rng(seed).standard_normal(120) + 0.5j
    F = ilu.ilu0(A)
    fn = bicgstab if solver == "bicgstab" else gmres
    res = fn(lambda v: A @ v, lambda r: ilu.precond_apply_fast(F, r), b, None, 1e-12, maxiter=500)
    assert res.status == OK
    np.testing.assert_allclose(res.x, np.linalg.solve(A.toarray(), b), atol=1e-11)


def test_unpreconditioned_gmres_full_restart_terminates_in_n_steps():
    n = 25
    A = _rand_sparse(n, 0.2, 7, dominance=1.0)
    b = np.ones(n, dtype=complex)
    res = gmres(lambda v: A @ v, lambda r: r, b, None, 1e-10, restart=n, maxiter=n)
    assert res.status == OK and res.iters <= n
    h = np.array(res.history[1:])
    assert np.all(np.diff(h) <= 1e-12 * h[0])          # minimal residual never increases


def test_exact_preconditioner_one_step():
    A = _rand_sparse(40, 0.1, 8)
    b = np.ones(40, dtype=complex)
    Ad = A.toarray()
    exact = lambda r: np.linalg.solve(Ad, r)           # noqa: E731
    assert bicgstab(lambda v: A @ v, exact, b, None, 1e-10).iters == 1
    assert gmres(lambda v: A @ v, exact, b, None, 1e-10).iters == 1


def test_bicgstab_breakdown_detected():
    """A skew-symmetric real A with r0 = b gives <r0, A r0> = 0: breakdown."""
    A = sp.csr_matrix(np.array([[0.0, 1.0], [-1.0, 0.0]], dtype=complex))
    res = bicgstab(lambda v: A @ v, lambda r: r, np.array([1.0, 0.0], dtype=complex), None, 1e-12)
    assert res.status == BREAKDOWN


def test_not_converged_status():
    A = _rand_sparse(200, 0.05, 9, dominance=0.05)
    b = np.ones(200, dtype=complex)
    res = bicgstab(lambda v: A @ v, lambda r: r, b, None, 1e-14, maxiter=3)
    assert res.status == NOT_CONVERGED and res.iters == 3


@pytest.mark.parametrize("method", ["bicgstab", "gmres", "inverse-power"])
@pytest.mark.parametrize("precond", ["ilu0", "ilut"])
@pytest.mark.parametrize("maker", [lambda: driven_cavity(n_th=0.2), lambda: jaynes_cummings_rwa(seed=1, N=8),
                                   lambda: kerr_oscillator(12, -0.7, 0.3, 1.1)],
                         ids=["cavity", "jc8", "kerr12"])
def test_sparse_iterative_steady_state_matches_dense(method, precond, maker):
    s = maker()
    ref = steady_state_dense(s.H, s.c_ops)
    res = steady_state_iterative(s.H, s.c_ops, method=method, precond=precond, tol=1e-12)
    assert res.status == OK and res.resid_Lrho <= 1e-12
    assert trace_distance(ref, res.rho) < 1e-10


def test_inverse_power_single_outer_step():
    """The inverse-power iteration converges in one outer step (section
    "Eigenvalue Methods")."""
    s = thermal_cavity(n_th=0.4)
    res = steady_state_iterative(s.H, s.c_ops, method="inverse-power", tol=1e-12)
    assert res.status == OK and res.outer_iters == 1


def test_weight_invariance():
    """rho does not depend on the weighting factor w of Eq. (linear)."""
    s = jaynes_cummings_rwa(seed=2, N=6)
    a = steady_state_iterative(s.H, s.c_ops, tol=1e-12)
    b = steady_state_iterative(s.H, s.c_ops, tol=1e-12, w=2 * a.w)
    assert a.status == OK and b.status == OK
    assert trace_distance(a.rho, b.rho) < 1e-10


def test_ordering_invariance():
    """The RCM-ordered and the naturally ordered solves reach the same rho."""
    s = driven_cavity(n_th=0.2)
    a = steady_state_iterative(s.H, s.c_ops, tol=1e-12, method="gmres")
    c = steady_state_iterative(s.H, s.c_ops, tol=1e-12, method="gmres", use_rcm=False)
    assert a.status == OK and c.status == OK
    assert trace_distance(a.rho, c.rho) < 1e-10


def test_splitmix64_published_vector():
    g = json.load(open(os.path.join(GOLD, "splitmix64_seed1234567.json")))
    G = 0x9E3779B97F4A7C15
    out = [splitmix64(g["seed"] + (k + 1) * G) for k in range(3)]
    assert out == g["outputs"]


def test_start_vector_counters():
    v = start_vector(1000, 42)
    assert np.all(np.abs(v.real) <= 1) and np.all(np.abs(v.imag) <= 1)
    G = 0x9E3779B97F4A7C15
    z = splitmix64(42 + 7 * G)                          # counter 6 = element 3, real part
    assert v[3].real == 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0


# ------------------------------------------------------------------ LGMRES

def _scipy_lgmres_cycles(op, b, m, k, cycles):
    """SciPy's independent LGMRES, unpreconditioned, run for exactly `cycles`
    restart cycles (a vanishing tolerance never ends a cycle early)."""
    from scipy.sparse.linalg import lgmres as sp_lgmres
    x, info = sp_lgmres(op, b, rtol=1e-300, atol=0.0, maxiter=cycles, inner_m=m, outer_k=k)
    assert info == cycles
    return x


@pytest.mark.parametrize("m,k", [(6, 2), (8, 3)])
def test_lgmres_matches_scipy_unpreconditioned(m, k):
    """With M = I, every cycle minimises over the same space as SciPy's
    LGMRES (Krylov directions of the restart residual plus the stored
    corrections), so the iterates agree after any number of cycles."""
    A = _rand_sparse(80, 0.06, 3, dominance=0.6)
    b = np.random.default_rng(3).standard_normal(80) + 0.3j
    for cycles in (1, 2, 5):
        ours = lgmres(lambda v: A @ v, lambda r: r, b, None, 0.0, restart=m, augment=k, maxiter=10**6,
                      max_cycles=cycles)
        ref = _scipy_lgmres_cycles(A, b, m, k, cycles)
        assert np.linalg.norm(ours.x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert ours.resid > 1e-8 * np.linalg.norm(b)          # still short of convergence: iterates carry the method


def test_lgmres_right_preconditioned_matches_scipy_on_a_minv():
    """Right preconditioning: the cycle space M^{-1} K_m(A M^{-1}, r) + span{dx_i}
    equals M^{-1} applied to the space SciPy's unpreconditioned LGMRES builds
    for the operator A M^{-1}, so x = M^{-1} u after each cycle."""
    from scipy.sparse.linalg import LinearOperator
    s = kerr_oscillator(10, -0.7, 0.3, 1.1)
    from oracle.liouvillian import default_weight, liouvillian_sparse, modified_liouvillian
    L = liouvillian_sparse(s.H, s.c_ops)
    A, b = modified_liouvillian(L, s.d, default_weight(L))
    A = sp.csr_matrix(A)
    A.sort_indices()
    F = ilu.ilut(A, drop_tol=5e-2, fill_factor=1.0)              # a deliberately rough M
    minv = lambda r: ilu.precond_apply_fast(F, r)                 # noqa: E731
    n = A.shape[0]
    op = LinearOperator((n, n), matvec=lambda u: A @ minv(u), dtype=np.complex128)
    for cycles in (1, 3, 4):
        ours = lgmres(lambda v: A @ v, minv, b, None, 0.0, restart=5, augment=2, maxiter=10**6,
                      max_cycles=cycles)
        ref = minv(_scipy_lgmres_cycles(op, b, 5, 2, cycles))
        assert np.linalg.norm(ours.x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert ours.resid > 1e-10 * np.linalg.norm(b)


def test_lgmres_without_augmentation_is_gmres():
    A = _rand_sparse(120, 0.05, 4)
    b = np.random.default_rng(4).standard_normal(120) + 0.1j
    F = ilu.ilut(A, drop_tol=0.3, fill_factor=1.0)                # rough M: several restart cycles
    ps = lambda r: ilu.precond_apply_fast(F, r)                   # noqa: E731
    a = lgmres(lambda v: A @ v, ps, b, None, 1e-12, restart=7, augment=0)
    g = gmres(lambda v: A @ v, ps, b, None, 1e-12, restart=7)
    assert a.status == g.status == OK and a.iters == g.iters
    np.testing.assert_allclose(a.x, g.x, rtol=0, atol=1e-13)


def test_lgmres_cycle_residuals_never_increase():
    """Each cycle minimises over a space that contains the zero correction."""
    A = _rand_sparse(150, 0.04, 5, dominance=0.4)
    b = np.ones(150, dtype=complex)
    prev = np.linalg.norm(b)
    x = None
    for _ in range(6):
        res = lgmres(lambda v: A @ v, lambda r: r, b, x, 0.0, restart=5, augment=3, maxiter=10**6,
                     max_cycles=1)
        x = res.x
        rn = np.linalg.norm(b - A @ x)
        assert rn <= prev * (1 + 1e-12)
        prev = rn


@pytest.mark.parametrize("maker", [lambda: driven_cavity(n_th=0.2), lambda: jaynes_cummings_rwa(seed=1, N=8)],
                         ids=["cavity", "jc8"])
def test_lgmres_steady_state_matches_dense(maker):
    s = maker()
    res = steady_state_iterative(s.H, s.c_ops, method="lgmres", augment=3, restart=10, tol=1e-12)
    assert res.status == OK and res.resid_Lrho <= 1e-12
    assert trace_distance(steady_state_dense(s.H, s.c_ops), res.rho) < 1e-10


# ------------------------------------------------------- method selection

def test_select_method_on_the_papers_printed_bandwidths():
    """Fig. 1 and Fig. 3 print the RCM bandwidths of L - sigma I and L~ for
    the three model systems; the selection rule reads them: GMRES on L~ for
    the Jaynes-Cummings and optomechanical models (bandwidth nearly
    unchanged), inverse power for the 5-spin chain (bandwidth 2.4x)."""
    from workloads import paper_jc_nonrwa, paper_optomechanics, paper_spin_chain
    gold = json.load(open(os.path.join(GOLD, "paper_rcm_bandwidth_profile.json")))["cases"]
    B = {(c["system"], c["matrix"]): c["B"] for c in gold}
    expect = {"jc": "gmres", "spin": "power-gmres", "opto": "gmres"}
    for name, maker in (("jc", paper_jc_nonrwa), ("spin", paper_spin_chain), ("opto", paper_optomechanics)):
        s = maker()
        method, bm, bs = select_method(s.H, s.c_ops)
        assert (bm, bs) == (B[(name, "modified")], B[(name, "shifted")])
        assert method == expect[name], name


def test_auto_steady_state_matches_dense():
    s = driven_cavity(n_th=0.2)
    res = steady_state_iterative(s.H, s.c_ops, method="auto", tol=1e-12, augment=2)
    assert res.status == OK
    assert trace_distance(steady_state_dense(s.H, s.c_ops), res.rho) < 1e-10
