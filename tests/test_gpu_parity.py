"""GPU parity: every step of the CUDA path, called through the C ABI, against
the CPU oracle on the same seeded inputs."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ilu as oilu
from oracle.liouvillian import (default_weight, liouvillian_apply, liouvillian_row, liouvillian_sparse,
                                modified_liouvillian, shifted_liouvillian)
from oracle.metrics import hermiticity_error, min_eigenvalue, trace_distance
from oracle.ordering import bandwidth_profile as o_bwp
from oracle.ordering import permute_symmetric, rcm_order
from oracle.steady import steady_state_dense
from workloads import (driven_cavity, jaynes_cummings_rwa, kerr_chain, kerr_oscillator, kerr_sweep, optomechanics,
                       paper_jc_nonrwa, paper_optomechanics, paper_spin_chain, random_system, thermal_cavity,
                       two_level_atom)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    import paper_1504_06768_gb300 as lib
    return lib


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.complex128, device="cuda")


def _same_pattern(a, b):
    a, b = sp.csr_matrix(a), sp.csr_matrix(b)
    a.sort_indices()
    b.sort_indices()
    return a.shape == b.shape and np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices)


def _assert_close_csr(got, ref, rtol=1e-14):
    got, ref = sp.csr_matrix(got), sp.csr_matrix(ref)
    got.sort_indices()
    ref.sort_indices()
    assert _same_pattern(got, ref)
    scale = max(np.max(np.abs(ref.data)), 1e-300) if ref.nnz else 1.0
    assert np.max(np.abs(got.data - ref.data), initial=0.0) <= rtol * scale


SMALL_SYSTEMS = {
    "random5": lambda: random_system(5, n_c=2, seed=0),
    "random7": lambda: random_system(7, n_c=3, density=0.3, seed=5),
    "cavity": lambda: driven_cavity(n_th=0.0),
    "cavity_thermal": lambda: driven_cavity(n_th=0.2),
    "thermal": lambda: thermal_cavity(),
    "jc8": lambda: jaynes_cummings_rwa(seed=3, N=8),
    "kerr17": lambda: kerr_oscillator(17, 0.4, 0.3, 1.2),
    "opto3x6": lambda: optomechanics(seed=1, Nc=3, Nm=6),
    "paper_jc": lambda: paper_jc_nonrwa(),
    "paper_spin": lambda: paper_spin_chain(),
    "paper_opto": lambda: paper_optomechanics(),
    "two_level": lambda: two_level_atom(),
}


# ------------------------------------------------------------------ assembly

@pytest.mark.parametrize("name", sorted(SMALL_SYSTEMS))
def test_assembly_matches_oracle(ss, name):
    s = SMALL_SYSTEMS[name]()
    L = ss.assemble_liouvillian(s.H, s.c_ops).to_scipy()
    _assert_close_csr(L, liouvillian_sparse(s.H, s.c_ops))


@pytest.mark.parametrize("maker", [lambda: jaynes_cummings_rwa(seed=0), lambda: optomechanics(seed=0)],
                         ids=["jc40_n6400", "opto10x40_n160000"])
def test_assembly_full_size_configs(ss, maker):
    s = maker()
    L = ss.assemble_liouvillian(s.H, s.c_ops).to_scipy()
    _assert_close_csr(L, liouvillian_sparse(s.H, s.c_ops))


def test_assembly_chain_full_size_by_action_and_rows(ss):
    """The 3-site Kerr chain (n = 2,985,984): L x on the GPU equals the
    matrix-free Eq. (lindblad) for a random x, and sampled rows equal the
    element-wise form."""
    import torch
    s = kerr_chain()
    Lm = ss.assemble_liouvillian(s.H, s.c_ops)
    n = s.n
    assert Lm.shape == (n, n)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = ss.spmv(Lm, _dev(x)).cpu().numpy()
    ref = liouvillian_apply(s.H, s.c_ops, x)
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    Ls = Lm.to_scipy()
    for p in list(rng.integers(0, n, size=12)) + [0, n - 1]:
        row = liouvillian_row(s.H, s.c_ops, int(p))
        got = np.zeros(n, dtype=complex)
        a, b = Ls.indptr[p], Ls.indptr[p + 1]
        got[Ls.indices[a:b]] = Ls.data[a:b]
        assert np.array_equal(np.flatnonzero(got), np.flatnonzero(row))
        assert np.max(np.abs(got - row)) <= 1e-14 * max(1.0, np.max(np.abs(row)))


# ---------------------------------------------------------- trace row, shift

@pytest.mark.parametrize("name", ["cavity", "jc8", "paper_jc", "paper_spin", "random5"])
def test_trace_row_and_shift(ss, name):
    s = SMALL_SYSTEMS[name]()
    Lm = ss.assemble_liouvillian(s.H, s.c_ops)
    L = Lm.to_scipy()
    Lt, w = ss.add_trace_row(Lm)
    assert w == pytest.approx(default_weight(L), rel=1e-13)
    ref, _ = modified_liouvillian(L, s.d, w)
    _assert_close_csr(Lt.to_scipy(), ref)
    Lt2, w2 = ss.add_trace_row(Lm, w=2.5)
    assert w2 == 2.5
    _assert_close_csr(Lt2.to_scipy(), modified_liouvillian(L, s.d, 2.5)[0])
    S = ss.add_shift(Lm, 1e-15).to_scipy()
    _assert_close_csr(S, shifted_liouvillian(L, 1e-15))


# ------------------------------------------------------------- ordering

@pytest.mark.parametrize("system", ["paper_jc", "paper_spin", "paper_opto"])
@pytest.mark.parametrize("kind", ["shifted", "modified"])
def test_rcm_bit_exact_and_printed_values(ss, system, kind):
    import json
    import os
    s = SMALL_SYSTEMS[system]()
    Lm = ss.assemble_liouvillian(s.H, s.c_ops)
    A = ss.add_shift(Lm, 1e-15) if kind == "shifted" else ss.add_trace_row(Lm)[0]
    perm, bw, prof = ss.rcm_permute(A)
    ref = rcm_order(A.to_scipy())
    assert np.array_equal(perm, ref)
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_rcm_bandwidth_profile.json")))
    case = [c for c in gold["cases"] if c["system"] == system.split("_")[1] and c["matrix"] == kind][0]
    assert bw == case["B"]
    if case["profile_exact"]:
        assert prof == case["P"]
    assert (bw, prof) == o_bwp(permute_symmetric(A.to_scipy(), ref))[:2]


@pytest.mark.parametrize("maker", [lambda: jaynes_cummings_rwa(seed=0), lambda: optomechanics(seed=0)],
                         ids=["jc40", "opto10x40"])
def test_rcm_bit_exact_full_size(ss, maker):
    s = maker()
    A, _ = ss.add_trace_row(ss.assemble_liouvillian(s.H, s.c_ops))
    perm, bw, prof = ss.rcm_permute(A)
    assert np.array_equal(perm, rcm_order(A.to_scipy()))


@pytest.mark.parametrize("name", ["cavity", "paper_opto", "random7"])
def test_permute_and_bandwidth(ss, name):
    s = SMALL_SYSTEMS[name]()
    A, _ = ss.add_trace_row(ss.assemble_liouvillian(s.H, s.c_ops))
    As = A.to_scipy()
    perm = np.random.default_rng(1).permutation(As.shape[0]).astype(np.int32)
    P = ss.permute(A, perm)
    ref = permute_symmetric(As, perm)
    got = P.to_scipy()
    assert _same_pattern(got, ref) and np.array_equal(got.data, sp.csr_matrix(ref).data)
    assert ss.bandwidth_profile(P) == o_bwp(ref)[:2]


# ---------------------------------------------------------- preconditioner

def _rcm_system(ss, s, shifted=False):
    Lm = ss.assemble_liouvillian(s.H, s.c_ops)
    A = ss.add_shift(Lm, 1e-15) if shifted else ss.add_trace_row(Lm)[0]
    perm, _, _ = ss.rcm_permute(A)
    return ss.permute(A, perm)


@pytest.mark.parametrize("name", ["cavity", "jc8", "kerr17", "paper_opto", "opto3x6"])
@pytest.mark.parametrize("shifted", [False, True])
def test_ilu0_matches_oracle(ss, name, shifted):
    Ap = _rcm_system(ss, SMALL_SYSTEMS[name](), shifted)
    M = ss.ilu_factor(Ap, "ilu0")
    n = Ap.shape[0]
    got = M.to_scipy(n)
    ref = oilu.ilu0(Ap.to_scipy())
    _assert_close_csr(got, ref, rtol=1e-12)
    assert M.condest == pytest.approx(oilu.condition_estimate(ref), rel=1e-9)


def test_ilu0_spin_chain(ss):
    """Eq. spinchain: the populations of L~ have no diagonal entry, so iLU(0)
    meets a zero pivot on both sides; for L - sigma I those pivots are -sigma
    (1e-15), the factors are of size 1e15 and only the pattern is compared."""
    s = paper_spin_chain()
    Ap = _rcm_system(ss, s, shifted=False)
    with pytest.raises(oilu.ZeroPivot):
        oilu.ilu0(Ap.to_scipy())
    with pytest.raises(ss.SolverError) as e:
        ss.ilu_factor(Ap, "ilu0")
    assert e.value.status == 5
    As = _rcm_system(ss, s, shifted=True)
    got = ss.ilu_factor(As, "ilu0").to_scipy(As.shape[0])
    ref = oilu.ilu0(As.to_scipy())
    assert _same_pattern(got, ref) and np.all(np.isfinite(got.data))


@pytest.mark.parametrize("maker", [lambda: driven_cavity(n_th=0.2), lambda: jaynes_cummings_rwa(seed=2, N=20)],
                         ids=["cavity", "jc20"])
def test_ilut_matches_oracle(ss, maker):
    Ap = _rcm_system(ss, maker())
    M = ss.ilu_factor(Ap, "ilut", drop_tol=1e-4, fill_factor=10)
    ref = oilu.ilut(Ap.to_scipy(), drop_tol=1e-4, fill_factor=10)
    _assert_close_csr(M.to_scipy(Ap.shape[0]), ref, rtol=1e-12)


@pytest.mark.parametrize("kind", ["ilu0", "ilut"])
@pytest.mark.parametrize("name", ["jc8", "paper_opto"])
def test_precond_apply_matches_oracle(ss, kind, name):
    Ap = _rcm_system(ss, SMALL_SYSTEMS[name]())
    M = ss.ilu_factor(Ap, kind, precision="mixed")
    n = Ap.shape[0]
    F = M.to_scipy(n)
    r = np.random.default_rng(4).standard_normal(n) + 1j * np.random.default_rng(5).standard_normal(n)
    z = ss.precond_apply(M, _dev(r)).cpu().numpy()
    ref = oilu.upper_solve(F, oilu.lower_solve(F, r))
    assert np.max(np.abs(z - ref)) <= 1e-12 * np.max(np.abs(ref))
    import torch
    z32 = ss.precond_apply_f32(M, _dev(r).to(torch.complex64)).cpu().numpy()
    assert np.max(np.abs(z32 - ref)) <= 1e-3 * np.max(np.abs(ref))


def test_precond_apply_repeated_launches_are_identical(ss):
    """Sync-free solves reuse their tickets and flags: 50 launches in a row
    give bit-identical results."""
    Ap = _rcm_system(ss, jaynes_cummings_rwa(seed=1, N=12))
    M = ss.ilu_factor(Ap, "ilu0")
    r = _dev(np.random.default_rng(0).standard_normal(Ap.shape[0]) + 0j)
    first = ss.precond_apply(M, r).cpu().numpy()
    for _ in range(50):
        z = ss.precond_apply(M, r).cpu().numpy()
    assert np.array_equal(first, z)


# ------------------------------------------------------------------ SpMV

@pytest.mark.parametrize("name", ["cavity", "paper_spin", "random7"])
def test_spmv_matches_oracle(ss, name):
    import torch
    Ap = _rcm_system(ss, SMALL_SYSTEMS[name]())
    As = Ap.to_scipy()
    n = As.shape[0]
    x = np.random.default_rng(2).standard_normal(n) + 1j * np.random.default_rng(3).standard_normal(n)
    y = ss.spmv(Ap, _dev(x)).cpu().numpy()
    ref = As @ x
    assert np.max(np.abs(y - ref)) <= 1e-14 * np.max(np.abs(As).sum(axis=1)) * np.max(np.abs(x))
    y32 = ss.spmv_f32(Ap, _dev(x).to(torch.complex64)).cpu().numpy()
    assert np.max(np.abs(y32 - ref)) <= 1e-5 * np.max(np.abs(As).sum(axis=1)) * np.max(np.abs(x))


# ----------------------------------------------------------------- Krylov

@pytest.mark.parametrize("method", ["bicgstab", "gmres"])
@pytest.mark.parametrize("name", ["cavity_thermal", "jc8", "kerr17"])
def test_krylov_solves_trace_row_system(ss, method, name):
    s = SMALL_SYSTEMS[name]()
    Lm = ss.assemble_liouvillian(s.H, s.c_ops)
    A, w = ss.add_trace_row(Lm)
    perm, _, _ = ss.rcm_permute(A)
    Ap = ss.permute(A, perm)
    M = ss.ilu_factor(Ap, "ilu0")
    n = Ap.shape[0]
    b = np.zeros(n, dtype=complex)
    b[np.flatnonzero(perm == 0)[0]] = w
    x, st, it, res = ss.krylov_solve(Ap, M, _dev(b), method=method, tol=1e-13 * w)
    assert st == 0 and res <= 1e-13 * w
    ref = np.linalg.solve(Ap.to_scipy().toarray(), b)
    assert np.max(np.abs(x.cpu().numpy() - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_bicgstab_breakdown_reported(ss):
    """A skew-symmetric real A with r0 = b gives <r0, A r0> = 0."""
    A = ss.Matrix.from_scipy(sp.csr_matrix(np.array([[0, 1.0], [-1.0, 0]], dtype=complex)))
    M = ss.ilu_factor(ss.Matrix.from_scipy(sp.identity(2, dtype=complex, format="csr")), "ilu0")
    x, st, it, res = ss.krylov_solve(A, M, _dev(np.array([1.0, 0.0])), method="bicgstab", tol=1e-12)
    assert st == 4 and it == 0


def test_not_converged_reported(ss):
    s = jaynes_cummings_rwa(seed=0, N=12)
    rho, info = ss.steady_state(s.H, s.c_ops, tol=1e-14, maxiter=3, raise_on_failure=False)
    assert info["status"] == 3 and info["iters"] <= 3
    assert rho.shape == (24, 24) and np.all(np.isfinite(rho))


def test_zero_pivot_reported(ss):
    A = ss.Matrix.from_scipy(sp.csr_matrix(np.array([[0, 1.0], [1.0, 1.0]], dtype=complex)))
    with pytest.raises(ss.SolverError) as e:
        ss.ilu_factor(A, "ilu0")
    assert e.value.status == 5


def test_invalid_inputs_reported(ss):
    with pytest.raises(ss.SolverError) as e:
        ss.steady_state(sp.csr_matrix(np.ones((2, 3), dtype=complex)), [])
    assert e.value.status == 1
    s = driven_cavity(N=4)
    with pytest.raises(ss.SolverError) as e:
        ss.steady_state(s.H, [sp.identity(3, dtype=complex, format="csr")])
    assert e.value.status == 1
    import ctypes as C
    from paper_1504_06768_gb300 import _binding as B
    opt = ss._options("direct", 1e-10, "ilu0", "fp64", 1000, 30, 1e-4, 10.0, 0.0, 1e-15, True, 0)
    opt.method = 9                                                    # no such method
    hv = ss._CsrHost(s.H)
    cvs = [ss._CsrHost(c) for c in s.c_ops]
    arr = (B.CsrView * len(cvs))(*[c.view for c in cvs])
    rho = np.empty(s.d * s.d, dtype=np.complex128)
    ctx = ss.get_context()
    assert B.load().steady_state(ctx.handle, C.byref(hv.view), len(cvs), arr, C.byref(opt), rho.ctypes.data, 0,
                                 None) == 1


# ------------------------------------------------------------ steady state

CONFIG1 = {"coherent": lambda: driven_cavity(n_th=0.0), "thermal_driven": lambda: driven_cavity(n_th=0.2),
           "thermal": lambda: thermal_cavity(n_th=0.2)}


@pytest.mark.parametrize("method", ["iterative-bicgstab", "iterative-lgmres", "inverse-power"])
@pytest.mark.parametrize("precond", ["ilu0", "ilut"])
@pytest.mark.parametrize("name", sorted(CONFIG1))
def test_steady_state_config1(ss, method, precond, name):
    s = CONFIG1[name]()
    rho, info = ss.steady_state(s.H, s.c_ops, method=method, precond=precond, tol=1e-12)
    ref = steady_state_dense(s.H, s.c_ops)
    assert info["status"] == 0 and info["resid_Lrho"] <= 1e-12
    assert trace_distance(rho, ref) <= 1e-10
    assert abs(np.trace(rho) - 1) < 1e-13
    assert hermiticity_error(rho) < 1e-10 and min_eigenvalue(rho) > -1e-10


def test_closed_forms_on_gpu(ss):
    import math
    s = driven_cavity(N=30, delta=0.5, E=0.3, kappa=1.0)
    rho, _ = ss.steady_state(s.H, s.c_ops, tol=1e-12)
    alpha = -1j * 0.3 / (1j * 0.5 + 0.5)
    k = np.arange(30)
    c = np.exp(-abs(alpha) ** 2 / 2) * alpha ** k / np.sqrt(np.array([math.factorial(int(i)) for i in k], dtype=float))
    c /= np.linalg.norm(c)
    assert trace_distance(rho, np.outer(c, c.conj())) < 1e-10
    s = thermal_cavity(n_th=0.2)
    rho, _ = ss.steady_state(s.H, s.c_ops, method="inverse-power", tol=1e-12)
    assert float(np.sum(np.arange(20) * np.diag(rho).real)) == pytest.approx(0.2, abs=1e-10)


@pytest.mark.parametrize("seed,method,precond", [(0, "iterative-bicgstab", "ilut"), (0, "iterative-lgmres", "ilut"),
                                                 (0, "inverse-power", "ilut"), (7, "iterative-bicgstab", "ilu0"),
                                                 (7, "iterative-lgmres", "ilu0"), (7, "inverse-power", "ilu0")])
def test_steady_state_config2_jc40(ss, seed, method, precond):
    s = jaynes_cummings_rwa(seed=seed)
    rho, info = ss.steady_state(s.H, s.c_ops, method=method, precond=precond, tol=1e-12)
    assert info["n"] == 6400 and info["status"] == 0
    ref = _dense_ref(seed)
    assert trace_distance(rho, ref) <= 1e-10


_DENSE_CACHE = {}


def _dense_ref(seed):
    if seed not in _DENSE_CACHE:
        s = jaynes_cummings_rwa(seed=seed)
        _DENSE_CACHE[seed] = steady_state_dense(s.H, s.c_ops)
    return _DENSE_CACHE[seed]


def test_edge_case_one_state(ss):
    H = sp.csr_matrix(np.array([[0.7]], dtype=complex))
    rho, info = ss.steady_state(H, [])
    assert info["status"] == 0 and rho.shape == (1, 1) and abs(rho[0, 0] - 1) < 1e-14


def test_two_level_atom_closed_form(ss):
    s = two_level_atom(omega=1.0, gamma=0.5)
    for method in ("iterative-bicgstab", "iterative-lgmres", "inverse-power"):
        rho, info = ss.steady_state(s.H, s.c_ops, method=method, tol=1e-13)
        assert rho[1, 1].real == pytest.approx(1.0 / (0.25 + 2.0), abs=1e-11)


def test_rho_written_to_device_buffer(ss):
    import torch
    s = driven_cavity(N=10, n_th=0.1)
    out = torch.empty(100, dtype=torch.complex128, device="cuda")
    rho, info = ss.steady_state(s.H, s.c_ops, out=out, tol=1e-12)
    assert trace_distance(rho.cpu().numpy(), steady_state_dense(s.H, s.c_ops)) < 1e-10


def test_config3_optomechanics_mixed(ss):
    """Optomechanics 10 x 40 (n = 160,000): the FP32-inner / FP64-refined
    solve reaches ||L rho|| <= 1e-10 and agrees with the FP64 GPU solve
    (trace distance <= 1e-8) and with the CPU sparse iterative oracle."""
    from oracle.krylov import steady_state_iterative
    s = optomechanics(seed=0)
    rho_m, info_m = ss.steady_state(s.H, s.c_ops, precision="mixed", tol=1e-10)
    assert info_m["status"] == 0 and info_m["resid_Lrho"] <= 1e-10 and info_m["n"] == 160000
    rho_d, info_d = ss.steady_state(s.H, s.c_ops, tol=1e-11)
    assert info_d["status"] == 0
    assert trace_distance(rho_m, rho_d) <= 1e-8
    ref = steady_state_iterative(s.H, s.c_ops, method="bicgstab", precond="ilu0", tol=1e-11)
    assert ref.status == 0
    assert trace_distance(rho_d, ref.rho) <= 1e-9


def test_config3_optomechanics_mixed_falls_back_to_fp64(ss):
    """The second optomechanics system (seed 1) is beyond FP32 for the inner
    solves: one stalls at its iteration cap, the remaining iterations run in
    FP64 from the refined iterate (fp64_fallback), and the result reaches
    ||L rho|| <= 1e-10 and agrees with the FP64 solve."""
    s = optomechanics(seed=1)
    rho_m, info_m = ss.steady_state(s.H, s.c_ops, precision="mixed", tol=1e-10)
    assert info_m["status"] == 0 and info_m["resid_Lrho"] <= 1e-10
    assert info_m["fp64_fallback"] == 1 and info_m["iters"] <= 1000
    rho_d, info_d = ss.steady_state(s.H, s.c_ops, tol=1e-11)
    assert info_d["status"] == 0 and info_d["fp64_fallback"] == 0
    assert trace_distance(rho_m, rho_d) <= 1e-8


@pytest.mark.parametrize("name", ["cavity_thermal", "kerr17", "jc8"])
def test_mixed_single_system_small(ss, name):
    s = SMALL_SYSTEMS[name]()
    rho, info = ss.steady_state(s.H, s.c_ops, precision="mixed", tol=1e-11)
    assert info["status"] == 0 and info["resid_Lrho"] <= 1e-11 and info["outer_iters"] >= 2
    assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-8


# ------------------------------------------------------------ direct method

@pytest.mark.parametrize("maker", [lambda: driven_cavity(n_th=0.0), lambda: driven_cavity(n_th=0.2),
                                   lambda: thermal_cavity(n_th=0.2), lambda: two_level_atom(),
                                   lambda: jaynes_cummings_rwa(seed=2, N=12), lambda: kerr_sweep(1, seed=4)[0]],
                         ids=["coherent", "thermal_driven", "thermal", "two_level", "jc12", "kerr"])
def test_direct_banded_lu_matches_oracle(ss, maker):
    """method=direct: banded LU with partial pivoting of the RCM-ordered L~ on
    the device, against the dense FP64 LU of the oracle."""
    s = maker()
    rho, info = ss.steady_state(s.H, s.c_ops, method="direct", tol=1e-10)
    assert info["status"] == 0 and info["iters"] == 0 and info["resid_Lrho"] <= 1e-10
    assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-10
    assert abs(np.trace(rho) - 1) < 1e-12


def test_direct_jc40_full_size(ss):
    s = jaynes_cummings_rwa(seed=0)
    rho, info = ss.steady_state(s.H, s.c_ops, method="direct", tol=1e-10)
    assert info["status"] == 0 and info["n"] == 6400
    assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-10


def test_direct_closed_form_coherent_state(ss):
    """The driven damped cavity's coherent steady state, alpha = -iE/(i Delta + kappa/2)."""
    s = driven_cavity(N=30, n_th=0.0)
    rho, info = ss.steady_state(s.H, s.c_ops, method="direct", tol=1e-10)
    delta, E, kappa = 0.5, 0.3, 1.0
    alpha = -1j * E / (1j * delta + kappa / 2)
    from math import factorial
    n = np.arange(30)
    psi = np.exp(-abs(alpha) ** 2 / 2) * alpha ** n / np.sqrt(np.array([float(factorial(int(k))) for k in n]))
    assert trace_distance(rho, np.outer(psi, psi.conj())) <= 1e-12


# ------------------------------------------------------------------ LGMRES

@pytest.mark.parametrize("m,k,cycles", [(10, 3, 3), (10, 3, 6), (6, 2, 8), (20, 0, 2)])
def test_lgmres_iterates_match_oracle_after_fixed_cycles(ss, m, k, cycles):
    """Unconverged iterates after a fixed number of LGMRES(m, k) cycles
    (tol = 0, maxiter = the Arnoldi steps of those cycles): the device's
    classical Gram-Schmidt and the oracle's modified Gram-Schmidt span the
    same spaces, so x agrees to rounding (the oracle's iterates move by
    ~1e-14 under perturbations of the inputs at rounding level)."""
    from oracle.krylov import lgmres
    s = jaynes_cummings_rwa(seed=1, N=8)
    L = liouvillian_sparse(s.H, s.c_ops)
    A, b = modified_liouvillian(L, s.d, default_weight(L))
    p = rcm_order(A)
    Aq = permute_symmetric(A, p)
    F = oilu.ilu0(Aq)
    ref = lgmres(lambda v: Aq @ v, lambda r: oilu.precond_apply_fast(F, r), b[p], None, 0.0, restart=m, augment=k,
                 maxiter=10**6, max_cycles=cycles)
    Ad, w = ss.add_trace_row(ss.assemble_liouvillian(s.H, s.c_ops))
    perm, _, _ = ss.rcm_permute(Ad)
    assert np.array_equal(perm, p)
    Ap = ss.permute(Ad, perm)
    M = ss.ilu_factor(Ap, "ilu0")
    bg = np.zeros(Ap.shape[0], dtype=complex)
    bg[np.flatnonzero(perm == 0)[0]] = w
    steps = sum(m + min(c, k) for c in range(cycles))
    x, st, it, res = ss.krylov_solve(Ap, M, _dev(bg), method="lgmres", restart=m, augment=k, tol=0.0, maxiter=steps)
    assert st == 3 and it == steps == ref.iters
    x = x.cpu().numpy()
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    assert np.linalg.norm(bg - Aq @ x) == pytest.approx(np.linalg.norm(b[p] - Aq @ ref.x), rel=1e-6)


def test_lgmres_solves_trace_row_system(ss):
    s = SMALL_SYSTEMS["kerr17"]()
    Ad, w = ss.add_trace_row(ss.assemble_liouvillian(s.H, s.c_ops))
    perm, _, _ = ss.rcm_permute(Ad)
    Ap = ss.permute(Ad, perm)
    M = ss.ilu_factor(Ap, "ilu0")
    b = np.zeros(Ap.shape[0], dtype=complex)
    b[np.flatnonzero(perm == 0)[0]] = w
    x, st, it, res = ss.krylov_solve(Ap, M, _dev(b), method="lgmres", restart=8, augment=3, tol=1e-13 * w)
    assert st == 0 and res <= 1e-13 * w
    L = liouvillian_sparse(s.H, s.c_ops)
    A, bo = modified_liouvillian(L, s.d, default_weight(L))
    xo = np.empty_like(b)
    xo[perm] = x.cpu().numpy()                       # back to natural order
    ref = np.linalg.solve(A.toarray(), bo)
    assert np.max(np.abs(xo - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_lgmres_rejects_bad_dimensions(ss):
    s = SMALL_SYSTEMS["cavity"]()
    with pytest.raises(ss.SolverError) as e:
        ss.steady_state(s.H, s.c_ops, method="iterative-lgmres", restart=60, lgmres_k=5)
    assert e.value.status == 1


@pytest.mark.parametrize("name", ["cavity_thermal", "jc8", "kerr17"])
def test_steady_state_lgmres_matches_dense(ss, name):
    s = SMALL_SYSTEMS[name]()
    rho, info = ss.steady_state(s.H, s.c_ops, method="iterative-lgmres", restart=10, lgmres_k=3, tol=1e-12)
    assert info["status"] == 0 and info["method_name"] == "iterative-lgmres"
    assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-10


def test_steady_state_config2_jc40_lgmres(ss):
    s = jaynes_cummings_rwa(seed=7)
    rho, info = ss.steady_state(s.H, s.c_ops, method="iterative-lgmres", precond="ilu0", restart=30, lgmres_k=3,
                                tol=1e-12)
    assert info["n"] == 6400 and info["status"] == 0
    assert trace_distance(rho, _dense_ref(7)) <= 1e-10


# ------------------------------------------------------ method selection

def test_auto_selection_on_the_papers_systems(ss):
    """The RCM bandwidths the rule compares are the ones printed in Fig. 1 and
    Fig. 3, and the choice is the oracle's (GMRES on L~ for the
    Jaynes-Cummings and optomechanical models, inverse power for the 5-spin
    chain).  Only the choice is checked here (maxiter 5)."""
    import json
    import os
    from oracle.krylov import select_method
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_rcm_bandwidth_profile.json")))
    B = {(c["system"], c["matrix"]): c["B"] for c in gold["cases"]}
    names = {"gmres": "iterative-lgmres", "power-gmres": "inverse-power"}
    for key, maker in (("jc", paper_jc_nonrwa), ("spin", paper_spin_chain), ("opto", paper_optomechanics)):
        s = maker()
        _, info = ss.steady_state(s.H, s.c_ops, method="auto", maxiter=5, raise_on_failure=False)
        assert (info["bw_modified"], info["bw_shifted"]) == (B[(key, "modified")], B[(key, "shifted")])
        assert info["method_name"] == names[select_method(s.H, s.c_ops)[0]], key


@pytest.mark.parametrize("maker,expect", [(lambda: paper_spin_chain(), "inverse-power"),
                                          (lambda: driven_cavity(n_th=0.2), "iterative-lgmres")],
                         ids=["spin5", "cavity"])
def test_auto_steady_state_matches_dense(ss, maker, expect):
    s = maker()
    rho, info = ss.steady_state(s.H, s.c_ops, method="auto", lgmres_k=3, tol=1e-10)
    assert info["status"] == 0 and info["method_name"] == expect and info["resid_Lrho"] <= 1e-10
    assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-8
