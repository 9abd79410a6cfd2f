"""GPU parity of the per-system persistent solver (steady_state_batched):
against the CPU oracle, against the single-system path, and alone versus in
a mixed batch."""
import numpy as np
import pytest

from oracle.metrics import trace_distance
from oracle.steady import steady_state_dense
from workloads import driven_cavity, jaynes_cummings_rwa, kerr_sweep, thermal_cavity, two_level_atom

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


def _mix():
    systems = [driven_cavity(n_th=0.0), driven_cavity(n_th=0.2), thermal_cavity(n_th=0.2), two_level_atom()]
    systems += kerr_sweep(6, seed=3)
    systems += [jaynes_cummings_rwa(seed=s, N=12) for s in range(3)]      # shared pattern
    return systems


@pytest.mark.parametrize("precision,tol,td", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-8)])
def test_batched_matches_oracle(ss, precision, tol, td):
    systems = _mix()
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=tol, precision=precision)
    for s, rho, info in zip(systems, rhos, infos):
        assert info["status"] == 0, (s.name, info)
        assert info["resid_Lrho"] <= tol
        assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= td, s.name
        assert abs(np.trace(rho) - 1) < 1e-12


def test_batched_alone_equals_in_mix(ss):
    """Each system's result is the same alone and inside a mixed batch."""
    systems = _mix()
    rhos, _ = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-10, precision="mixed")
    for k in (0, 5, len(systems) - 1):
        alone, _ = ss.steady_state_batched([(systems[k].H, systems[k].c_ops)], tol=1e-10, precision="mixed")
        assert np.array_equal(alone[0], rhos[k])


def test_batched_agrees_with_single_system_path(ss):
    systems = [jaynes_cummings_rwa(seed=s, N=16) for s in range(4)]
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-12)
    for s, rho in zip(systems, rhos):
        single, _ = ss.steady_state(s.H, s.c_ops, tol=1e-12)
        assert trace_distance(rho, single) <= 1e-10


def test_batched_jc40_full_size(ss):
    systems = [jaynes_cummings_rwa(seed=s) for s in (0, 5)]
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-12)
    for s, rho, info in zip(systems, rhos, infos):
        assert info["n"] == 6400 and info["status"] == 0
        assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-10


def test_batched_kerr_sweep_uneven(ss):
    """The uneven Kerr sweep (cutoffs 8..64, n = 64..4096), mixed precision,
    against FP64 single-system solves on a sample."""
    systems = kerr_sweep(48, seed=0)
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-10, precision="mixed")
    assert all(i["status"] == 0 and i["resid_Lrho"] <= 1e-10 for i in infos)
    for k in range(0, 48, 8):
        ref = steady_state_dense(systems[k].H, systems[k].c_ops)
        assert trace_distance(rhos[k], ref) <= 1e-8


def test_batched_falls_back_for_other_methods(ss):
    systems = [driven_cavity(n_th=0.2), thermal_cavity()]
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], method="iterative-lgmres",
                                          tol=1e-12)
    for s, rho, info in zip(systems, rhos, infos):
        assert info["status"] == 0
        assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-10


def _device_view(m):
    import scipy.sparse as sp
    import torch
    m = sp.csr_matrix(m)
    m.sort_indices()
    return (torch.as_tensor(m.indptr.astype(np.int32), device="cuda"),
            torch.as_tensor(m.indices.astype(np.int32), device="cuda"),
            torch.as_tensor(m.data.astype(np.complex128), device="cuda"), m.shape[1])


def test_assemble_trace_batched_equals_single_calls(ss):
    """The batched assembly (block-diagonal operator stacks, one launch per
    stage) gives, entry for entry, the matrix of assemble_liouvillian +
    add_trace_row for every system, with host and device views, uneven sizes
    and different numbers of collapse operators."""
    systems = _mix() + [driven_cavity(N=5, n_th=0.0)]
    batch = []
    for k, s in enumerate(systems):
        if k % 2:
            batch.append((_device_view(s.H), [_device_view(c) for c in s.c_ops]))
        else:
            batch.append((s.H, s.c_ops))
    out = ss.assemble_trace_batched(batch)
    for s, (Lt, w) in zip(systems, out):
        ref, w_ref = ss.add_trace_row(ss.assemble_liouvillian(s.H, s.c_ops))
        assert w == w_ref, s.name
        a, b = Lt.to_scipy(), ref.to_scipy()
        assert a.shape == b.shape and a.nnz == b.nnz, s.name
        assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices), s.name
        assert np.array_equal(a.data, b.data), s.name
    # a given weight is used as it is
    out2 = ss.assemble_trace_batched([(systems[0].H, systems[0].c_ops)], w=2.5)
    ref2, _ = ss.add_trace_row(ss.assemble_liouvillian(systems[0].H, systems[0].c_ops), 2.5)
    assert out2[0][1] == 2.5
    assert np.array_equal(out2[0][0].to_scipy().toarray(), ref2.to_scipy().toarray())


def test_batched_device_and_host_views_agree(ss):
    """steady_state_batched through device views gives the same rho as through
    host views (the bench's two legs)."""
    import ctypes as C
    import torch
    from paper_1504_06768_gb300 import _binding as B
    systems = [jaynes_cummings_rwa(seed=s, N=10) for s in range(3)] + [driven_cavity(n_th=0.2)]
    host, _ = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-10, precision="mixed")
    ctx = ss.get_context()
    keep = []
    Hs = (B.CsrView * len(systems))(*[ss._view(_device_view(s.H), keep) for s in systems])
    carrs = [(B.CsrView * len(s.c_ops))(*[ss._view(_device_view(c), keep) for c in s.c_ops]) for s in systems]
    cptrs = (C.POINTER(B.CsrView) * len(systems))(*[C.cast(a, C.POINTER(B.CsrView)) for a in carrs])
    ncs = (C.c_int * len(systems))(*[len(s.c_ops) for s in systems])
    rho = [torch.empty(s.d * s.d, dtype=torch.complex128, device="cuda") for s in systems]
    outs = (C.c_void_p * len(systems))(*[r.data_ptr() for r in rho])
    infos = (B.Info * len(systems))()
    opt = ss._options("iterative-bicgstab", 1e-10, "ilu0", "mixed", 1000, 30, 1e-4, 10.0, 0.0, 1e-15, True, 0, 1e-5)
    st = B.load().steady_state_batched(ctx.handle, len(systems), Hs, ncs, cptrs, C.byref(opt), outs, 1, infos)
    torch.cuda.synchronize()
    assert st == 0, B.load().ss_last_error(ctx.handle).decode()
    for s, r, h in zip(systems, rho, host):
        assert np.array_equal(r.cpu().numpy().reshape((s.d, s.d), order="F"), h)


def test_batched_autotune_same_states_and_cached_choice(ss):
    """The autotuner times capped probe launches of candidate lanes-per-row
    and staging choices and keeps the fastest; the states are the rule
    choice's to the solve tolerance, the choice is reported per system and
    kept for a second batch of the same shape."""
    systems = [jaynes_cummings_rwa(seed=s, N=16) for s in range(24)]
    pairs = [(s.H, s.c_ops) for s in systems]
    for precision, td in (("mixed", 1e-8), ("fp64", 1e-10)):
        ref, _ = ss.steady_state_batched(pairs, tol=1e-11, precision=precision)
        tuned, ti = ss.steady_state_batched(pairs, tol=1e-11, precision=precision, autotune=True)
        again, ai = ss.steady_state_batched(pairs, tol=1e-11, precision=precision, autotune=True)
        for a, b, c, i in zip(ref, tuned, again, ti):
            assert i["status"] == 0 and i["resid_Lrho"] <= 1e-11
            assert trace_distance(a, b) <= td and np.array_equal(b, c)
        assert all(-1 <= v <= 2 for v in ti[0]["tune_lanes_shift"]) and ti[0]["tune_stage"] in (0, 1)
        assert ti[0]["tune_lanes_shift"] == ai[0]["tune_lanes_shift"] and ti[0]["tune_stage"] == ai[0]["tune_stage"]
        assert trace_distance(tuned[3], steady_state_dense(systems[3].H, systems[3].c_ops)) <= td
