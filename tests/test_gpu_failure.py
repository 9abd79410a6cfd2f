"""Failure detection without a GPU fault: a bounded device-side wait is made
to run out on purpose, and the call reports SS_ERR_TIMEOUT while the device
and the preconditioner stay usable.

The sync-free triangular solve waits for the rows it depends on.  Here the
lower solve is told to skip one row (ss_diag_prec_skip_row: its value is
never written, like a flag nothing sets), the wait limit is cut to 1 ms
(ss_set_wait_limit), and the rows that depend on the skipped one give up.
Every wait is bounded, so the launch ends by itself."""
import ctypes
import time

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ilu as oilu
from workloads import jaynes_cummings_rwa

pytestmark = pytest.mark.gpu

SS_ERR_TIMEOUT = 6


@pytest.fixture(scope="module")
def ss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    import paper_1504_06768_gb300 as lib
    return lib


def _system(ss):
    s = jaynes_cummings_rwa(seed=2, N=10)
    A, w = ss.add_trace_row(ss.assemble_liouvillian(s.H, s.c_ops))
    perm, _, _ = ss.rcm_permute(A)
    Ap = ss.permute(A, perm)
    M = ss.ilu_factor(Ap, "ilu0", precision="mixed")
    return Ap, M, w


def _busiest_row(F):
    """The row most other rows of the strict lower factor depend on."""
    low = sp.tril(F, k=-1).tocsr()
    return int(np.argmax(np.bincount(low.indices, minlength=F.shape[0])))


def test_triangular_solve_wait_runs_out_and_recovers(ss):
    import torch
    from paper_1504_06768_gb300 import _binding as B
    lib = B.load()
    Ap, M, _ = _system(ss)
    n = Ap.shape[0]
    F = M.to_scipy(n)
    row = _busiest_row(F)
    ctx = M.ctx.handle
    r = torch.as_tensor(np.random.default_rng(3).standard_normal(n) + 0j, device="cuda")
    z = torch.empty_like(r)
    r32, z32 = r.to(torch.complex64), torch.empty(n, dtype=torch.complex64, device="cuda")
    assert lib.ss_set_wait_limit(ctx, 1_000_000) == 0             # 1 ms
    assert lib.ss_diag_prec_skip_row(ctx, M.handle, row, 0) == 0
    try:
        for fn, a, b in ((lib.precond_apply, r, z), (lib.precond_apply_f32, r32, z32)):
            t0 = time.perf_counter()
            st = fn(ctx, M.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()))
            torch.cuda.synchronize()
            assert st == SS_ERR_TIMEOUT, (st, lib.ss_last_error(ctx).decode())
            assert time.perf_counter() - t0 < 5.0
        # a Krylov solve on the same factors reports the timeout as well
        bvec = torch.zeros(n, dtype=torch.complex128, device="cuda")
        bvec[0] = 1.0
        x = torch.zeros_like(bvec)
        it, res = ctypes.c_int(), ctypes.c_double()
        st = lib.krylov_solve(ctx, Ap.handle, M.handle, 0, ctypes.c_void_p(bvec.data_ptr()),
                              ctypes.c_void_p(x.data_ptr()), 1e-12, 50, 30, ctypes.byref(it), ctypes.byref(res))
        assert st == SS_ERR_TIMEOUT
    finally:
        assert lib.ss_diag_prec_skip_row(ctx, M.handle, row, 1) == 0
        assert lib.ss_set_wait_limit(ctx, 2_000_000_000) == 0
    # the same context and factors work again, with the oracle's result
    zz = ss.precond_apply(M, r).cpu().numpy()
    ref = oilu.upper_solve(F, oilu.lower_solve(F, r.cpu().numpy()))
    assert np.max(np.abs(zz - ref)) <= 1e-12 * np.max(np.abs(ref))
    again = ss.precond_apply(M, r).cpu().numpy()
    assert np.array_equal(zz, again)


def test_wait_limit_rejects_zero(ss):
    from paper_1504_06768_gb300 import _binding as B
    ctx = ss.get_context()
    assert B.load().ss_set_wait_limit(ctx.handle, 0) == 1


def test_batched_staging_wait_runs_out_and_recovers(ss):
    """The FP64 batched solver stages the levels of its triangular solves in
    a shared-memory ring filled by bulk copies, each slot guarded by an
    mbarrier whose wait is bounded.  ss_diag_batched_stall(5) makes every
    block's sixth staging arm its barrier without issuing the copies (a
    transfer that never arrives); with a 1 ms limit the waits give up, the
    blocks stop staging, drain what they issued, and the call reports
    SS_ERR_TIMEOUT.  The same context then solves correctly."""
    from paper_1504_06768_gb300 import _binding as B
    from oracle.metrics import trace_distance
    from oracle.steady import steady_state_dense
    lib = B.load()
    systems = [jaynes_cummings_rwa(seed=s, N=12) for s in range(4)]
    pairs = [(s.H, s.c_ops) for s in systems]
    ctx = ss.get_context()
    assert lib.ss_diag_batched_stall(ctx.handle, -2) == 1
    assert lib.ss_set_wait_limit(ctx.handle, 1_000_000) == 0
    assert lib.ss_diag_batched_stall(ctx.handle, 5) == 0
    try:
        t0 = time.perf_counter()
        with pytest.raises(ss.SolverError) as e:
            ss.steady_state_batched(pairs, tol=1e-10, precision="fp64", ctx=ctx)
        assert e.value.status == SS_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 20.0
    finally:
        assert lib.ss_diag_batched_stall(ctx.handle, -1) == 0
        assert lib.ss_set_wait_limit(ctx.handle, 2_000_000_000) == 0
    rhos, infos = ss.steady_state_batched(pairs, tol=1e-10, precision="fp64", ctx=ctx)
    for s, rho, info in zip(systems, rhos, infos):
        assert info["status"] == 0
        assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-9
