"""The allocation-free BiCGSTAB entry point, for callers that cannot allocate
device memory during a call (a fixed memory budget, or a host that owns every
allocation through its own pool).  It must give the same answer as the
ordinary krylov_solve, call after call, although its workspace is one shared
fixed array that each call overwrites.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

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


def _system(ss, seed, N):
    from workloads import jaynes_cummings_rwa
    s = jaynes_cummings_rwa(seed=seed, N=N)
    A, w = ss.add_trace_row(ss.assemble_liouvillian(s.H, s.c_ops))
    perm, _, _ = ss.rcm_permute(A)
    Ap = ss.permute(A, perm)
    M = ss.ilu_factor(Ap, "ilu0")
    n = Ap.shape[0]
    b = np.zeros(n, dtype=complex)
    b[np.flatnonzero(perm == 0)[0]] = w
    return Ap, M, b, w


def test_noalloc_matches_krylov_solve_twice(ss):
    import torch
    from paper_1504_06768_gb300 import _binding as B
    lib = B.load()
    for seed, N in ((0, 16), (3, 40)):               # n = 1,024 and the full 6,400
        Ap, M, b, w = _system(ss, seed, N)
        n = Ap.shape[0]
        bd = torch.as_tensor(b, device="cuda")
        ref, st, it_ref, res_ref = ss.krylov_solve(Ap, M, bd, method="bicgstab", tol=1e-12 * w)
        assert st == 0
        for call in range(2):                        # the second call reuses the dirty shared array
            x = torch.zeros(n, dtype=torch.complex128, device="cuda")
            it, res = ctypes.c_int(), ctypes.c_double()
            torch.cuda.synchronize()
            allocs0, free0 = lib.ss_alloc_count(), torch.cuda.mem_get_info()[0]
            st = lib.krylov_solve_noalloc(Ap.ctx.handle, Ap.handle, M.handle, ctypes.c_void_p(bd.data_ptr()),
                                          ctypes.c_void_p(x.data_ptr()), 1e-12 * w, 1000, ctypes.byref(it),
                                          ctypes.byref(res))
            torch.cuda.synchronize()
            assert st == 0, lib.ss_last_error(Ap.ctx.handle).decode()
            # nothing was allocated: not by the library (its allocation counter),
            # and no new device memory was taken by anyone in the call
            assert lib.ss_alloc_count() == allocs0, call
            assert torch.cuda.mem_get_info()[0] == free0, call
            assert res.value <= 1e-12 * w and it.value == it_ref
            err = (x - ref).abs().max().item()
            assert err <= 1e-10 * ref.abs().max().item(), (call, err)


def test_noalloc_rejects_oversized_system(ss):
    import torch
    n = ss.NOALLOC_MAX_N + 1
    A = ss.Matrix.from_scipy(sp.identity(n, dtype=complex, format="csr"))
    M = ss.ilu_factor(A, "ilu0")
    b = torch.ones(n, dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(ss.SolverError) as e:
        ss.krylov_solve_noalloc(A, M, b, x)
    assert e.value.status == 1 and "no-allocation limit" in e.value.message
