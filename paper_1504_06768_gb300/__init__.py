"""GB300 steady-state solver for open quantum systems (arXiv:1504.06768).

A thin Python layer over the C ABI of liblindblad_ss.so (include/lindblad_ss.h):
it converts SciPy sparse operators to CSR views and torch CUDA tensors to
device pointers, and nothing else.  The functions keep the C names:

    assemble_liouvillian, add_trace_row, add_shift, rcm_permute, permute,
    bandwidth_profile, ilu_factor, spmv, precond_apply, krylov_solve,
    steady_state

Device memory and streams come from PyTorch; all arithmetic runs in the CUDA
library.  Importing works without a GPU; calls need one.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np

from . import _binding as B

__all__ = ["SolverError", "Context", "Matrix", "Preconditioner", "get_context", "assemble_liouvillian",
           "add_trace_row", "add_shift", "rcm_permute", "permute", "bandwidth_profile", "ilu_factor",
           "spmv", "spmv_f32", "precond_apply", "precond_apply_f32", "krylov_solve", "steady_state",
           "steady_state_batched", "krylov_solve_noalloc", "NOALLOC_MAX_N", "library_path",
           "assemble_trace_batched", "Server"]

NOALLOC_MAX_N = 65536


def library_path() -> str:
    return B.LIB_PATH


class SolverError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{B.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Context:
    """Owns an ss_ctx bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        lib = B.load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.device = device
        self.stream = stream
        h = C.c_void_p()
        st = lib.ss_ctx_create(device, C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != 0:
            raise SolverError(st, "ss_ctx_create failed")
        self.handle = h

    def check(self, st: int, what: str):
        if st != 0:
            msg = B.load().ss_last_error(self.handle).decode()
            raise SolverError(st, f"{what}: {msg}")

    def synchronize(self):
        self.stream.synchronize()

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and B._lib is not None:
            B._lib.ss_ctx_destroy(h)
            self.handle = None


_contexts: dict = {}


def get_context(device: int = 0) -> Context:
    ctx = _contexts.get(device)
    if ctx is None:
        ctx = Context(device)
        _contexts[device] = ctx
    return ctx


class _CsrHost:
    """Keeps the numpy arrays of a CSR view alive for the duration of a call."""

    def __init__(self, m):
        import scipy.sparse as sp
        m = sp.csr_matrix(m, dtype=np.complex128)
        m.sum_duplicates()
        m.sort_indices()
        self.rp = np.ascontiguousarray(m.indptr, dtype=np.int32)
        self.col = np.ascontiguousarray(m.indices, dtype=np.int32)
        self.val = np.ascontiguousarray(m.data, dtype=np.complex128)
        self.view = B.CsrView(m.shape[0], m.shape[1], m.nnz, self.rp.ctypes.data, self.col.ctypes.data,
                              self.val.ctypes.data, 0)


def _host_status(st: int, what: str):
    if st != B.SS_OK:
        raise SolverError(st, f"{what}: {B.STATUS_NAMES.get(st, st)}")


def rcm_order_host(A):
    """Reverse Cuthill-McKee order of the pattern of A + A^T computed on the
    host (no GPU): perm[new] = old."""
    h = _CsrHost(A)
    n = h.view.n_rows
    perm = np.empty(n, dtype=np.int32)
    _host_status(B.load().ss_rcm_order_host(n, h.rp.ctypes.data, h.col.ctypes.data, perm.ctypes.data),
                 "ss_rcm_order_host")
    return perm


def mbm_host(A):
    """Weighted maximum bipartite matching on the host (no GPU): (match,
    matched) with match[j] = the row assigned to column j (-1 if none), so
    that A[match, :] has a zero-free diagonal when matched == n."""
    h = _CsrHost(A)
    n = h.view.n_rows
    match = np.empty(n, dtype=np.int32)
    matched = C.c_int64()
    _host_status(B.load().ss_mbm_host(n, h.rp.ctypes.data, h.col.ctypes.data, h.val.ctypes.data, match.ctypes.data,
                                      C.byref(matched)), "ss_mbm_host")
    return match, matched.value


def tune_search_host(cost_table, max_probes: int = 64):
    """The batched solver's autotuner search on a table of costs (no GPU):
    cost_table has shape (4, 4, 4, 2) over the lanes-per-row shifts -1..2 of
    the lower triangle, the upper triangle and L~, and the staging flag.
    Returns (best choice (lo, up, a, stage), number of evaluations)."""
    t = np.ascontiguousarray(np.asarray(cost_table, dtype=np.float64).reshape(4, 4, 4, 2))
    best = (C.c_int32 * 4)()
    probes = C.c_int32()
    _host_status(B.load().ss_tune_search_host(t.ctypes.data, max_probes, best, C.byref(probes)), "ss_tune_search_host")
    return tuple(best), probes.value


def level_sets_host(A, lower: bool = True):
    """Level sets of the strict lower (or upper) triangle of A's pattern on
    the host: (order, level_ptr)."""
    h = _CsrHost(A)
    n = h.view.n_rows
    order = np.empty(n, dtype=np.int32)
    ptr = np.empty(n + 1, dtype=np.int32)
    nl = C.c_int32()
    _host_status(B.load().ss_level_sets_host(n, h.rp.ctypes.data, h.col.ctypes.data, int(lower), order.ctypes.data,
                                             ptr.ctypes.data, C.byref(nl)), "ss_level_sets_host")
    return order, ptr[:nl.value + 1].copy()


def ilu0_schedule_host(A):
    """The iLU(0) elimination schedule of A's pattern on the host (no GPU):
    (ptr, tgt, src) over A's CSR with sorted columns, as
    ss_ilu0_schedule_host describes them."""
    h = _CsrHost(A)
    n = h.view.n_rows
    lib = B.load()
    cnt = C.c_int64(-1)
    ptr = np.empty(int(h.rp[-1]) + 1, dtype=np.int32)
    st = lib.ss_ilu0_schedule_host(n, h.rp.ctypes.data, h.col.ctypes.data, 0, ptr.ctypes.data, None, None,
                                   C.byref(cnt))
    if st == B.SS_ZERO_PIVOT:
        raise SolverError(st, "ss_ilu0_schedule_host: a diagonal entry is missing")
    if cnt.value < 0:
        _host_status(st, "ss_ilu0_schedule_host")
    tgt = np.empty(max(cnt.value, 1), dtype=np.int32)
    src = np.empty(max(cnt.value, 1), dtype=np.int32)
    _host_status(lib.ss_ilu0_schedule_host(n, h.rp.ctypes.data, h.col.ctypes.data, cnt.value, ptr.ctypes.data,
                                           tgt.ctypes.data, src.ctypes.data, C.byref(cnt)), "ss_ilu0_schedule_host")
    return ptr, tgt[:cnt.value].copy(), src[:cnt.value].copy()


def ilut_host(A, drop_tol: float = 1e-4, fill_factor: float = 10.0):
    """ILUT factors of A computed on the host (no GPU), as a scipy CSR matrix
    of the combined factors (strict lower = L with unit diagonal, rest = U)."""
    import scipy.sparse as sp
    h = _CsrHost(A)
    n = h.view.n_rows
    lib = B.load()
    nnz, bad = C.c_int64(), C.c_int64()
    st = lib.ss_ilut_host(n, h.rp.ctypes.data, h.col.ctypes.data, h.val.ctypes.data, drop_tol, fill_factor, 0,
                          None, None, None, C.byref(nnz), C.byref(bad))
    if st == B.SS_ZERO_PIVOT:
        raise SolverError(st, f"ss_ilut_host: zero pivot in row {bad.value}")
    rp = np.empty(n + 1, dtype=np.int32)
    col = np.empty(max(nnz.value, 1), dtype=np.int32)
    val = np.empty(max(nnz.value, 1), dtype=np.complex128)
    _host_status(lib.ss_ilut_host(n, h.rp.ctypes.data, h.col.ctypes.data, h.val.ctypes.data, drop_tol, fill_factor,
                                  nnz.value, rp.ctypes.data, col.ctypes.data, val.ctypes.data, C.byref(nnz),
                                  C.byref(bad)), "ss_ilut_host")
    return sp.csr_matrix((val[:nnz.value], col[:nnz.value], rp), shape=(n, n))


class Matrix:
    """A library-owned complex FP64 CSR matrix on the device."""

    def __init__(self, ctx: Context, handle: C.c_void_p):
        self.ctx = ctx
        self.handle = handle

    @property
    def shape(self):
        n, nnz = C.c_int64(), C.c_int64()
        B.load().ss_mat_shape(self.handle, C.byref(n), C.byref(nnz))
        return (n.value, n.value)

    @property
    def nnz(self) -> int:
        n, nnz = C.c_int64(), C.c_int64()
        B.load().ss_mat_shape(self.handle, C.byref(n), C.byref(nnz))
        return nnz.value

    def to_scipy(self):
        import scipy.sparse as sp
        n, nnz = self.shape[0], self.nnz
        rp = np.empty(n + 1, dtype=np.int32)
        col = np.empty(max(nnz, 1), dtype=np.int32)
        val = np.empty(max(nnz, 1), dtype=np.complex128)
        self.ctx.check(B.load().ss_mat_export(self.ctx.handle, self.handle, rp.ctypes.data, col.ctypes.data,
                                              val.ctypes.data), "ss_mat_export")
        return sp.csr_matrix((val[:nnz], col[:nnz], rp), shape=(n, n))

    @classmethod
    def from_scipy(cls, m, ctx: Optional[Context] = None) -> "Matrix":
        ctx = ctx or get_context()
        hv = _CsrHost(m)
        h = C.c_void_p()
        ctx.check(B.load().ss_mat_import(ctx.handle, C.byref(hv.view), C.byref(h)), "ss_mat_import")
        return cls(ctx, h)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and B._lib is not None:
            B._lib.ss_mat_free(h)
            self.handle = None


class Preconditioner:
    def __init__(self, ctx: Context, handle: C.c_void_p, condest: float):
        self.ctx = ctx
        self.handle = handle
        self.condest = condest

    def info(self) -> dict:
        nnz, lo, up = C.c_int64(), C.c_int32(), C.c_int32()
        B.load().ss_prec_info(self.handle, C.byref(nnz), C.byref(lo), C.byref(up))
        return {"nnz": nnz.value, "levels_lower": lo.value, "levels_upper": up.value}

    def to_scipy(self, n: int):
        import scipy.sparse as sp
        nnz = self.info()["nnz"]
        rp = np.empty(n + 1, dtype=np.int32)
        col = np.empty(max(nnz, 1), dtype=np.int32)
        val = np.empty(max(nnz, 1), dtype=np.complex128)
        self.ctx.check(B.load().ss_prec_export(self.ctx.handle, self.handle, rp.ctypes.data, col.ctypes.data,
                                               val.ctypes.data), "ss_prec_export")
        return sp.csr_matrix((val[:nnz], col[:nnz], rp), shape=(n, n))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and B._lib is not None:
            B._lib.ss_prec_free(h)
            self.handle = None


def _dev_ptr(t, dtype_name: str, n: int):
    import torch
    want = {"c128": torch.complex128, "c64": torch.complex64}[dtype_name]
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == want and t.is_contiguous()
            and t.numel() == n):
        raise ValueError(f"expected a contiguous CUDA {want} tensor of {n} elements")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------- API

def assemble_liouvillian(H, c_ops: Sequence, ctx: Optional[Context] = None) -> Matrix:
    """L of Eq. (lindblad), column-stacked (Eq. eigval), assembled on the GPU."""
    ctx = ctx or get_context()
    hv = _CsrHost(H)
    cvs = [_CsrHost(c) for c in c_ops]
    arr = (B.CsrView * max(len(cvs), 1))(*[c.view for c in cvs])
    h = C.c_void_p()
    ctx.check(B.load().assemble_liouvillian(ctx.handle, C.byref(hv.view), len(cvs), arr, C.byref(h)),
              "assemble_liouvillian")
    return Matrix(ctx, h)


def add_trace_row(L: Matrix, w: float = 0.0):
    """Eq. (linear): returns (L + w T, w_used); w <= 0 selects mean |L_ii|."""
    h, wu = C.c_void_p(), C.c_double()
    L.ctx.check(B.load().add_trace_row(L.ctx.handle, L.handle, w, C.byref(h), C.byref(wu)), "add_trace_row")
    return Matrix(L.ctx, h), wu.value


def assemble_trace_batched(systems: Sequence, w: float = 0.0, ctx: Optional[Context] = None):
    """Eq. (lindblad) and Eq. (linear) for many systems (H, c_ops) in one call:
    returns a list of (L + w_k T, w_k).  CSR views may be scipy matrices (host)
    or (row_ptr, col, val, n) tuples of device tensors."""
    ctx = ctx or get_context()
    views, keep = [], []
    for H, cs in systems:
        hv = _view(H, keep)
        views.append((hv, [_view(c, keep) for c in cs]))
    ns = len(views)
    Hs = (B.CsrView * max(ns, 1))(*[h for h, _ in views])
    ncs = (C.c_int * max(ns, 1))(*[len(cs) for _, cs in views])
    carrs = [(B.CsrView * max(len(cs), 1))(*cs) for _, cs in views]
    cptrs = (C.POINTER(B.CsrView) * max(ns, 1))(*[C.cast(a, C.POINTER(B.CsrView)) for a in carrs])
    outs = (C.c_void_p * max(ns, 1))()
    wu = (C.c_double * max(ns, 1))()
    ctx.check(B.load().assemble_trace_batched(ctx.handle, ns, Hs, ncs, cptrs, w, outs, wu), "assemble_trace_batched")
    return [(Matrix(ctx, C.c_void_p(outs[k])), wu[k]) for k in range(ns)]


def _view(m, keep):
    """CSR view of a scipy matrix (host) or of a (row_ptr, col, val, n_cols)
    tuple of device tensors (int32, int32, complex128)."""
    if isinstance(m, tuple):
        rp, col, val, n_cols = m
        keep.append(m)
        return B.CsrView(rp.numel() - 1, n_cols, val.numel(), rp.data_ptr(), col.data_ptr(), val.data_ptr(), 1)
    h = _CsrHost(m)
    keep.append(h)
    return h.view


def add_shift(L: Matrix, sigma: float = 1e-15) -> Matrix:
    """Eq. (inverse): L - sigma I."""
    h = C.c_void_p()
    L.ctx.check(B.load().add_shift(L.ctx.handle, L.handle, sigma, C.byref(h)), "add_shift")
    return Matrix(L.ctx, h)


def rcm_permute(A: Matrix):
    """Reverse Cuthill-McKee of A + A^T: (perm with perm[new] = old, B, P)."""
    n = A.shape[0]
    perm = np.empty(n, dtype=np.int32)
    bw, prof = C.c_int64(), C.c_int64()
    A.ctx.check(B.load().rcm_permute(A.ctx.handle, A.handle, perm.ctypes.data, C.byref(bw), C.byref(prof)),
                "rcm_permute")
    return perm, bw.value, prof.value


def permute(A: Matrix, perm) -> Matrix:
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    h = C.c_void_p()
    A.ctx.check(B.load().permute(A.ctx.handle, A.handle, perm.ctypes.data, C.byref(h)), "permute")
    return Matrix(A.ctx, h)


def bandwidth_profile(A: Matrix):
    bw, prof = C.c_int64(), C.c_int64()
    A.ctx.check(B.load().bandwidth_profile(A.ctx.handle, A.handle, C.byref(bw), C.byref(prof)),
                "bandwidth_profile")
    return bw.value, prof.value


def ilu_factor(A: Matrix, kind: str = "ilu0", drop_tol: float = 1e-4, fill_factor: float = 10.0,
               precision: str = "fp64") -> Preconditioner:
    h, ce = C.c_void_p(), C.c_double()
    A.ctx.check(B.load().ilu_factor(A.ctx.handle, A.handle, B.PRECONDS[kind], drop_tol, fill_factor,
                                    B.PRECISIONS[precision], C.byref(h), C.byref(ce)), "ilu_factor")
    return Preconditioner(A.ctx, h, ce.value)


def spmv(A: Matrix, x):
    import torch
    n = A.shape[0]
    y = torch.empty(n, dtype=torch.complex128, device=x.device)
    A.ctx.check(B.load().spmv(A.ctx.handle, A.handle, _dev_ptr(x, "c128", n), _dev_ptr(y, "c128", n)), "spmv")
    return y


def spmv_f32(A: Matrix, x):
    import torch
    n = A.shape[0]
    y = torch.empty(n, dtype=torch.complex64, device=x.device)
    A.ctx.check(B.load().spmv_f32(A.ctx.handle, A.handle, _dev_ptr(x, "c64", n), _dev_ptr(y, "c64", n)),
                "spmv_f32")
    return y


def precond_apply(M: Preconditioner, r):
    import torch
    n = r.numel()
    z = torch.empty_like(r)
    M.ctx.check(B.load().precond_apply(M.ctx.handle, M.handle, _dev_ptr(r, "c128", n), _dev_ptr(z, "c128", n)),
                "precond_apply")
    return z


def precond_apply_f32(M: Preconditioner, r):
    import torch
    n = r.numel()
    z = torch.empty_like(r)
    M.ctx.check(B.load().precond_apply_f32(M.ctx.handle, M.handle, _dev_ptr(r, "c64", n),
                                           _dev_ptr(z, "c64", n)), "precond_apply_f32")
    return z


def krylov_solve(A: Matrix, M: Preconditioner, b, x0=None, method: str = "bicgstab", tol: float = 1e-12,
                 maxiter: int = 1000, restart: int = 30, raise_on_failure: bool = False, augment: int = 0):
    """Right-preconditioned BiCGSTAB / GMRES(m) on A x = b; method "lgmres"
    runs LGMRES(restart, augment).  Returns (x, status, iters, resid)."""
    import torch
    n = A.shape[0]
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    it, res = C.c_int(), C.c_double()
    if method == "lgmres":
        st = B.load().lgmres_solve(A.ctx.handle, A.handle, M.handle, _dev_ptr(b, "c128", n), _dev_ptr(x, "c128", n),
                                   tol, maxiter, restart, augment, C.byref(it), C.byref(res))
    else:
        st = B.load().krylov_solve(A.ctx.handle, A.handle, M.handle, B.KRYLOV[method], _dev_ptr(b, "c128", n),
                                   _dev_ptr(x, "c128", n), tol, maxiter, restart, C.byref(it), C.byref(res))
    if st not in (B.SS_OK, B.SS_NOT_CONVERGED, B.SS_BREAKDOWN) or (raise_on_failure and st != 0):
        A.ctx.check(st, "krylov_solve")
    return x, st, it.value, res.value


def _options(method, tol, precond, precision, maxiter, restart, drop_tol, fill_factor, w, sigma, use_rcm, seed,
             inner_rtol=1e-5, lgmres_k=0, warm_start=0, autotune=0):
    opt = B.Options()
    B.load().ss_options_default(C.byref(opt))
    opt.method = B.METHODS[method]
    opt.precond = B.PRECONDS[precond]
    opt.precision = B.PRECISIONS[precision]
    opt.tol, opt.maxiter, opt.restart = tol, maxiter, restart
    opt.drop_tol, opt.fill_factor, opt.w, opt.sigma = drop_tol, fill_factor, w, sigma
    opt.use_rcm, opt.seed = int(bool(use_rcm)), seed
    opt.inner_rtol = inner_rtol
    opt.lgmres_k = lgmres_k
    opt.warm_start = int(bool(warm_start))
    opt.autotune = int(bool(autotune))
    return opt


def steady_state_batched(systems: Sequence, method: str = "iterative-bicgstab", tol: float = 1e-10,
                         precond: str = "ilu0", precision: str = "fp64", maxiter: int = 1000, restart: int = 30,
                         drop_tol: float = 1e-4, fill_factor: float = 10.0, w: float = 0.0, sigma: float = 1e-15,
                         use_rcm: bool = True, seed: int = 0, ctx: Optional[Context] = None,
                         raise_on_failure: bool = True, inner_rtol: float = 1e-5, lgmres_k: int = 0,
                         rho_init: Optional[Sequence] = None, autotune: bool = False):
    """Steady states of many systems, each given as (H, c_ops); returns a list
    of rho (numpy, d x d) and a list of info dicts.  rho_init: optional
    initial guesses (one d x d matrix per system, e.g. the steady states of
    neighbouring sweep points): the solves start from them (warm start)."""
    ctx = ctx or get_context()
    hosts = [(_CsrHost(H), [_CsrHost(c) for c in cs]) for H, cs in systems]
    ns = len(hosts)
    Hs = (B.CsrView * max(ns, 1))(*[h.view for h, _ in hosts])
    ncs = (C.c_int * max(ns, 1))(*[len(cs) for _, cs in hosts])
    carrs = [(B.CsrView * max(len(cs), 1))(*[c.view for c in cs]) for _, cs in hosts]
    cptrs = (C.POINTER(B.CsrView) * max(ns, 1))(*[C.cast(a, C.POINTER(B.CsrView)) for a in carrs])
    rhos = [np.empty(h.view.n_rows ** 2, dtype=np.complex128) for h, _ in hosts]
    if rho_init is not None:
        for r, r0 in zip(rhos, rho_init):
            r[:] = np.asarray(r0, dtype=np.complex128).reshape(-1, order="F")
    outs = (C.c_void_p * max(ns, 1))(*[r.ctypes.data for r in rhos])
    infos = (B.Info * max(ns, 1))()
    opt = _options(method, tol, precond, precision, maxiter, restart, drop_tol, fill_factor, w, sigma, use_rcm, seed,
                   inner_rtol, lgmres_k, rho_init is not None, autotune)
    st = B.load().steady_state_batched(ctx.handle, ns, Hs, ncs, cptrs, C.byref(opt), outs, 0, infos)
    if st != 0 and (raise_on_failure or st not in (B.SS_NOT_CONVERGED, B.SS_BREAKDOWN)):
        ctx.check(st, "steady_state_batched")
    d = [h.view.n_rows for h, _ in hosts]
    return [r.reshape((dk, dk), order="F") for r, dk in zip(rhos, d)], [infos[k].as_dict() for k in range(ns)]


def krylov_solve_noalloc(A: Matrix, M: Preconditioner, b, x, tol: float = 1e-12, maxiter: int = 1000):
    """BiCGSTAB on A x = b in place on the caller's x, without any allocation
    inside the call (for callers that cannot allocate; n <= NOALLOC_MAX_N).
    Returns (status, iters, resid); x holds the initial guess on entry."""
    n = A.shape[0]
    it, res = C.c_int(), C.c_double()
    st = B.load().krylov_solve_noalloc(A.ctx.handle, A.handle, M.handle, _dev_ptr(b, "c128", n),
                                       _dev_ptr(x, "c128", n), tol, maxiter, C.byref(it), C.byref(res))
    if st not in (B.SS_OK, B.SS_NOT_CONVERGED, B.SS_BREAKDOWN):
        A.ctx.check(st, "krylov_solve_noalloc")
    return st, it.value, res.value


def steady_state(H, c_ops: Sequence, method: str = "iterative-bicgstab", tol: float = 1e-10,
                 precond: str = "ilu0", precision: str = "fp64", maxiter: int = 1000, restart: int = 30,
                 drop_tol: float = 1e-4, fill_factor: float = 10.0, w: float = 0.0, sigma: float = 1e-15,
                 use_rcm: bool = True, seed: int = 0, ctx: Optional[Context] = None, out=None,
                 raise_on_failure: bool = True, inner_rtol: float = 1e-5, lgmres_k: int = 0, rho_init=None):
    """rho_ss (d x d complex128, trace one) and the solve's info dict.
    rho_init: optional initial guess (d x d), e.g. a neighbouring sweep
    point's steady state (warm start).

    out: optional CUDA complex128 tensor of d*d elements (column-major rho);
    when given, rho is written there and returned as a (d, d) view (transposed
    storage); otherwise a numpy array is returned.
    """
    ctx = ctx or get_context()
    hv = _CsrHost(H)
    cvs = [_CsrHost(c) for c in c_ops]
    arr = (B.CsrView * max(len(cvs), 1))(*[c.view for c in cvs])
    opt = _options(method, tol, precond, precision, maxiter, restart, drop_tol, fill_factor, w, sigma, use_rcm, seed,
                   inner_rtol, lgmres_k, rho_init is not None)
    d = hv.view.n_rows
    info = B.Info()
    if out is None:
        rho = np.empty(d * d, dtype=np.complex128)
        if rho_init is not None:
            rho[:] = np.asarray(rho_init, dtype=np.complex128).reshape(-1, order="F")
        ptr, on_dev = rho.ctypes.data, 0
    else:
        ptr, on_dev = _dev_ptr(out, "c128", d * d), 1
        if rho_init is not None:
            import torch
            out.copy_(torch.as_tensor(np.asarray(rho_init, dtype=np.complex128).reshape(-1, order="F")))
    st = B.load().steady_state(ctx.handle, C.byref(hv.view), len(cvs), arr, C.byref(opt), ptr, on_dev,
                               C.byref(info))
    if st != 0 and (raise_on_failure or st not in (B.SS_NOT_CONVERGED, B.SS_BREAKDOWN)):
        ctx.check(st, "steady_state")
    result = rho.reshape((d, d), order="F") if out is None else out.view(d, d).T
    return result, info.as_dict()


class Server:
    """Serving loop (ss_server_*): submit steady-state requests at any time,
    wait for them by ticket.  Inputs are copied at submission; each result is
    written to a host buffer that this object keeps until the request is
    waited for."""

    def __init__(self, method: str = "iterative-bicgstab", tol: float = 1e-10, precond: str = "ilu0",
                 precision: str = "mixed", maxiter: int = 1000, restart: int = 30, drop_tol: float = 1e-4,
                 fill_factor: float = 10.0, w: float = 0.0, sigma: float = 1e-15, use_rcm: bool = True,
                 seed: int = 0, inner_rtol: float = 1e-5, hbm_budget_mb: float = 0.0, max_waves: int = 4,
                 max_wave_systems: int = 0, device: int = 0, lgmres_k: int = 0, warm_start: bool = False):
        lib = B.load()
        opt = _options(method, tol, precond, precision, maxiter, restart, drop_tol, fill_factor, w, sigma, use_rcm,
                       seed, inner_rtol, lgmres_k)
        so = B.ServerOptions()
        lib.ss_server_options_default(C.byref(so))
        so.hbm_budget_mb = hbm_budget_mb
        so.max_waves = max_waves
        so.max_wave_systems = max_wave_systems
        so.warm_start = int(bool(warm_start))
        h = C.c_void_p()
        st = lib.ss_server_create(device, C.byref(opt), C.byref(so), C.byref(h))
        if st != 0:
            raise SolverError(st, "ss_server_create failed")
        self.handle = h
        self._out = {}

    def _check(self, st, what):
        if st != 0:
            raise SolverError(st, f"{what}: {B.load().ss_server_last_error(self.handle).decode()}")

    def submit(self, H, c_ops) -> int:
        hv = _CsrHost(H)
        cvs = [_CsrHost(c) for c in c_ops]
        arr = (B.CsrView * max(len(cvs), 1))(*[c.view for c in cvs])
        d = hv.view.n_rows
        rho = np.empty(d * d, dtype=np.complex128)
        t = C.c_uint64()
        self._check(B.load().ss_submit(self.handle, C.byref(hv.view), len(cvs), arr, rho.ctypes.data, C.byref(t)),
                    "ss_submit")
        self._out[t.value] = (rho, d)
        return t.value

    def poll(self, ticket: int) -> bool:
        done = C.c_int()
        self._check(B.load().ss_poll(self.handle, ticket, C.byref(done)), "ss_poll")
        return bool(done.value)

    def wait(self, ticket: int, timeout_s: Optional[float] = None, raise_on_failure: bool = True):
        """Returns (rho (d x d), info dict, latency in ms)."""
        info = B.Info()
        lat = C.c_double()
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        st = B.load().ss_wait(self.handle, ticket, us, C.byref(info), C.byref(lat))
        if st == B.SS_ERR_TIMEOUT and not self.poll(ticket):
            raise TimeoutError(f"request {ticket} still pending")
        rho, d = self._out.pop(ticket)
        if st != 0 and (raise_on_failure or st not in (B.SS_NOT_CONVERGED, B.SS_BREAKDOWN)):
            self._check(st, "ss_wait")
        return rho.reshape((d, d), order="F"), info.as_dict(), lat.value

    def stats(self):
        waves, done = C.c_uint64(), C.c_uint64()
        used, budget = C.c_double(), C.c_double()
        self._check(B.load().ss_server_stats(self.handle, C.byref(waves), C.byref(done), C.byref(used),
                                             C.byref(budget)), "ss_server_stats")
        return {"waves": waves.value, "completed": done.value, "in_use_mb": used.value, "budget_mb": budget.value}

    def close(self):
        if self.handle is not None:
            B.load().ss_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        if getattr(self, "handle", None) is not None and B._lib is not None:
            B._lib.ss_server_destroy(self.handle)
            self.handle = None
