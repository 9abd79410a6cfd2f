"""Preconditioned Krylov solvers and the steady-state drivers (oracle; test
infrastructure only).

Section "Iterative solvers" solves Eq. (linear) with an iLU preconditioner M
by restarted GMRES (Saad and Schultz 1986) or BiCGSTAB (van der Vorst 1992),
stopping on the L2 norm of the residual with an iteration cap (1000 in the
numerical section). Both are written here with right preconditioning,
A M^{-1} u = b, x = M^{-1} u, which has the same solution as the left form of
Eq. (modified) and whose recursively updated residual is the residual of the
unpreconditioned system.

The doubly-iterative inverse-power method (sections "Eigenvalue Methods" and
"Iterative solvers") applies power iteration to (L - sigma I)^{-1}
(Eq. inverseiter) with each product computed by a preconditioned Krylov solve
whose tolerance is one tenth of the outer tolerance.

Inner products are <a, b> = sum conj(a_i) b_i.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp

from . import ilu as _ilu
from .liouvillian import (default_weight, liouvillian_sparse, modified_liouvillian,
                          shifted_liouvillian, trace_columns)
from .ordering import permute_symmetric, rcm_order
from .rng import start_vector

OK, NOT_CONVERGED, BREAKDOWN = 0, 3, 4


@dataclass
class KrylovResult:
    x: np.ndarray
    status: int
    iters: int
    resid: float
    history: list = field(default_factory=list)


def _breakdown(a: complex, u: np.ndarray, v: np.ndarray, rel: float = 1e-15) -> bool:
    """|<u, v>| negligible against ||u|| ||v|| (or exactly zero)."""
    return abs(a) == 0.0 or abs(a) < rel * np.linalg.norm(u) * np.linalg.norm(v)


def bicgstab(matvec: Callable, psolve: Callable, b: np.ndarray, x0: Optional[np.ndarray],
             tol: float, maxiter: int = 1000) -> KrylovResult:
    """Right-preconditioned BiCGSTAB; stops when ||b - A x||_2 <= tol (absolute).

    Per iteration: rho = <r^, r>; p = r + beta (p - omega v) with
    beta = (rho / rho_prev)(alpha / omega); p^ = M^{-1} p; v = A p^;
    alpha = rho / <r^, v>; s = r - alpha v; s^ = M^{-1} s; t = A s^;
    omega = <t, s> / <t, t>; x += alpha p^ + omega s^; r = s - omega t.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    r = b - matvec(x)
    rn = np.linalg.norm(r)
    hist = [rn]
    if rn <= tol:
        return KrylovResult(x, OK, 0, rn, hist)
    rhat = r.copy()
    rho_prev = alpha = omega = 1.0 + 0j
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    for it in range(1, maxiter + 1):
        rho = np.vdot(rhat, r)
        if _breakdown(rho, rhat, r):
            return KrylovResult(x, BREAKDOWN, it - 1, rn, hist)
        if it == 1:
            p = r.copy()
        else:
            beta = (rho / rho_prev) * (alpha / omega)
            p = r + beta * (p - omega * v)
        phat = psolve(p)
        v = matvec(phat)
        rv = np.vdot(rhat, v)
        if _breakdown(rv, rhat, v):
            return KrylovResult(x, BREAKDOWN, it - 1, rn, hist)
        alpha = rho / rv
        s = r - alpha * v
        sn = np.linalg.norm(s)
        if sn <= tol:
            x = x + alpha * phat
            hist.append(sn)
            return KrylovResult(x, OK, it, sn, hist)
        shat = psolve(s)
        t = matvec(shat)
        tt = np.vdot(t, t).real
        if tt == 0.0:
            return KrylovResult(x, BREAKDOWN, it, rn, hist)
        omega = np.vdot(t, s) / tt
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rn = np.linalg.norm(r)
        hist.append(rn)
        if rn <= tol:
            return KrylovResult(x, OK, it, rn, hist)
        if omega == 0.0:
            return KrylovResult(x, BREAKDOWN, it, rn, hist)
        rho_prev = rho
    return KrylovResult(x, NOT_CONVERGED, maxiter, rn, hist)


def _givens(a: complex, b: complex):
    """(c, s, r) with c real, [[c, s], [-conj(s), c]] [a, b]^T = [r, 0]^T."""
    if b == 0:
        return 1.0, 0.0 + 0j, a
    if a == 0:
        return 0.0, 1.0 + 0j, b
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    phase = a / abs(a)
    s = phase * np.conj(b) / t
    return c, s, phase * t


def gmres(matvec: Callable, psolve: Callable, b: np.ndarray, x0: Optional[np.ndarray],
          tol: float, restart: int = 30, maxiter: int = 1000) -> KrylovResult:
    """Right-preconditioned restarted GMRES(m) with Arnoldi (modified
    Gram-Schmidt) and Givens rotations; stops when the residual norm of the
    least-squares problem, ||b - A x||_2, is <= tol (absolute). maxiter counts
    inner (Arnoldi) steps."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    m = restart
    total = 0
    hist = []
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta)
        if beta <= tol:
            return KrylovResult(x, OK, total, beta, hist)
        if total >= maxiter:
            return KrylovResult(x, NOT_CONVERGED, total, beta, hist)
        V = [r / beta]
        Z = []
        Hm = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        resid = beta
        for j in range(m):
            z = psolve(V[j])
            Z.append(z)
            w = matvec(z)
            for i in range(j + 1):
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            V.append(w / Hm[j + 1, j] if Hm[j + 1, j] != 0 else w)
            for i in range(j):
                a_, b_ = Hm[i, j], Hm[i + 1, j]
                Hm[i, j] = cs[i] * a_ + sn[i] * b_
                Hm[i + 1, j] = -np.conj(sn[i]) * a_ + cs[i] * b_
            c, s, rr = _givens(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = c, s
            Hm[j, j] = rr
            Hm[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            k = j + 1
            total += 1
            resid = abs(g[j + 1])
            hist.append(resid)
            if resid <= tol or total >= maxiter or Hm[j, j] == 0:
                break
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(Hm[i, i + 1:k], y[i + 1:k])) / Hm[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]


def lgmres(matvec: Callable, psolve: Callable, b: np.ndarray, x0: Optional[np.ndarray],
           tol: float, restart: int = 30, augment: int = 3, maxiter: int = 1000,
           max_cycles: Optional[int] = None) -> KrylovResult:
    """Right-preconditioned LGMRES(m, k) (Baker, Jessup and Manteuffel 2005):
    the restarted GMRES of section "Iterative solvers" with each restart
    space augmented by the corrections of earlier cycles (the solver named
    "iterative-lgmres").

    A cycle starting from x with residual r = b - A x minimises
    ||b - A (x + Z y)||_2 over the columns of
        Z = [M^{-1} v_0, ..., M^{-1} v_{m-1}, e_1, ..., e_k'],
    where v_0 = r / ||r|| and each v_{j+1} comes from orthonormalising A z_j
    against v_0..v_j (Arnoldi, modified Gram-Schmidt), and e_1..e_k' are the
    normalised corrections x_{c} - x_{c-1} of the k' <= k most recent cycles
    (oldest first). The correction of this cycle, Z y, is normalised and
    appended; the oldest is dropped beyond k. With k = 0 this is GMRES(m).
    Stops when the least-squares residual is <= tol (absolute). maxiter counts
    Arnoldi steps (an augmented direction costs one product with A and no
    preconditioner application); max_cycles, when given, ends the solve after
    that many cycles."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    m = restart
    corrections: list = []
    total = 0
    cycles = 0
    hist = []
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta)
        if beta <= tol:
            return KrylovResult(x, OK, total, beta, hist)
        if total >= maxiter or (max_cycles is not None and cycles >= max_cycles):
            return KrylovResult(x, NOT_CONVERGED, total, beta, hist)
        dim = m + len(corrections)
        V = [r / beta]
        Z = []
        Hm = np.zeros((dim + 1, dim), dtype=np.complex128)
        cs = np.zeros(dim)
        sn = np.zeros(dim, dtype=np.complex128)
        g = np.zeros(dim + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(dim):
            z = psolve(V[j]) if j < m else corrections[j - m]
            Z.append(z)
            w = matvec(z)
            for i in range(j + 1):
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            V.append(w / Hm[j + 1, j] if Hm[j + 1, j] != 0 else w)
            for i in range(j):
                a_, b_ = Hm[i, j], Hm[i + 1, j]
                Hm[i, j] = cs[i] * a_ + sn[i] * b_
                Hm[i + 1, j] = -np.conj(sn[i]) * a_ + cs[i] * b_
            c, s, rr = _givens(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = c, s
            Hm[j, j] = rr
            Hm[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            k = j + 1
            total += 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol or total >= maxiter or Hm[j, j] == 0:
                break
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(Hm[i, i + 1:k], y[i + 1:k])) / Hm[i, i]
        dx = np.zeros_like(x)
        for i in range(k):
            dx = dx + y[i] * Z[i]
        x = x + dx
        cycles += 1
        nd = np.linalg.norm(dx)
        if augment > 0 and nd > 0:
            corrections.append(dx / nd)
            if len(corrections) > augment:
                corrections.pop(0)


# Ratio of RCM bandwidths above which the trace row is taken to spoil the
# bandwidth reduction (section "Results"/"Conclusion": GMRES on L~ when the
# RCM bandwidths of L~ and L - sigma I are nearly the same, the
# doubly-iterative inverse-power method otherwise). The paper prints the two
# bandwidths for three systems (Fig. 1 and Fig. 3): ratios 139/137 and
# 239/229 for the Jaynes-Cummings and optomechanical models, where GMRES on L~
# is the method of choice, and 405/167 for the 5-spin chain, whose bandwidth
# grows enough to favour inverse power; 1.5 separates them.
AUTO_BANDWIDTH_RATIO = 1.5


def select_method(H, c_ops, sigma: float = 1e-15, w: Optional[float] = None,
                  ratio: float = AUTO_BANDWIDTH_RATIO):
    """The paper's choice of iterative method from the RCM bandwidths of the
    modified Liouvillian L~ = L + wT (Eq. linear) and the shifted L - sigma I
    (Eq. inverse). Returns (method, B_modified, B_shifted) with method
    "gmres" when B_modified <= ratio * B_shifted, else "power-gmres"."""
    from .ordering import bandwidth_profile
    d = H.shape[0]
    L = liouvillian_sparse(H, c_ops)
    wv = default_weight(L) if (w is None or w <= 0) else float(w)
    Am = modified_liouvillian(L, d, wv)[0]
    As = shifted_liouvillian(L, sigma)
    bm = bandwidth_profile(permute_symmetric(Am, rcm_order(Am)))[0]
    bs = bandwidth_profile(permute_symmetric(As, rcm_order(As)))[0]
    return ("gmres" if bm <= ratio * bs else "power-gmres"), bm, bs


# ---------------------------------------------------------------------------
# Steady-state drivers on the CPU (the "plain CPU sparse iterative solver")
# ---------------------------------------------------------------------------

@dataclass
class SteadyResult:
    rho: np.ndarray
    status: int
    iters: int
    outer_iters: int
    resid_Lrho: float
    perm: np.ndarray
    w: float = 0.0


def _trace(x: np.ndarray, d: int) -> complex:
    return complex(np.sum(x[trace_columns(d)]))


def _lrho_norm(L: sp.csr_matrix, x: np.ndarray, d: int) -> float:
    return float(np.linalg.norm(L @ (x / _trace(x, d))))


def steady_state_iterative(H, c_ops, method: str = "bicgstab", precond: str = "ilu0",
                           tol: float = 1e-10, maxiter: int = 1000, restart: int = 30,
                           drop_tol: float = 1e-4, fill_factor: float = 10.0,
                           w: Optional[float] = None, sigma: float = 1e-15, seed: int = 0,
                           use_rcm: bool = True, fast_triangular: bool = True,
                           augment: int = 0) -> SteadyResult:
    """Sparse steady state on the CPU: L, then L~ = L + wT (or L - sigma I for
    inverse power), RCM of the symmetrised pattern, iLU, Krylov, and the
    trace-normalised rho. The accepted result satisfies ||L rho||_2 <= tol.

    The Krylov stop is an absolute residual bound that starts at tol / 2 and is
    tightened tenfold (restarting from the current iterate) whenever the
    acceptance test ||L rho||_2 <= tol fails; a BiCGSTAB breakdown after at
    least one iteration restarts from the current iterate with a fresh shadow
    residual (at most 8 passes, 1000 iterations in all). For inverse power
    each inner solve uses tol / 10 relative to ||x_k|| = 1 (section
    "Iterative solvers").

    method "gmres"/"lgmres" (and "power-gmres") run LGMRES(restart, augment),
    which is GMRES(restart) for augment = 0; method "auto" takes
    select_method's choice.
    """
    if method == "auto":
        method = select_method(H, c_ops, sigma=sigma, w=w)[0]
    d = H.shape[0]
    n = d * d
    L = liouvillian_sparse(H, c_ops)
    power = method in ("inverse-power", "power-bicgstab", "power-gmres")
    if power:
        A = shifted_liouvillian(L, sigma)
        wv = 0.0
    else:
        wv = default_weight(L) if (w is None or w <= 0) else float(w)
        A, b = modified_liouvillian(L, d, wv)
    perm = rcm_order(A) if use_rcm else np.arange(n)
    Ap = permute_symmetric(A, perm)
    if precond == "ilu0":
        F = _ilu.ilu0(Ap)
    elif precond == "ilut":
        F = _ilu.ilut(Ap, drop_tol=drop_tol, fill_factor=fill_factor)
    else:
        raise ValueError(precond)
    if fast_triangular:
        Lf, Uf = _ilu.split_factors(F)
        from scipy.sparse.linalg import spsolve_triangular

        def psolve(r):
            return spsolve_triangular(Uf, spsolve_triangular(Lf, r, lower=True, unit_diagonal=True),
                                      lower=False)
    else:
        def psolve(r):
            return _ilu.upper_solve(F, _ilu.lower_solve(F, r))

    def matvec(v):
        return Ap @ v

    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)

    def unpermute(xp):
        x = np.empty_like(xp)
        x[perm] = xp
        return x

    if method in ("gmres", "lgmres", "power-gmres"):
        krylov = gmres if augment == 0 else lgmres
        kw = dict(restart=restart) if augment == 0 else dict(restart=restart, augment=augment)
    else:
        krylov = bicgstab
        kw = {}

    if power:
        x = start_vector(n, seed)
        x = x / np.linalg.norm(x)
        total = 0
        for outer in range(1, 101):
            res = krylov(matvec, psolve, x[perm], None, tol / 10.0, maxiter=maxiter, **kw)
            total += res.iters
            v = unpermute(res.x)
            x = v / np.linalg.norm(v)
            lr = _lrho_norm(L, x, d)
            if lr <= tol:
                return SteadyResult(_unvec_norm(x, d), OK, total, outer, lr, perm, 0.0)
        return SteadyResult(_unvec_norm(x, d), NOT_CONVERGED, total, outer, lr, perm, 0.0)

    bp = b[perm]
    inner = 0.5 * tol
    xp = None
    total = 0
    status = NOT_CONVERGED
    lr = np.inf
    for _ in range(8):
        res = krylov(matvec, psolve, bp, xp, inner, maxiter=maxiter - total, **kw)
        total += res.iters
        xp = res.x
        x = unpermute(xp)
        lr = _lrho_norm(L, x, d)
        if lr <= tol:
            status = OK
            break
        if total >= maxiter or res.status == NOT_CONVERGED or (res.status == BREAKDOWN and res.iters == 0):
            status = res.status if res.status != OK else NOT_CONVERGED
            break
        if res.status == OK:
            inner /= 10.0
        # BREAKDOWN after progress: restart from the current iterate with a new shadow residual
    return SteadyResult(_unvec_norm(x, d), status, total, 1, lr, perm, wv)


def _unvec_norm(x: np.ndarray, d: int) -> np.ndarray:
    rho = x.reshape((d, d), order="F").copy()
    return rho / np.trace(rho)
