"""Lindblad Liouvillian in matrix form (oracle; test infrastructure only).

Eq. (lindblad) with the dissipator D[C, rho] = C rho C^+ - (rho C^+C + C^+C rho)/2,
vectorised by column stacking as in Eq. (eigval): vec(rho)[i + d*j] = rho[i, j],
so vec(A rho B) = (B^T kron A) vec(rho) and

    L = -i (I kron H - H^T kron I)
        + sum_k ( conj(C_k) kron C_k - 1/2 I kron C_k^+C_k - 1/2 (C_k^+C_k)^T kron I ).

Pattern convention: an entry of L is stored iff its summed value is nonzero
(exact cancellations are dropped), so the pattern is that of the dense matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _dense(m) -> np.ndarray:
    return m.toarray() if sp.issparse(m) else np.asarray(m, dtype=np.complex128)


def liouvillian_dense(H, c_ops) -> np.ndarray:
    """Dense n x n L (n = d^2) from numpy.kron, term by term as written above."""
    Hd = _dense(H)
    d = Hd.shape[0]
    eye = np.eye(d, dtype=np.complex128)
    L = -1j * (np.kron(eye, Hd) - np.kron(Hd.T, eye))
    for C in c_ops:
        Cd = _dense(C)
        CdC = Cd.conj().T @ Cd
        L = L + np.kron(Cd.conj(), Cd) - 0.5 * np.kron(eye, CdC) - 0.5 * np.kron(CdC.T, eye)
    return L


def liouvillian_sparse(H, c_ops) -> sp.csr_matrix:
    """The same L built with scipy.sparse.kron (for sizes where dense is too big)."""
    H = sp.csr_matrix(H, dtype=np.complex128)
    d = H.shape[0]
    eye = sp.identity(d, dtype=np.complex128, format="csr")
    L = -1j * (sp.kron(eye, H) - sp.kron(H.T, eye))
    for C in c_ops:
        C = sp.csr_matrix(C, dtype=np.complex128)
        CdC = (C.conj().T @ C).tocsr()
        L = L + sp.kron(C.conj(), C) - 0.5 * sp.kron(eye, CdC) - 0.5 * sp.kron(CdC.T, eye)
    L = sp.csr_matrix(L)
    L.sum_duplicates()
    L.eliminate_zeros()
    L.sort_indices()
    return L


def liouvillian_apply(H, c_ops, x: np.ndarray) -> np.ndarray:
    """Matrix-free L x: unstack x to rho, evaluate Eq. (lindblad), restack."""
    d = H.shape[0]
    X = np.asarray(x, dtype=np.complex128).reshape((d, d), order="F")
    Hs = sp.csr_matrix(H)
    Y = -1j * (Hs @ X - (Hs.T @ X.T).T)
    for C in c_ops:
        Cs = sp.csr_matrix(C)
        CX = Cs @ X
        Y = Y + (Cs.conj() @ CX.T).T                      # C X C^+
        CdC = (Cs.conj().T @ Cs).tocsr()
        Y = Y - 0.5 * ((CdC.T @ X.T).T + CdC @ X)          # X C^+C + C^+C X
    return np.asarray(Y).reshape(-1, order="F")


def liouvillian_row(H, c_ops, p: int) -> np.ndarray:
    """Row p of L (dense, length d^2) from the element-wise form of Eq. (lindblad).

    With p = i + d j (the equation for drho_ij/dt) and column q = k + d l (rho_kl):
      L[p, q] = -i (delta_jl H_ik - delta_ik H_lj)
                + sum_c ( C_ik conj(C_jl) - 1/2 delta_jl (C^+C)_ik - 1/2 delta_ik (C^+C)_lj ).
    """
    d = H.shape[0]
    i, j = p % d, p // d
    Hs = sp.csr_matrix(H)
    M = np.zeros((d, d), dtype=np.complex128)            # M[k, l] = L[p, k + d l]
    M[:, j] += -1j * Hs.getrow(i).toarray().ravel()
    M[i, :] += 1j * Hs.getcol(j).toarray().ravel()
    for C in c_ops:
        Cs = sp.csr_matrix(C)
        CdC = (Cs.conj().T @ Cs).tocsr()
        M += np.outer(Cs.getrow(i).toarray().ravel(), Cs.getrow(j).toarray().ravel().conj())
        M[:, j] += -0.5 * CdC.getrow(i).toarray().ravel()
        M[i, :] += -0.5 * CdC.getcol(j).toarray().ravel()
    return M.reshape(-1, order="F")


def trace_columns(d: int) -> np.ndarray:
    """Indices of the diagonal elements rho_ii in vec(rho): i (d + 1)."""
    return np.arange(d, dtype=np.int64) * (d + 1)


def modified_liouvillian(L, d: int, w: float):
    """Eq. (linear): L~ = L + w T with T = ones in row 0 at the diagonal-element
    columns; returns (L~, b) with b = (w, 0, ..., 0)."""
    n = d * d
    rows = np.zeros(d, dtype=np.int64)
    T = sp.csr_matrix((np.ones(d, dtype=np.complex128), (rows, trace_columns(d))), shape=(n, n))
    if sp.issparse(L):
        Lt = sp.csr_matrix(L + w * T)
        Lt.sum_duplicates()
        Lt.eliminate_zeros()
        Lt.sort_indices()
    else:
        Lt = L + w * T.toarray()
    b = np.zeros(n, dtype=np.complex128)
    b[0] = w
    return Lt, b


def default_weight(L) -> float:
    """The weighting factor w read as the mean modulus of L's diagonal (1 when
    that mean is zero, since any positive w gives the same solution)."""
    diag = L.diagonal() if sp.issparse(L) else np.diag(L)
    w = float(np.mean(np.abs(diag)))
    return w if w > 0.0 else 1.0


def shifted_liouvillian(L, sigma: float = 1e-15):
    """Eq. (inverse): L - sigma I (the diagonal is always stored)."""
    n = L.shape[0]
    if sp.issparse(L):
        S = sp.csr_matrix(L - sigma * sp.identity(n, dtype=np.complex128, format="csr"))
        S.sum_duplicates()
        S.sort_indices()
        return S
    return L - sigma * np.eye(n, dtype=np.complex128)
