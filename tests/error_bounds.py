"""Tolerances derived from the arithmetic (test infrastructure).

precond_error_bound gives a componentwise bound on the error of
z = U^{-1} (L^{-1} r) computed by forward then back substitution in a
floating-point format with unit roundoff u, for the incomplete factors F
(strict lower part = L with unit diagonal, diagonal and upper part = U, the
layout of the solver's exported factors).

Backward error of substitution (Higham, "Accuracy and Stability of Numerical
Algorithms", 2nd ed., Thm 8.5): the computed solution of T x = b satisfies
(T + dT) x_hat = b with |dT| <= c |T| componentwise, c = gamma_{k+1} for rows
of at most k entries in real arithmetic; complex multiply-adds carried out as
real operations add a factor sqrt(2) and two more roundings per row
(Higham, Lemma 3.5), and the upper solve's multiplication by a rounded
1 / u_ii adds two more.  Forward error: x_hat - x = -T^{-1} dT x_hat, and for
a triangular T, |T^{-1}| <= M(T)^{-1} with M(T) the comparison matrix
(|t_ii| on the diagonal, -|t_ij| off it; Higham Thm 8.12), so

    |y_hat - y| <= c_L M(L)^{-1} |L| |y|
    |z_hat - z| <= M(U)^{-1} (|y_hat - y| + c_U |U| |z|)

to first order.  Every solve here has nonnegative data, so it is computed
without cancellation.  The caller multiplies by a small factor for the
second-order terms and for the rounding of a reference solve done in the
same format.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular

U_FP32 = 2.0 ** -24
U_FP64 = 2.0 ** -53


def _gamma(m: int, u: float) -> float:
    return m * u / (1.0 - m * u)


def split(F: sp.csr_matrix):
    """Unit lower L and upper U (with the diagonal) of the combined factors."""
    F = sp.csr_matrix(F)
    n = F.shape[0]
    L = sp.tril(F, k=-1, format="csr") + sp.identity(n, dtype=F.dtype, format="csr")
    U = sp.triu(F, k=0, format="csr")
    return L.tocsr(), U.tocsr()


def precond_error_bound(F: sp.csr_matrix, y: np.ndarray, z: np.ndarray, u: float) -> np.ndarray:
    """First-order componentwise bound on |z_hat - z| (see the module text);
    y = L^{-1} r and z = U^{-1} y are the exact (reference) solutions."""
    L, U = split(F)
    kl = int(np.max(np.diff(L.indptr)))          # entries per row, diagonal included
    ku = int(np.max(np.diff(U.indptr)))
    c_l = np.sqrt(2.0) * _gamma(kl + 3, u)
    c_u = np.sqrt(2.0) * _gamma(ku + 5, u)
    aL, aU = abs(L).tocsr(), abs(U).tocsr()
    d = np.abs(U.diagonal())
    ML = (2 * sp.identity(L.shape[0], format="csr") - aL).tocsr()          # I - |strict L|
    MU = (2 * sp.diags(d, format="csr") - aU).tocsr()                      # diag|u_ii| - |strict U|
    ey = c_l * spsolve_triangular(ML, aL @ np.abs(y), lower=True)
    return spsolve_triangular(MU, ey + c_u * (aU @ np.abs(z)), lower=False)
