"""Tolerances derived from the arithmetic (test infrastructure).

precond_backward_check bounds the componentwise backward error of
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
1 / u_ii adds two more.  With (L + dL) y_hat = r and (U + dU) z_hat = y_hat:

    r - L U z_hat = L dU z_hat + dL y_hat,   |y_hat| <= (1 + c_U) |U| |z_hat|

so, componentwise,

    |r - L U z_hat| <= (c_U + c_L (1 + c_U)) |L| |U| |z_hat|.

The left side is evaluated here in FP64, whose own rounding (at most
sqrt(2) gamma_{kL+kU+2}(2^-53) |L| |U| |z_hat| for the two products and the
subtraction, the same lemma) is added to the bound.  The test needs only
the kernel's output: it holds whatever the conditioning of the factors (the
forward error is this backward error magnified by the condition, which for
iLU factors of the Liouvillians can be very large), and a wrong value or a
dropped term leaves a residual of the size of that term, orders of magnitude
above the bound.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

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


def precond_backward_check(F: sp.csr_matrix, r: np.ndarray, z_hat: np.ndarray, u: float):
    """(|r - L U z_hat|, bound) componentwise, for z_hat computed from r by
    substitution in a format with unit roundoff u (see the module text).
    The constants are per row (c_L(i), c_U(i) from the row's entry count), so

        bound = |L| (c_U .* (|U| |z|)) + (c_L (1 + max c_U) + c_eval) .* (|L| |U| |z|)."""
    L, U = split(F)
    kl = np.diff(L.indptr)                        # entries per row, diagonal included
    ku = np.diff(U.indptr)
    c_l = np.sqrt(2.0) * _gamma(kl + 3, u)
    c_u = np.sqrt(2.0) * _gamma(ku + 5, u)
    c_eval = np.sqrt(2.0) * _gamma(kl + int(np.max(ku)) + 2, U_FP64)
    z = np.asarray(z_hat, dtype=np.complex128)
    resid = np.abs(np.asarray(r, dtype=np.complex128) - L @ (U @ z))
    aL, aU = abs(L), abs(U)
    uz = aU @ np.abs(z)
    scale = aL @ uz
    return resid, aL @ (c_u * uz) + (c_l * (1.0 + np.max(c_u)) + c_eval) * scale
