"""Density-matrix metrics (oracle; test infrastructure only).

Trace distance and fidelity are the diagnostics the paper suggests for
spotting an ill-conditioned zero eigenvalue (section "Eigenvalue Methods").
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as la


def hermitian_part(rho: np.ndarray) -> np.ndarray:
    return 0.5 * (rho + rho.conj().T)


def trace_distance(rho1: np.ndarray, rho2: np.ndarray) -> float:
    """T = 1/2 sum |eig(h1 - h2)| with h = Hermitian part of each argument."""
    diff = hermitian_part(np.asarray(rho1)) - hermitian_part(np.asarray(rho2))
    return 0.5 * float(np.sum(np.abs(np.linalg.eigvalsh(diff))))


def fidelity(rho1: np.ndarray, rho2: np.ndarray) -> float:
    """Uhlmann fidelity Tr sqrt(sqrt(r1) r2 sqrt(r1))."""
    s = la.sqrtm(hermitian_part(rho1))
    m = la.sqrtm(s @ hermitian_part(rho2) @ s)
    return float(np.real(np.trace(m)))


def hermiticity_error(rho: np.ndarray) -> float:
    return float(np.max(np.abs(rho - rho.conj().T)))


def min_eigenvalue(rho: np.ndarray) -> float:
    return float(np.min(np.linalg.eigvalsh(hermitian_part(rho))))


def residual_norm(L, rho: np.ndarray) -> float:
    """||L vec(rho)||_2 for a given L (dense or sparse)."""
    x = np.asarray(rho).reshape(-1, order="F")
    return float(np.linalg.norm(L @ x))
