"""Pins for the oracle's dense steady state: closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle.liouvillian import liouvillian_dense
from oracle.metrics import hermiticity_error, min_eigenvalue, residual_norm, trace_distance
from oracle.steady import steady_state_dense, steady_state_svd
from workloads import driven_cavity, kerr_oscillator, random_system, thermal_cavity, two_level_atom


def _coherent(N, alpha):
    n = np.arange(N)
    logf = np.array([math.lgamma(k + 1) for k in n])
    c = np.exp(-abs(alpha) ** 2 / 2) * np.exp(n * np.log(abs(alpha)) - 0.5 * logf) * np.exp(1j * n * np.angle(alpha))
    c = c / np.linalg.norm(c)
    return np.outer(c, c.conj())


@pytest.mark.parametrize("delta,E,kappa", [(0.5, 0.3, 1.0), (0.0, 0.8, 2.0), (-1.0, 0.5, 0.7)])
def test_coherent_state_closed_form(delta, E, kappa):
    """Driven damped cavity at zero temperature: rho = |alpha><alpha| with
    alpha = -iE / (i delta + kappa / 2). The Fock cutoff N = 30 keeps the
    truncation error (of order |alpha|^N / sqrt(N!)) far below the bound."""
    s = driven_cavity(N=30, delta=delta, E=E, kappa=kappa, n_th=0.0)
    rho = steady_state_dense(s.H, s.c_ops)
    alpha = -1j * E / (1j * delta + kappa / 2)
    assert trace_distance(rho, _coherent(30, alpha)) < 1e-12


def test_coherent_wrong_sign_fails():
    """The pin is sensitive to a sign error in alpha."""
    s = driven_cavity(N=20, n_th=0.0)
    rho = steady_state_dense(s.H, s.c_ops)
    alpha = +1j * 0.3 / (1j * 0.5 + 0.5)
    assert trace_distance(rho, _coherent(20, alpha)) > 1e-2


@pytest.mark.parametrize("n_th", [0.2, 1.0])
def test_thermal_state_closed_form(n_th):
    """Undriven cavity in a thermal bath: rho_nn = (1 - q) q^n / (1 - q^N),
    q = n_th / (1 + n_th), no coherences, <n> -> n_th."""
    N = 20
    s = thermal_cavity(N=N, n_th=n_th)
    rho = steady_state_dense(s.H, s.c_ops)
    q = n_th / (1 + n_th)
    p = (1 - q) * q ** np.arange(N) / (1 - q ** N)
    np.testing.assert_allclose(np.diag(rho).real, p, atol=1e-13)
    off = rho - np.diag(np.diag(rho))
    assert np.max(np.abs(off)) < 1e-13
    if n_th == 0.2:
        assert float(np.sum(np.arange(N) * np.diag(rho).real)) == pytest.approx(0.2, abs=1e-12)


@pytest.mark.parametrize("omega,gamma", [(1.0, 0.5), (0.3, 2.0)])
def test_resonant_two_level_atom(omega, gamma):
    """Optical Bloch equations on resonance: rho_ee = omega^2 / (gamma^2 + 2 omega^2)."""
    s = two_level_atom(omega=omega, gamma=gamma)
    rho = steady_state_dense(s.H, s.c_ops)
    assert rho[1, 1].real == pytest.approx(omega ** 2 / (gamma ** 2 + 2 * omega ** 2), abs=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_invariants_random_systems(seed):
    s = random_system(6, n_c=2, seed=seed)
    rho = steady_state_dense(s.H, s.c_ops)
    L = liouvillian_dense(s.H, s.c_ops)
    assert abs(np.trace(rho) - 1) < 1e-14
    assert hermiticity_error(rho) < 1e-12
    assert min_eigenvalue(rho) > -1e-12
    assert residual_norm(L, rho) < 1e-12
    assert trace_distance(rho, steady_state_svd(s.H, s.c_ops)) < 1e-11


def test_kerr_matches_svd_null_vector():
    s = kerr_oscillator(16, 0.3, 0.2, 0.9)
    assert trace_distance(steady_state_dense(s.H, s.c_ops), steady_state_svd(s.H, s.c_ops)) < 1e-11
