"""Pins for the oracle's density-matrix metrics (trace distance, fidelity),
the checkers every parity test relies on.

Each case has a value fixed by the mathematics, not by the function under
test: Bloch-vector closed forms for qubits, the overlap formulas for pure
states, and the classical (commuting) limits.
"""
import numpy as np
import pytest

from oracle.metrics import fidelity, hermitian_part, trace_distance

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
SZ = np.array([[1, 0], [0, -1]], dtype=complex)


def _qubit(r):
    """rho = (I + r . sigma) / 2 for a Bloch vector |r| <= 1."""
    return 0.5 * (np.eye(2) + r[0] * SX + r[1] * SY + r[2] * SZ)


def _ket(v):
    v = np.asarray(v, dtype=complex)
    return v / np.linalg.norm(v)


def _random_state(d, rng, rank=None):
    rank = rank or d
    g = rng.standard_normal((d, rank)) + 1j * rng.standard_normal((d, rank))
    rho = g @ g.conj().T
    return rho / np.trace(rho)


def test_trace_distance_zero_for_equal_states():
    rng = np.random.default_rng(0)
    rho = _random_state(6, rng)
    assert trace_distance(rho, rho) == 0.0


def test_trace_distance_one_for_orthogonal_pure_states():
    a, b = _ket([1, 1j, 0]), _ket([1, -1j, 0])      # <a|b> = 0
    assert abs(np.vdot(a, b)) < 1e-15
    assert trace_distance(np.outer(a, a.conj()), np.outer(b, b.conj())) == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("r1,r2", [((0, 0, 1), (0, 0, -1)), ((0.3, -0.2, 0.5), (-0.1, 0.4, 0.2)),
                                   ((0, 0, 0), (0.6, 0.0, 0.8)), ((0.5, 0.5, 0.5), (0.5, 0.5, 0.4))])
def test_trace_distance_qubit_bloch_closed_form(r1, r2):
    """For qubits T = |r1 - r2| / 2 (the eigenvalues of (r1 - r2) . sigma / 2
    are +-|r1 - r2| / 2)."""
    expect = 0.5 * np.linalg.norm(np.subtract(r1, r2))
    assert trace_distance(_qubit(r1), _qubit(r2)) == pytest.approx(expect, abs=1e-15)


def test_trace_distance_pure_states_overlap():
    """For pure states T = sqrt(1 - |<a|b>|^2)."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = _ket(rng.standard_normal(5) + 1j * rng.standard_normal(5))
        b = _ket(rng.standard_normal(5) + 1j * rng.standard_normal(5))
        expect = np.sqrt(1 - abs(np.vdot(a, b)) ** 2)
        assert trace_distance(np.outer(a, a.conj()), np.outer(b, b.conj())) == pytest.approx(expect, abs=1e-12)


def test_trace_distance_commuting_states_total_variation():
    """Diagonal states: T is the total-variation distance 1/2 sum |p_i - q_i|."""
    p = np.array([0.5, 0.3, 0.2, 0.0])
    q = np.array([0.1, 0.1, 0.4, 0.4])
    assert trace_distance(np.diag(p), np.diag(q)) == pytest.approx(0.5 * np.abs(p - q).sum(), abs=1e-15)


def test_trace_distance_uses_hermitian_parts_and_is_a_metric():
    """An anti-Hermitian perturbation does not count (the iterate is compared
    through its Hermitian part); symmetry and the triangle inequality hold."""
    rng = np.random.default_rng(2)
    r1, r2, r3 = (_random_state(5, rng) for _ in range(3))
    k = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    anti = 1e-3 * (k - k.conj().T)
    assert np.allclose(hermitian_part(anti), 0)
    assert trace_distance(r1 + anti, r2) == pytest.approx(trace_distance(r1, r2), abs=1e-14)
    assert trace_distance(r1, r2) == pytest.approx(trace_distance(r2, r1), abs=1e-15)
    assert trace_distance(r1, r3) <= trace_distance(r1, r2) + trace_distance(r2, r3) + 1e-15


def test_fidelity_pure_states_is_overlap():
    """Uhlmann (root) fidelity of pure states is |<a|b>|; of a state with
    itself, 1."""
    rng = np.random.default_rng(3)
    a = _ket(rng.standard_normal(4) + 1j * rng.standard_normal(4))
    b = _ket(rng.standard_normal(4) + 1j * rng.standard_normal(4))
    pa, pb = np.outer(a, a.conj()), np.outer(b, b.conj())
    assert fidelity(pa, pb) == pytest.approx(abs(np.vdot(a, b)), abs=1e-7)
    rho = _random_state(4, rng)
    assert fidelity(rho, rho) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("r1,r2", [((0.3, -0.2, 0.5), (-0.1, 0.4, 0.2)), ((0, 0, 0), (0.6, 0.0, 0.8)),
                                   ((0.1, 0.2, 0.3), (0.1, 0.2, 0.3))])
def test_fidelity_qubit_closed_form(r1, r2):
    """Qubits: F^2 = Tr(r1 r2) + 2 sqrt(det r1 det r2), with
    Tr(rho1 rho2) = (1 + r1 . r2) / 2 and det rho = (1 - |r|^2) / 4."""
    r1, r2 = np.asarray(r1, float), np.asarray(r2, float)
    f2 = 0.5 * (1 + r1 @ r2) + 2 * np.sqrt((1 - r1 @ r1) / 4 * (1 - r2 @ r2) / 4)
    assert fidelity(_qubit(r1), _qubit(r2)) == pytest.approx(np.sqrt(f2), abs=1e-10)


def test_fidelity_commuting_states_bhattacharyya():
    p = np.array([0.5, 0.3, 0.2])
    q = np.array([0.1, 0.6, 0.3])
    assert fidelity(np.diag(p), np.diag(q)) == pytest.approx(np.sqrt(p * q).sum(), abs=1e-12)


def test_fuchs_van_de_graaf_bounds():
    """1 - F <= T <= sqrt(1 - F^2) ties the two metrics together."""
    rng = np.random.default_rng(4)
    for _ in range(5):
        r1, r2 = _random_state(4, rng), _random_state(4, rng)
        t, f = trace_distance(r1, r2), fidelity(r1, r2)
        assert 1 - f <= t + 1e-9 and t <= np.sqrt(max(1 - f * f, 0.0)) + 1e-9
