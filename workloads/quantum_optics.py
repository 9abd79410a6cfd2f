"""Operator builders for the synthetic workloads (Fock basis for oscillators,
z basis for spins, tensor order stated per system).

Parameter draws use ``numpy.random.default_rng(seed)`` (PCG64) in the order
listed in each builder's docstring, so a seed names one system exactly.

Conventions
-----------
* ``destroy(N)`` is the truncated annihilation operator, a|n> = sqrt(n)|n-1>.
* Two-level operators use the basis order (|g>, |e>), ground state first as
  for the Fock vacuum: sigma_z = |e><e| - |g><g| = diag(-1, 1) and
  sigma_minus = |g><e| maps index 1 to index 0.
* Collapse operators with a zero rate are omitted (they add nothing to the
  Liouvillian).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List

import numpy as np
import scipy.sparse as sp


@dataclass
class System:
    """One open system: H and collapse operators as CSR complex128 (d x d)."""

    name: str
    H: sp.csr_matrix
    c_ops: List[sp.csr_matrix]
    params: Dict[str, float] = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.H.shape[0]

    @property
    def n(self) -> int:
        return self.d * self.d


def _csr(m) -> sp.csr_matrix:
    m = sp.csr_matrix(m, dtype=np.complex128)
    m.sum_duplicates()
    m.eliminate_zeros()
    m.sort_indices()
    return m


def destroy(N: int) -> sp.csr_matrix:
    """Truncated annihilation operator on N Fock states."""
    return _csr(sp.diags(np.sqrt(np.arange(1, N, dtype=np.float64)), 1, shape=(N, N)))


def identity(N: int) -> sp.csr_matrix:
    return _csr(sp.identity(N, dtype=np.complex128))


def sigma_minus() -> sp.csr_matrix:
    return _csr(np.array([[0, 1], [0, 0]], dtype=np.complex128))


def sigma_x() -> sp.csr_matrix:
    return _csr(np.array([[0, 1], [1, 0]], dtype=np.complex128))


def sigma_y() -> sp.csr_matrix:
    return _csr(np.array([[0, -1j], [1j, 0]], dtype=np.complex128))


def sigma_z() -> sp.csr_matrix:
    return _csr(np.array([[-1, 0], [0, 1]], dtype=np.complex128))


def tensor(*ops) -> sp.csr_matrix:
    """Kronecker product of subsystem operators, leftmost factor slowest."""
    out = ops[0]
    for o in ops[1:]:
        out = sp.kron(out, o, format="csr")
    return _csr(out)


def _dag(m: sp.csr_matrix) -> sp.csr_matrix:
    return _csr(m.conj().T)


def _keep(rate: float, op: sp.csr_matrix, out: list) -> None:
    if rate > 0.0:
        out.append(_csr(np.sqrt(rate) * op))


# ---------------------------------------------------------------------------
# Systems of the benchmark configurations
# ---------------------------------------------------------------------------

def driven_cavity(N: int = 20, delta: float = 0.5, E: float = 0.3, kappa: float = 1.0,
                  n_th: float = 0.0) -> System:
    """H = delta a^+a + E(a + a^+); C = sqrt(kappa(n_th+1)) a, sqrt(kappa n_th) a^+."""
    a = destroy(N)
    ad = _dag(a)
    H = _csr(delta * (ad @ a) + E * (a + ad))
    c_ops: list = []
    _keep(kappa * (n_th + 1.0), a, c_ops)
    _keep(kappa * n_th, ad, c_ops)
    return System("driven_cavity", H, c_ops,
                  dict(N=N, delta=delta, E=E, kappa=kappa, n_th=n_th))


def thermal_cavity(N: int = 20, delta: float = 0.5, kappa: float = 1.0, n_th: float = 0.2) -> System:
    """The undriven (E = 0) cavity in a thermal bath."""
    s = driven_cavity(N=N, delta=delta, E=0.0, kappa=kappa, n_th=n_th)
    s.name = "thermal_cavity"
    return s


def jaynes_cummings_rwa(seed: int = 0, N: int = 40, delta_c: float = 0.0, delta_a: float = 0.0,
                        g: float = 1.0, kappa: float = 0.5, gamma: float = 0.1,
                        E: float | None = None) -> System:
    """Driven dissipative Jaynes-Cummings model in the rotating-wave form.

    Order: sigma_minus (x) I_N for the atom, I_2 (x) a for the cavity
    (d = 2N).  H = dc a^+a + da s+s- + g(a^+ s- + a s+) + E(a + a^+),
    C = sqrt(kappa) a, sqrt(gamma) s-.  Draw: E ~ U[0.2, 1.5].
    """
    if E is None:
        E = float(np.random.default_rng(seed).uniform(0.2, 1.5))
    sm = tensor(sigma_minus(), identity(N))
    a = tensor(identity(2), destroy(N))
    ad, sp_ = _dag(a), _dag(sm)
    H = _csr(delta_c * (ad @ a) + delta_a * (sp_ @ sm) + g * (ad @ sm + a @ sp_) + E * (a + ad))
    c_ops: list = []
    _keep(kappa, a, c_ops)
    _keep(gamma, sm, c_ops)
    return System("jaynes_cummings_rwa", H, c_ops,
                  dict(seed=seed, N=N, delta_c=delta_c, delta_a=delta_a, g=g, E=E,
                       kappa=kappa, gamma=gamma))


def optomechanics(seed: int = 0, Nc: int = 10, Nm: int = 40, omega_m: float = 1.0, g0: float = 0.1,
                  kappa: float = 0.2, gamma: float = 0.005, n_th: float = 2.0,
                  delta: float | None = None, E: float | None = None) -> System:
    """Driven optomechanical system, order a = a (x) I, b = I (x) b (d = Nc Nm).

    H = delta a^+a + wm b^+b - g0 a^+a (b + b^+) + E(a + a^+),
    C = sqrt(kappa) a, sqrt(gamma(n_th+1)) b, sqrt(gamma n_th) b^+.
    Draws in order: delta ~ U[-1.5, 1.5], E ~ U[0.1, 0.5].
    """
    rng = np.random.default_rng(seed)
    d_draw = float(rng.uniform(-1.5, 1.5))
    e_draw = float(rng.uniform(0.1, 0.5))
    delta = d_draw if delta is None else delta
    E = e_draw if E is None else E
    a = tensor(destroy(Nc), identity(Nm))
    b = tensor(identity(Nc), destroy(Nm))
    ad, bd = _dag(a), _dag(b)
    H = _csr(delta * (ad @ a) + omega_m * (bd @ b) - g0 * (ad @ a) @ (b + bd) + E * (a + ad))
    c_ops: list = []
    _keep(kappa, a, c_ops)
    _keep(gamma * (n_th + 1.0), b, c_ops)
    _keep(gamma * n_th, bd, c_ops)
    return System("optomechanics", H, c_ops,
                  dict(seed=seed, Nc=Nc, Nm=Nm, omega_m=omega_m, g0=g0, delta=delta, E=E,
                       kappa=kappa, gamma=gamma, n_th=n_th))


def kerr_oscillator(N: int, delta: float, K: float, E: float, kappa: float = 1.0) -> System:
    """H = delta a^+a + (K/2) a^+a^+aa + E(a + a^+); C = sqrt(kappa) a."""
    a = destroy(N)
    ad = _dag(a)
    H = _csr(delta * (ad @ a) + 0.5 * K * (ad @ ad @ a @ a) + E * (a + ad))
    c_ops: list = []
    _keep(kappa, a, c_ops)
    return System("kerr", H, c_ops, dict(N=N, delta=delta, K=K, E=E, kappa=kappa))


def kerr_sweep(count: int = 512, seed: int = 0, n_min: int = 8, n_max: int = 64) -> List[System]:
    """Uneven batch of driven Kerr oscillators.

    One generator for the whole batch; per system, in order:
    N ~ U{n_min..n_max}, delta ~ U[-2, 2], K ~ U[0.05, 0.5], E ~ U[0.1, 2].
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.integers(n_min, n_max + 1))
        delta = float(rng.uniform(-2.0, 2.0))
        K = float(rng.uniform(0.05, 0.5))
        E = float(rng.uniform(0.1, 2.0))
        out.append(kerr_oscillator(N, delta, K, E))
    return out


def kerr_chain(sites: int = 3, N: int = 12, J: float = 1.0, K: float = 0.3, delta: float = 0.0,
               E: float = 0.5, kappa: float = 0.5) -> System:
    """Coupled Kerr cavities, site 1 leftmost in the tensor order (d = N**sites).

    H = sum_i [delta a_i^+a_i + (K/2) a_i^+a_i^+a_i a_i] + J sum_i (a_i^+ a_{i+1} + h.c.)
        + E (a_1 + a_1^+);  C_i = sqrt(kappa) a_i.
    """
    ops = []
    for i in range(sites):
        fac = [identity(N)] * sites
        fac[i] = destroy(N)
        ops.append(tensor(*fac))
    dim = N ** sites
    H = sp.csr_matrix((dim, dim), dtype=np.complex128)
    for i, a in enumerate(ops):
        ad = _dag(a)
        H = H + delta * (ad @ a) + 0.5 * K * (ad @ ad @ a @ a)
    for i in range(sites - 1):
        hop = _dag(ops[i]) @ ops[i + 1]
        H = H + J * (hop + _dag(hop))
    H = _csr(H + E * (ops[0] + _dag(ops[0])))
    c_ops: list = []
    for a in ops:
        _keep(kappa, a, c_ops)
    return System("kerr_chain", H, c_ops, dict(sites=sites, N=N, J=J, K=K, delta=delta, E=E,
                                               kappa=kappa))


def two_level_atom(omega: float = 1.0, gamma: float = 0.5, delta: float = 0.0) -> System:
    """Resonantly driven decaying two-level atom: H = (delta/2) sz + (omega/2) sx,
    C = sqrt(gamma) s-."""
    H = _csr(0.5 * delta * sigma_z() + 0.5 * omega * sigma_x())
    c_ops: list = []
    _keep(gamma, sigma_minus(), c_ops)
    return System("two_level_atom", H, c_ops, dict(omega=omega, gamma=gamma, delta=delta))


def random_system(d: int, n_c: int = 2, density: float = 0.4, seed: int = 0) -> System:
    """A random Hermitian H and random sparse collapse operators (test input).

    Draws in order: H's real part, H's imaginary part, then per operator its
    real and imaginary parts (scipy.sparse.random with the same generator).
    """
    rng = np.random.default_rng(seed)
    hr = sp.random(d, d, density=density, random_state=rng, format="csr")
    hi = sp.random(d, d, density=density, random_state=rng, format="csr")
    h = hr + 1j * hi
    H = _csr(h + h.conj().T)
    c_ops = []
    for _ in range(n_c):
        cr = sp.random(d, d, density=density, random_state=rng, format="csr")
        ci = sp.random(d, d, density=density, random_state=rng, format="csr")
        c_ops.append(_csr(cr + 1j * ci))
    return System("random", H, c_ops, dict(d=d, n_c=n_c, density=density, seed=seed))


# ---------------------------------------------------------------------------
# The three structure examples of the paper's numerical section
# ---------------------------------------------------------------------------

def paper_jc_nonrwa(N: int = 16, delta: float = 0.0, omega_a: float = 1.0, g: float = 0.25,
                    E: float = 1.0, kappa: float = 5e-3, gamma: float = 0.05,
                    n_th: float = 1.0) -> System:
    """Driven Jaynes-Cummings model without the rotating-wave approximation
    (Eq. jc), order s- = s- (x) I, a = I (x) a."""
    sm = tensor(sigma_minus(), identity(N))
    a = tensor(identity(2), destroy(N))
    ad, sp_ = _dag(a), _dag(sm)
    H = _csr(-delta * (ad @ a) + omega_a * (sp_ @ sm) + g * (a + ad) @ (sm + sp_) + E * (a + ad))
    c_ops: list = []
    _keep(kappa * (1.0 + n_th), a, c_ops)
    _keep(kappa * n_th, ad, c_ops)
    _keep(gamma * (1.0 + n_th), sm, c_ops)
    return System("paper_jc_nonrwa", H, c_ops, dict(N=N))


def paper_spin_chain(N: int = 5, delta: float = 0.0, omega: float = 2 * np.pi,
                     J: float = 0.1 * 2 * np.pi, gamma: float = 0.01) -> System:
    """Driven spin chain (Eq. spinchain) with dephasing sqrt(gamma) sz on each
    spin; omega_n = omega, J_x = J_y = J_z = J, Omega = omega_1 / 2."""
    def site(op, n):
        fac = [identity(2)] * N
        fac[n] = op
        return tensor(*fac)

    sx = [site(sigma_x(), n) for n in range(N)]
    sy = [site(sigma_y(), n) for n in range(N)]
    sz = [site(sigma_z(), n) for n in range(N)]
    Omega = omega / 2.0
    H = -0.5 * delta * sz[0] - 0.5 * Omega * sx[0]
    for n in range(1, N):
        H = H - 0.5 * omega * sz[n]
    for n in range(N - 1):
        H = H - 0.5 * (J * sx[n] @ sx[n + 1] + J * sy[n] @ sy[n + 1] + J * sz[n] @ sz[n + 1])
    H = _csr(H)
    c_ops: list = []
    for n in range(N):
        _keep(gamma, sz[n], c_ops)
    return System("paper_spin_chain", H, c_ops, dict(N=N, delta=delta))


def paper_optomechanics(Nc: int = 4, Nm: int = 8, delta: float = 0.0, omega_m: float = 1.0,
                        g0: float = 0.4, E: float = 0.1, kappa: float = 0.3, gamma: float = 1e-4,
                        n_th: float = 1.0) -> System:
    """Optomechanical system of Eq. opto, order a = a (x) I, b = I (x) b."""
    a = tensor(destroy(Nc), identity(Nm))
    b = tensor(identity(Nc), destroy(Nm))
    ad, bd = _dag(a), _dag(b)
    H = _csr(-delta * (ad @ a) + omega_m * (bd @ b) + g0 * (b + bd) @ (ad @ a) + E * (a + ad))
    c_ops: list = []
    _keep(kappa, a, c_ops)
    _keep(gamma * (1.0 + n_th), b, c_ops)
    _keep(gamma * n_th, bd, c_ops)
    return System("paper_optomechanics", H, c_ops, dict(Nc=Nc, Nm=Nm))


def config_systems(name: str, count: int | None = None) -> List[System]:
    """Named workload sets: 'cavity', 'jc', 'opto', 'kerr', 'chain'."""
    if name == "cavity":
        return [driven_cavity(n_th=0.0), driven_cavity(n_th=0.2), thermal_cavity(n_th=0.2)]
    if name == "jc":
        return [jaynes_cummings_rwa(seed=s) for s in range(32 if count is None else count)]
    if name == "opto":
        return [optomechanics(seed=s) for s in range(8 if count is None else count)]
    if name == "kerr":
        return kerr_sweep(512 if count is None else count)
    if name == "chain":
        return [kerr_chain()]
    raise ValueError(f"unknown workload {name!r}")
