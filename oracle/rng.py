"""Counter-based start vector for the inverse-power method (oracle; test
infrastructure only).

The shifted-inverse power iteration starts from a random vector (section
"Eigenvalue Methods"). So that the CUDA path and the oracle start from the
same vector, both evaluate SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) at counter values:
element k of the start vector is
    re = u(2k), im = u(2k + 1),   u(c) = 2 * (splitmix64(seed + (c + 1) * G) >> 11) * 2^-53 - 1,
with G = 0x9E3779B97F4A7C15 and all arithmetic modulo 2^64, so each part is
uniform on [-1, 1).
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(z: int) -> int:
    """The SplitMix64 output function applied to state z."""
    z &= _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def start_vector(n: int, seed: int) -> np.ndarray:
    """Complex vector of length n, parts uniform on [-1, 1), from counters."""
    c = np.arange(1, 2 * n + 1, dtype=np.uint64)            # counters c + 1
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + c * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = 2.0 * ((z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53) - 1.0
    return u[0::2] + 1j * u[1::2]
