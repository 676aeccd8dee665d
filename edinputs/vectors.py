"""Counter-based seeded vectors keyed by the state integer.

SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the finaliser constants are those published there)
maps (seed, state) to 64 random bits; the top 53 bits give a uniform double in
[0, 1).  Keying by the state integer rather than the vector index lets the
oracle evaluate a vector entry for any basis state without knowing its index.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
GOLDEN = np.uint64(0x9E3779B97F4A7C15)
C1 = np.uint64(0xBF58476D1CE4E5B9)
C2 = np.uint64(0x94D049BB133111EB)


def splitmix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * C1
        z = (z ^ (z >> np.uint64(27))) * C2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, states: np.ndarray, stream: int = 0) -> np.ndarray:
    """u in [0,1) for each state: splitmix64(splitmix64(seed*2^8 + stream) ^ state) >> 11 * 2^-53."""
    key = splitmix64(np.array([np.uint64(seed) * np.uint64(256) + np.uint64(stream)], dtype=np.uint64))[0]
    h = splitmix64(np.asarray(states, dtype=np.uint64) ^ key)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def state_vector(seed: int, states: np.ndarray, complex_: bool = False) -> np.ndarray:
    """x(state) uniform in [-1, 1) (real, or real + i*imag with independent streams)."""
    re = 2.0 * uniform01(seed, states, 0) - 1.0
    if not complex_:
        return re
    im = 2.0 * uniform01(seed, states, 1) - 1.0
    return re + 1j * im
