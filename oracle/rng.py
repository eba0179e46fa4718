"""Seeded random draws made by the method itself (oracle; test infrastructure only).

The paper uses random initial vectors for regular graphs (Sec. 6.2.1) but does
not say how they are drawn.  The reading taken here: entry (i, j) of the
n x b initial block is 2u - 1 with u the (i*b + j + 1)-th output of a SplitMix64
generator (Steele, Lea, Flood, OOPSLA 2014) whose state starts at
mix(seed + gamma), mapped to [0, 1) by its top 53 bits.  The start vector of the
polynomial preconditioner's Lanczos process (Sec. 5.2) uses the same rule with
state mix(seed + 3 gamma) and counter i + 1, and the reference block that fixes
the rotation of eigenvectors inside a cluster of equal Ritz values (see
sphynx.canonical_rotation) uses state mix(seed + 5 gamma) and counter i*d + j + 1.

This is written from the published generator definition, independently of the
GPU library's copy; the tests check the two agree bit for bit.
"""

from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def mix64(z: int) -> int:
    """SplitMix64 output function on a Python int (exact 64-bit arithmetic)."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * np.uint64(0xBF58476D1CE4E5B9)
        z = z ^ (z >> np.uint64(27))
        z = z * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _stream(state: int, count: int) -> np.ndarray:
    """Outputs 1..count of SplitMix64 started at ``state``, as doubles in [-1, 1)."""
    ctr = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state) + ctr * np.uint64(GAMMA)
    u = (_mix64_np(z) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return 2.0 * u - 1.0


def splitmix64_block(n: int, b: int, seed: int) -> np.ndarray:
    """The n x b random initial block of LOBPCG (row-major)."""
    state = mix64((seed + GAMMA) & MASK)
    return _stream(state, n * b).reshape(n, b)


def reference_block(n: int, d: int, seed: int) -> np.ndarray:
    """The n x d reference block of the embedding's cluster rotation."""
    state = mix64((seed + 5 * GAMMA) & MASK)
    return _stream(state, n * d).reshape(n, d)


def poly_start_vector(n: int, seed: int) -> np.ndarray:
    """Start vector of the Lanczos process that builds the GMRES polynomial."""
    state = mix64((seed + 3 * GAMMA) & MASK)
    return _stream(state, n)
