"""SplitMix64 counter-based generator -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper initialises each new mode without saying how ("Initialize u_x, u_y", Section
3.3).  The reading used here: a mode that has a counterpart in the previous step's
solution starts from it; any other mode starts from pseudo-random entries in [0.5, 1.5)
drawn by SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) keyed by (seed, step, mode, dimension, node).  This module and
the CUDA path each implement the published SplitMix64 finaliser independently.
"""
from __future__ import annotations

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def mix64(x: int) -> int:
    """The SplitMix64 output function applied to ``x + golden gamma`` (mod 2^64)."""
    z = (x + GOLDEN) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def mode_init_value(seed: int, step: int, mode: int, dim: int, node: int) -> float:
    """Entry ``node`` of the random start vector of ``mode`` in ``dim`` at time ``step``.

    Chained key: ``h = mix(mix(mix(mix(seed) ^ step) ^ (4 mode + dim)) ^ node)``; the top 53
    bits give ``u in [0, 1)`` and the value is ``0.5 + u``.
    """
    h = mix64(seed & MASK)
    h = mix64(h ^ (step & MASK))
    h = mix64(h ^ ((4 * mode + dim) & MASK))
    h = mix64(h ^ (node & MASK))
    return 0.5 + (h >> 11) * (1.0 / (1 << 53))


def mode_init_vector(seed: int, step: int, mode: int, dim: int, n: int):
    import numpy as np
    return np.array([mode_init_value(seed, step, mode, dim, i) for i in range(n)])
