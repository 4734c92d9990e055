"""Random permutation parameters (oracle side).

Def. 1 (§II-A) needs an invertible sigma mod N; for N a power of two any odd
integer is invertible (§V-E).  Algorithm 1 draws a set of sigma per dimension.
The draws come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; the
reference C of Vigna's splitmix64.c): the n-th output of the sequence seeded
with ``seed`` is mix(seed + (n + 1) * 0x9E3779B97F4A7C15 mod 2^64).  The draw
for loop l and dimension d is output number l * D + d, reduced to an odd value
in [N_d] by (z mod N_d) | 1, which is uniform over the odd residues.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def splitmix64_at(seed: int, n: int) -> int:
    """The n-th (0-based) output of SplitMix64 started from state ``seed``."""
    return _mix((seed + (n + 1) * _GAMMA) & _MASK)


def splitmix64(seed: int, count: int) -> list:
    """The first ``count`` outputs of SplitMix64 started from state ``seed``."""
    return [splitmix64_at(seed, i) for i in range(count)]


def draw_sigmas(seed: int, loops: int, n: tuple) -> np.ndarray:
    """sigma[l, d]: odd, uniform in [N_d] (Def. 1; §V-E: any odd integer)."""
    d = len(n)
    out = np.zeros((loops, d), dtype=np.int64)
    for l in range(loops):
        for dd in range(d):
            z = splitmix64_at(seed, l * d + dd)
            out[l, dd] = (z % int(n[dd])) | 1
    return out


def inverse_mod(sigma: int, n: int) -> int:
    """sigma^{-1} with sigma sigma^{-1} = 1 mod N (eq. (mod_inv))."""
    return pow(int(sigma), -1, int(n))
