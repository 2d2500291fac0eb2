"""Philox4x64-10 counter-based generator and the Rademacher sketch signs.

Oracle; test infrastructure only.  Philox4x64-10 follows its published
definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11): four 64-bit counter words, two key words, ten
rounds; round r uses the key bumped r times by the Weyl constants.  The
output stream is the one of numpy.random.Philox with key = seed +
(problem_id << 64): block b is the round function of counter (b+1, 0, 0, 0)
and emits its four words in order.  Rademacher sign e (a set bit meaning
-1) is bit e % 64 of stream word e // 64.
"""
from __future__ import annotations

from typing import List

import numpy as np

_MASK = (1 << 64) - 1
_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B


def philox4x64_10(ctr, key):
    """Ten Philox4x64 rounds on counter ``ctr`` (4 words) with ``key`` (2 words)."""
    x0, x1, x2, x3 = (int(c) & _MASK for c in ctr)
    k0, k1 = (int(k) & _MASK for k in key)
    for _ in range(10):
        p0 = _M0 * x0
        p1 = _M1 * x2
        hi0, lo0 = p0 >> 64, p0 & _MASK
        hi1, lo1 = p1 >> 64, p1 & _MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return x0, x1, x2, x3


def philox_words(seed: int, problem_id: int, n_words: int) -> List[int]:
    """First ``n_words`` 64-bit outputs of the stream keyed (seed, problem_id)."""
    out: List[int] = []
    b = 0
    while len(out) < n_words:
        out.extend(philox4x64_10((b + 1, 0, 0, 0), (seed, problem_id)))
        b += 1
    return out[:n_words]


def rademacher_signs(seed: int, problem_id: int, n: int) -> np.ndarray:
    """n signs in {+1, -1}: sign e is -1 iff bit e % 64 of word e // 64 is set."""
    words = philox_words(seed, problem_id, (n + 63) // 64)
    out = np.empty(n, dtype=np.float64)
    for e in range(n):
        out[e] = -1.0 if (words[e // 64] >> (e % 64)) & 1 else 1.0
    return out
