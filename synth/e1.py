"""Inputs of the paper's nonzero-count benchmark (Sec. 2.1, Figs. 3-4).

A state is N occupied single-particle states out of S, stored in the MBS
form of Sec. 2.1: the ascending tuple of occupied state indices (uint16).
The paper draws its random states biased towards the lowest states but does
not give the law.  Here every particle's state is k = floor(log(u) / log(r))
for a SplitMix64 uniform u (a geometric law, P(k) proportional to r**k),
redrawn when k >= S or when k is already occupied.  With N = 8, S = 128 and
r = 0.972 the fraction of off-diagonal pairs that differ in at most four
states is about 6e-6, the median density quoted for the 8-particle runs.
"""

import numpy as np

from .tbme import splitmix64_mix

E1_RATIO = 0.972
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _uniforms(seed, rows, cols, col0):
    """uniforms u[i, j] in (0, 1) at counter (i, col0 + j) of the seed."""
    i = np.arange(rows, dtype=np.uint64)[:, None]
    j = np.arange(col0, col0 + cols, dtype=np.uint64)[None, :]
    pos = (i << np.uint64(20)) + j + np.uint64(1)
    with np.errstate(over="ignore"):
        z = splitmix64_mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + pos * _GAMMA)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


def e1_states(n, N=8, S=128, r=E1_RATIO, seed=0):
    """n random N-particle states over S <= 128 states, uint16 [n][N]."""
    if not (0 < N <= S <= 128):
        raise ValueError("need 0 < N <= S <= 128")
    mask = np.zeros((n, 2), np.uint64)
    filled = np.zeros(n, np.int64)
    col = 0
    while n and filled.min() < N:
        u = _uniforms(seed, n, 64, col)
        k = np.floor(np.log(u) / np.log(r)).astype(np.int64)
        for j in range(64):
            kj = k[:, j]
            ok = (kj < S) & (filled < N)
            w = np.where(kj >= 64, 1, 0)
            b = np.uint64(1) << (np.clip(kj, 0, 127) % 64).astype(np.uint64)
            cur = mask[np.arange(n), w]
            ok &= (cur & b) == 0
            mask[np.arange(n)[ok], w[ok]] |= b[ok]
            filled += ok
        col += 64
    bits = np.zeros((n, 128), bool)
    for w in range(2):
        for b in range(64):
            bits[:, 64 * w + b] = (mask[:, w] >> np.uint64(b)) & np.uint64(1) == 1
    _, cols = np.nonzero(bits)
    return cols.reshape(n, N).astype(np.uint16)
