"""Seeded two-body matrix elements (TBMEs) from a counter-based generator.

The Hamiltonian's two-body part is given by three flat tables indexed
``((a*S + b)*S + c)*S + d`` (S = number of s.p. states per species):

* ``pp`` and ``nn``: antisymmetrised like-particle elements <ab|V|cd>_A with
  V_abcd = -V_bacd = -V_abdc = V_badc, and V = 0 when a == b or c == d;
* ``pn``: proton-neutron elements <a_p b_n|V|c_p d_n> (distinguishable
  particles, no antisymmetrisation; a, c are proton states, b, d neutron);

all real, Hermitian (V_abcd = V_cdab) and zero unless m_a + m_b = m_c + m_d.

Each independent element is one draw g(seed, channel, P, Q) on the canonical
pair of pair-indices P <= Q:

* like pairs a < b have index P = b(b-1)/2 + a; pn pairs (a, b) have
  P = a*S + b (S <= 256, so P < 2**16);
* the counter is c = (channel << 32) | (P << 16) | Q;
* twelve SplitMix64 outputs (Steele, Lea and Flood, OOPSLA 2014) are taken at
  stream positions 12c + 1 ... 12c + 12, i.e. z_k = mix(seed + (12c+k+1)*gamma)
  mod 2**64 with gamma = 0x9E3779B97F4A7C15;
* g = sum_k (z_k >> 32) * 2**-32 - 6, the Irwin-Hall approximation of a
  standard normal (mean 0, variance 1).  Every partial sum fits in 36 bits,
  so g is exact in binary64 whatever the summation order, and the float32
  table (round-to-nearest of g) is the same on every machine.
"""

import numpy as np

CH_PP, CH_NN, CH_PN = 0, 1, 2

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z):
    """SplitMix64 output function on a uint64 array (arithmetic mod 2**64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def tbme_gaussian(seed, channel, P, Q):
    """Draw g(seed, channel, P, Q) for arrays P <= Q (see module docstring)."""
    P = np.asarray(P, dtype=np.uint64)
    Q = np.asarray(Q, dtype=np.uint64)
    counter = (np.uint64(channel) << np.uint64(32)) | (P << np.uint64(16)) | Q
    s = np.zeros(counter.shape, dtype=np.float64)
    seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        base = counter * np.uint64(12)
        for k in range(12):
            z = splitmix64_mix(seed + (base + np.uint64(k + 1)) * _GAMMA)
            s += (z >> np.uint64(32)).astype(np.float64) * 2.0 ** -32
    return s - 6.0


def _pairs_by_m(twom, like):
    """Group pair indices by pair 2M; returns {2M: (a, b, P)} arrays."""
    S = len(twom)
    groups = {}
    for a in range(S):
        for b in range(S):
            if like and not a < b:
                continue
            P = b * (b - 1) // 2 + a if like else a * S + b
            groups.setdefault(int(twom[a] + twom[b]), []).append((a, b, P))
    return {k: np.array(v, dtype=np.int64) for k, v in groups.items()}


def _fill_channel(V, S, groups, seed, channel, like):
    for _, arr in sorted(groups.items()):
        n = len(arr)
        i, j = np.triu_indices(n)  # canonical P <= Q (pairs sorted by P)
        order = np.argsort(arr[:, 2], kind="stable")
        arr = arr[order]
        a, b, P = arr[i, 0], arr[i, 1], arr[i, 2]
        c, d, Q = arr[j, 0], arr[j, 1], arr[j, 2]
        g = tbme_gaussian(seed, channel, P, Q)
        def put(w, x, y, z, val):
            V[((w * S + x) * S + y) * S + z] = val
        for (w, x, y, z) in ((a, b, c, d), (c, d, a, b)):
            put(w, x, y, z, g)
            if like:
                put(x, w, y, z, -g)
                put(w, x, z, y, -g)
                put(x, w, z, y, g)


def tbme_tables(sp, seed, dtype=np.float32):
    """Return {'pp', 'nn', 'pn'} flat TBME tables of length S**4.

    ``dtype`` float32 gives the round-to-nearest of the exact binary64 draws;
    float64 gives the draws themselves.
    """
    twom = np.asarray(sp["twom"])
    S = len(twom)
    if S > 256:
        raise ValueError("at most 256 s.p. states per species")
    out = {}
    like_groups = _pairs_by_m(twom, like=True)
    pn_groups = _pairs_by_m(twom, like=False)
    for name, ch, like, groups in (("pp", CH_PP, True, like_groups),
                                   ("nn", CH_NN, True, like_groups),
                                   ("pn", CH_PN, False, pn_groups)):
        V = np.zeros(S ** 4, dtype=np.float64)
        _fill_channel(V, S, groups, seed, ch, like)
        out[name] = V.astype(dtype)
    return out


def tbme_tables_zero(S, dtype=np.float32):
    """All-zero tables (the one-body-only Hamiltonian)."""
    return {k: np.zeros(S ** 4, dtype=dtype) for k in ("pp", "nn", "pn")}
