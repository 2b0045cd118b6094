"""H by brute-force second quantisation on tiny spaces.  Test infrastructure.

Independent of ``ci_oracle.c``: the determinants come from
``itertools.combinations``, the fermion phase of every operator comes from
moving it to its place in the ordered string of creators, and every term of

    H = sum_a eps_a a+_a a_a  (both species)
      + 1/4 sum_abcd V^pp_abcd a+_a a+_b a_d a_c  (and nn)
      + sum_abcd V^pn_abcd a+_{a,p} a+_{b,n} a_{d,n} a_{c,p}

is applied literally.  A determinant is the sorted tuple of its occupied
modes, mode = species * S + state (protons are species 0), i.e. the state
prod_{modes ascending} a+_mode |0>.
"""

import itertools

import numpy as np


def _apply(op, state):
    """Apply one operator ('c' create / 'a' annihilate, mode) to a state."""
    kind, mode = op
    if kind == "a":
        if mode not in state:
            return 0, None
        k = state.index(mode)
        return (-1) ** k, state[:k] + state[k + 1:]
    if mode in state:
        return 0, None
    k = sum(1 for x in state if x < mode)
    return (-1) ** k, state[:k] + (mode,) + state[k:]


def apply_string(ops, state):
    """Apply an operator product written left to right (rightmost acts first)."""
    sign = 1
    for op in reversed(ops):
        s, state = _apply(op, state)
        if s == 0:
            return 0, None
        sign *= s
    return sign, state


def species_dets(sp_N, A, nmax):
    """All A-subsets of the states with excess quanta q <= nmax (nmax < 0: all)."""
    S = len(sp_N)
    nmin = sum(sorted(int(x) for x in sp_N)[:A])
    out = []
    for occ in itertools.combinations(range(S), A):
        q = sum(int(sp_N[o]) for o in occ) - nmin
        if nmax < 0 or q <= nmax:
            out.append((occ, q))
    return out


def basis(sp, Z, N, nmax, twoM):
    """Basis states as sorted mode tuples (protons: mode = state, neutrons:
    mode = S + state), with total 2M = twoM and q_p + q_n <= nmax."""
    S = len(sp["N"])
    tw = [int(x) for x in sp["twom"]]
    out = []
    for po, pq in species_dets(sp["N"], Z, nmax):
        for no, nq in species_dets(sp["N"], N, nmax):
            if sum(tw[o] for o in po) + sum(tw[o] for o in no) != twoM:
                continue
            if nmax >= 0 and pq + nq > nmax:
                continue
            out.append(tuple(po) + tuple(S + o for o in no))
    return out


def _terms(S, eps, V, state):
    """The terms of H whose annihilators all hit occupied modes of state."""
    occ_p = [m for m in state if m < S]
    occ_n = [m for m in state if m >= S]
    Vpp = V["pp"].reshape(S, S, S, S)
    Vnn = V["nn"].reshape(S, S, S, S)
    Vpn = V["pn"].reshape(S, S, S, S)
    for m in state:  # one-body
        yield float(eps[m % S]), (("c", m), ("a", m))
    for occ, T, off in ((occ_p, Vpp, 0), (occ_n, Vnn, S)):
        for c in occ:
            for d in occ:
                for a in range(S):
                    for b in range(S):
                        v = T[a, b, c - off, d - off]
                        if v != 0.0:
                            yield 0.25 * float(v), (("c", off + a), ("c", off + b),
                                                     ("a", d), ("a", c))
    for c in occ_p:
        for d in occ_n:
            for a in range(S):
                for b in range(S):
                    v = Vpn[a, b, c, d - S]
                    if v != 0.0:
                        yield float(v), (("c", a), ("c", S + b), ("a", d), ("a", c))


def hamiltonian(sp, Z, N, nmax, twoM, eps, tables):
    """Dense H over ``basis(...)`` (same order).  Returns (states, H)."""
    S = len(sp["N"])
    V = {k: np.asarray(tables[k], dtype=np.float64) for k in ("pp", "nn", "pn")}
    states = basis(sp, Z, N, nmax, twoM)
    index = {s: i for i, s in enumerate(states)}
    H = np.zeros((len(states), len(states)))
    for j, ket in enumerate(states):
        for coef, ops in _terms(S, eps, V, ket):
            sign, out = apply_string(ops, ket)
            if sign == 0:
                continue
            i = index.get(out)
            if i is None:
                # outside the Nmax cut: H is projected onto the basis; a
                # change of 2M would be a broken interaction table
                tw = [int(x) for x in sp["twom"]]
                if sum(tw[m % S] for m in out) != twoM:
                    raise AssertionError("H changed the total 2M")
                continue
            H[i, j] += sign * coef
    return states, H
