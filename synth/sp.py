"""Harmonic-oscillator single-particle table, the alphabet of the bit strings.

A determinant is a bit string with one bit per s.p. state (Sec. 2.1); the
states carry the quantum numbers (n, l, j, m) the paper groups determinants
by (Sec. 2).  The paper does not fix their order; this package reads it as

    N ascending, then l descending, then j = l + 1/2 before j = l - 1/2,
    then m ascending,

with N = 2n + l the HO shell.  Shell N holds (N + 1)(N + 2) states, so shells
0..1 give 8 states, 0..3 give 40 and 0..4 give 70.  The order fixes the
fermion signs, so it is part of the interface.
"""

import numpy as np


def ho_sp_table(n_shell_max):
    """Return the s.p. table of HO shells 0..n_shell_max.

    Returns a dict of int32 arrays ``N``, ``l``, ``twoj``, ``twom`` (the last
    two are 2j and 2m), all of length S.
    """
    if n_shell_max < 0:
        raise ValueError("n_shell_max must be >= 0")
    rows = []
    for N in range(n_shell_max + 1):
        for l in range(N, -1, -2):
            js = [2 * l + 1, 2 * l - 1] if l > 0 else [1]
            for twoj in js:
                for twom in range(-twoj, twoj + 1, 2):
                    rows.append((N, l, twoj, twom))
    a = np.array(rows, dtype=np.int32)
    return {"N": a[:, 0].copy(), "l": a[:, 1].copy(),
            "twoj": a[:, 2].copy(), "twom": a[:, 3].copy()}


def sp_orbitals(sp):
    """Orbital label of every s.p. state: states with the same (N, l, 2j)
    (one orbital, differing only in 2m) share a label, numbered 0, 1, ... in
    table order."""
    ids = {}
    return np.array([ids.setdefault((int(N), int(l), int(j)), len(ids))
                     for N, l, j in zip(sp["N"], sp["l"], sp["twoj"])], dtype=np.int32)


def sp_energies(sp, hbar_omega):
    """One-body energies eps_a = hbar_omega * (N_a + 3/2) of the HO basis.

    These are inputs of the Hamiltonian (its one-body term), as float64.
    """
    return hbar_omega * (sp["N"].astype(np.float64) + 1.5)

