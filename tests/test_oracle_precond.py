"""Pins of the oracle's many-body basis orbitals and block-diagonal LOBPCG
preconditioner (Sec. 2) against counting, linear algebra and interlacing,
not against the oracle itself."""

from collections import Counter

import numpy as np
import pytest

import oracle
import synth
from helpers import inputs, oracle_problem

P = oracle.precond


def _groups(inp):
    o = oracle_problem(inp)
    occ_p, occ_n = o.species(0)["occ"], o.species(1)["occ"]
    blk, nb = P.orbital_blocks(occ_p, occ_n, o.p_idx, o.n_idx, synth.sp_orbitals(inp["sp"]))
    return o, blk, nb


def _mpoly(twoj, k):
    """{2M: number of k-particle subsets of the 2j+1 substates of one
    orbital with that total 2M} (generating function prod_m (1 + y x^2m))."""
    poly = {(0, 0): 1}
    for m in range(-twoj, twoj + 1, 2):
        nxt = Counter(poly)
        for (c, M), w in poly.items():
            nxt[(c + 1, M + m)] += w
        poly = nxt
    return {M: w for (c, M), w in poly.items() if c == k}


def _conv(a, b):
    out = Counter()
    for x, u in a.items():
        for y, v in b.items():
            out[x + y] += u * v
    return out


def _species_occupations(sp, A, nmax):
    """Every way to put A particles into the orbitals of sp (capacities
    2j+1): ({orbital: count}, excess quanta q, {2M: substate count})."""
    orbs = sorted({(int(n), int(l), int(j)) for n, l, j in zip(sp["N"], sp["l"], sp["twoj"])})
    cap = [j + 1 for (_, _, j) in orbs]
    shells = [n for (n, _, _) in orbs]
    q0 = sum(sorted(np.asarray(sp["N"]).tolist())[:A])
    out = []

    def rec(i, left, cnt):
        if i == len(orbs):
            if left == 0:
                q = sum(c * shells[t] for t, c in enumerate(cnt)) - q0
                if nmax < 0 or q <= nmax:
                    dist = {0: 1}
                    for t, c in enumerate(cnt):
                        if c:
                            dist = _conv(dist, _mpoly(orbs[t][2], c))
                    out.append((tuple(cnt), q, dict(dist)))
            return
        for c in range(min(cap[i], left) + 1):
            rec(i + 1, left - c, cnt + [c])

    rec(0, A, [])
    return out


@pytest.mark.parametrize("case", [(2, 2, 3, 2, 1), (2, 3, 3, -1, 0), (3, 2, 2, 3, 0), (2, 4, 1, 2, 3)])
def test_orbital_group_sizes_from_generating_functions(case):
    """The number of groups and their sizes follow from placing particles
    into orbitals and counting substates with total 2M, computed without
    enumerating determinants."""
    n_shell, Z, N, nmax, twoM = case
    inp = inputs(n_shell, Z, N, nmax, seed=1, twoM=twoM)
    o, blk, nb = _groups(inp)
    sizes = sorted(np.bincount(blk, minlength=nb).tolist())
    pred = []
    for cp, qp, dp in _species_occupations(inp["sp"], Z, nmax):
        for cn, qn, dn in _species_occupations(inp["sp"], N, nmax):
            if nmax >= 0 and qp + qn > nmax:
                continue
            s = sum(w * dn.get(twoM - M, 0) for M, w in dp.items())
            if s:
                pred.append(s)
    assert nb == len(pred) and sizes == sorted(pred)
    assert blk.min() == 0 and blk.max() == nb - 1
    first = [int(np.nonzero(blk == g)[0][0]) for g in range(nb)]
    assert first == sorted(first)            # numbered by first appearance


def test_orbital_groups_share_excess_quanta_and_label_extremes():
    inp = inputs(2, 2, 3, 2, seed=1, twoM=1)
    o, blk, nb = _groups(inp)
    q = o.species(0)["q"][o.p_idx] + o.species(1)["q"][o.n_idx]
    for g in range(nb):
        assert len(set(q[blk == g].tolist())) == 1
    occ_p, occ_n = o.species(0)["occ"], o.species(1)["occ"]
    S = len(inp["sp"]["N"])
    b1, n1 = P.orbital_blocks(occ_p, occ_n, o.p_idx, o.n_idx, np.arange(S))
    assert n1 == o.dim and np.array_equal(b1, np.arange(o.dim))
    b0, n0 = P.orbital_blocks(occ_p, occ_n, o.p_idx, o.n_idx, np.zeros(S, np.int32))
    assert n0 == 1 and np.all(b0 == 0)


def test_sub_block_split_rule():
    for c, want in [(1, [1]), (128, [128]), (129, [65, 64]), (257, [86, 86, 85]), (300, [100, 100, 100])]:
        block = np.zeros(c, np.int32)
        assert [len(r) for r in P.sub_blocks(block, 1)] == want
    block = np.array([1, 0, 1, 2, 0, 1], np.int32)
    subs = P.sub_blocks(block, 4)                 # group 3 is empty
    assert [r.tolist() for r in subs] == [[1, 4], [0, 2, 5], [3]]


def _csr(inp):
    o = oracle_problem(inp)
    rp, col, val, _ = o.csr()
    return o, rp, col, val, oracle.dense_from_csr(rp, col, val, o.dim)


def test_single_block_is_the_shifted_inverse():
    """One group of at most 128 rows: T = (H - sigma I)^-1, checked by
    multiplying back with the full H."""
    inp = inputs(1, 2, 1, -1, seed=3, dtype=np.float64)
    o, rp, col, val, H = _csr(inp)
    assert 1 < o.dim <= P.SUB_MAX
    sigma = np.linalg.eigvalsh(H)[0] - 1.0
    R = np.random.default_rng(0).standard_normal((o.dim, 3))
    W, shift, _ = P.block_precond(rp, col, val, np.zeros(o.dim, np.int32), 1, sigma, R)
    assert np.all(shift == sigma)
    assert np.allclose((H - sigma * np.eye(o.dim)) @ W, R, atol=1e-9)


def test_large_group_is_cut_into_two_inverses():
    """One group of 190 rows: two sub-blocks of 95, each the inverse of its
    own diagonal block of H - sigma I (the coupling between them dropped)."""
    inp = inputs(1, 2, 2, -1, seed=3, dtype=np.float64)
    o, rp, col, val, H = _csr(inp)
    assert o.dim == 190
    sigma = np.linalg.eigvalsh(H)[0] - 1.0
    R = np.random.default_rng(0).standard_normal((o.dim, 2))
    W, shift, _ = P.block_precond(rp, col, val, np.zeros(o.dim, np.int32), 1, sigma, R)
    for sl in (slice(0, 95), slice(95, 190)):
        Hs = H[sl, sl] - sigma * np.eye(95)
        assert np.allclose(Hs @ W[sl], R[sl], atol=1e-9)
    assert not np.allclose((H - sigma * np.eye(o.dim)) @ W, R, atol=1e-6)


def test_one_row_blocks_reduce_to_the_diagonal():
    """Every row its own group: T = diag(1 / (H_ii - sigma_i)) with
    sigma_i = sigma where H_ii > sigma, else H_ii - 1e-3 max(|H_ii|, |sigma|)."""
    inp = inputs(2, 2, 1, 2, seed=4, dtype=np.float64)
    o, rp, col, val, H = _csr(inp)
    d = np.diag(H)
    sigma = float(np.median(d))
    R = np.random.default_rng(1).standard_normal((o.dim, 2))
    W, shift, _ = P.block_precond(rp, col, val, np.arange(o.dim, dtype=np.int32), o.dim, sigma, R)
    want = np.where(d > sigma, sigma, d - 1e-3 * np.maximum(np.abs(d), abs(sigma)))
    assert np.allclose(shift, want, rtol=0, atol=1e-12)
    assert np.allclose(W, R / (d - want)[:, None], rtol=1e-12)


def test_preconditioner_is_spd_and_block_local():
    inp = inputs(2, 2, 3, 2, seed=5, dtype=np.float64, twoM=1)
    o, blk, nb = _groups(inp)
    _, rp, col, val, H = _csr(inp)
    sigma = float(np.median(np.diag(H)))         # inside the spectrum: some blocks need the fallback
    T, shift, _ = P.block_precond(rp, col, val, blk, nb, sigma, np.eye(o.dim))
    assert np.allclose(T, T.T, atol=1e-10)
    assert np.linalg.eigvalsh(0.5 * (T + T.T))[0] > 0
    assert np.all(T[blk[:, None] != blk[None, :]] == 0)
    assert np.any(shift < sigma) and np.any(shift == sigma)
    assert np.all(shift <= sigma)


def test_shift_below_the_spectrum_needs_no_fallback():
    """Cauchy interlacing: every principal submatrix has its lowest
    eigenvalue >= lambda_min(H), so sigma < lambda_min(H) keeps every
    shifted block positive definite."""
    inp = inputs(2, 3, 2, 3, seed=6, dtype=np.float64, twoM=1)
    o, blk, nb = _groups(inp)
    _, rp, col, val, H = _csr(inp)
    sigma = np.linalg.eigvalsh(H)[0] - 1e-3
    _, shift, _ = P.block_precond(rp, col, val, blk, nb, sigma, np.ones((o.dim, 1)))
    assert np.all(shift == sigma)
