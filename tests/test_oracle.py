"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: brute-force
second quantisation, itertools enumeration, bit-string popcounts, closed
forms of special cases, invariants, and library routines on special cases.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import brute


def _problem(n_shell, Z, N, nmax, seed=0, dtype=np.float64, zero=False, twoM=None):
    sp = synth.ho_sp_table(n_shell)
    eps = synth.sp_energies(sp, 20.0)
    S = len(sp["N"])
    T = synth.tbme_tables_zero(S, dtype) if zero else synth.tbme_tables(sp, seed, dtype)
    if twoM is None:
        twoM = (Z + N) % 2
    return sp, eps, T, oracle.OracleProblem(sp, Z, N, nmax, twoM, eps, T)


def _states_of(o):
    P, Nn = o.species(0)["occ"], o.species(1)["occ"]
    S = o.S
    return [tuple(int(x) for x in P[o.p_idx[i]]) + tuple(S + int(x) for x in Nn[o.n_idx[i]])
            for i in range(o.dim)]


# ---------------------------------------------------------------- inputs

def test_sp_table_shells():
    """HO shell N holds (N+1)(N+2) states; order N asc, l desc, j=l+1/2 first, m asc."""
    for nsh, total in ((1, 8), (3, 40), (4, 70)):
        sp = synth.ho_sp_table(nsh)
        assert len(sp["N"]) == total
        for N in range(nsh + 1):
            assert int((sp["N"] == N).sum()) == (N + 1) * (N + 2)
    sp = synth.ho_sp_table(1)
    assert list(zip(sp["l"], sp["twoj"], sp["twom"])) == [
        (0, 1, -1), (0, 1, 1), (1, 3, -3), (1, 3, -1), (1, 3, 1), (1, 3, 3), (1, 1, -1), (1, 1, 1)]
    assert np.allclose(synth.sp_energies(sp, 20.0), [30, 30, 50, 50, 50, 50, 50, 50])


def _splitmix64_python(seed, n):
    """SplitMix64 with Python integers (Steele et al. 2014), first n outputs."""
    out, x, mask = [], seed, (1 << 64) - 1
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & mask
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_matches_reference_sequence():
    # first output of SplitMix64 from state 0 is the published 0xE220A8397B1DCDAF
    ref = _splitmix64_python(0, 3)
    assert ref[0] == 0xE220A8397B1DCDAF
    gamma = 0x9E3779B97F4A7C15
    for seed in (0, 1, 12345, (1 << 64) - 1):
        ref = _splitmix64_python(seed, 5)
        pos = np.array([(seed + (i + 1) * gamma) & ((1 << 64) - 1) for i in range(5)], dtype=np.uint64)
        assert [int(z) for z in synth.splitmix64_mix(pos)] == ref


def test_tbme_symmetries_and_exactness():
    sp = synth.ho_sp_table(2)
    S = len(sp["N"])
    T = synth.tbme_tables(sp, 11, np.float64)
    m = sp["twom"]
    for name in ("pp", "nn"):
        V = T[name].reshape(S, S, S, S)
        assert np.array_equal(V, -V.transpose(1, 0, 2, 3))
        assert np.array_equal(V, -V.transpose(0, 1, 3, 2))
        assert np.array_equal(V, V.transpose(2, 3, 0, 1))
        for a in range(S):
            assert not V[a, a].any() and not V[:, :, a, a].any()
    V = T["pn"].reshape(S, S, S, S)
    assert np.array_equal(V, V.transpose(2, 3, 0, 1))
    for name in ("pp", "nn", "pn"):
        V = T[name].reshape(S, S, S, S)
        a, b, c, d = np.nonzero(V)
        assert np.all(m[a] + m[b] == m[c] + m[d])
        # every draw is a multiple of 2**-32 inside (-6, 6): exact in binary64
        x = V[a, b, c, d] * 2.0 ** 32
        assert np.all(x == np.round(x)) and np.all(np.abs(V) < 6)
    assert not np.array_equal(T["pp"], T["nn"])
    T32 = synth.tbme_tables(sp, 11, np.float32)
    assert np.array_equal(T32["pn"], T["pn"].astype(np.float32))


def test_tbme_draw_moments():
    """Irwin-Hall(12) - 6: mean 0, variance 1, |g| < 6."""
    P = np.arange(20000) % 5000
    Q = np.arange(20000) // 5000 + 5000
    g = synth.tbme_gaussian(5, synth.CH_PN, P, Q)
    assert abs(g.mean()) < 0.03 and abs(g.var() - 1) < 0.05
    # matches the definition evaluated with Python integers
    counter = (2 << 32) | (int(P[7]) << 16) | int(Q[7])
    gamma, mask = 0x9E3779B97F4A7C15, (1 << 64) - 1
    s = 0
    for k in range(12):
        x = (5 + (12 * counter + k + 1) * gamma) & mask
        z = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        s += z >> 32
    assert g[7] == s / 2.0 ** 32 - 6


# ---------------------------------------------------------------- basis

@pytest.mark.parametrize("nsh,A,nmax", [(1, 4, -1), (1, 3, 1), (2, 3, 2), (3, 2, 2), (2, 0, -1), (3, 4, 0)])
def test_species_lists_match_itertools(nsh, A, nmax):
    sp, eps, T, o = _problem(nsh, A, 2, nmax, zero=True)
    ref = brute.species_dets(sp["N"], A, nmax)
    got = o.species(0)
    assert len(ref) == len(got["occ"])
    tw = sp["twom"]
    keys = []
    for occ, q in ref:
        bits = sum(1 << o_ for o_ in occ)
        keys.append((int(sum(tw[list(occ)])), q, bits, occ))
    keys.sort()
    for i, (m, q, bits, occ) in enumerate(keys):
        assert tuple(int(x) for x in got["occ"][i]) == occ
        assert got["q"][i] == q and got["twoM"][i] == m
        assert sum(int(w) << (64 * k) for k, w in enumerate(got["bits"][i])) == bits


def _dim_by_histograms(sp, Z, N, nmax, twoM):
    hp, hn = {}, {}
    tw = sp["twom"]
    for h, A in ((hp, Z), (hn, N)):
        for occ, q in brute.species_dets(sp["N"], A, nmax):
            key = (int(sum(tw[list(occ)])), q)
            h[key] = h.get(key, 0) + 1
    dim = 0
    for (mp, qp), cp in hp.items():
        for (mn, qn), cn in hn.items():
            if mp + mn == twoM and (nmax < 0 or qp + qn <= nmax):
                dim += cp * cn
    return dim


def test_basis_dimensions():
    sp, eps, T, o = _problem(1, 4, 4, -1, zero=True)
    assert o.dim == 1014 == _dim_by_histograms(sp, 4, 4, -1, 0)
    assert math.comb(8, 4) ** 2 == 4900 > o.dim
    sp = synth.ho_sp_table(4)
    o1 = oracle.OracleProblem(sp, 4, 4, 4, 0, synth.sp_energies(sp, 20.0), synth.tbme_tables_zero(70))
    assert o1.dim == _dim_by_histograms(sp, 4, 4, 4, 0) == 172684
    assert len(o1.species(0)["occ"]) == 8900


def test_basis_order_and_quantum_numbers():
    sp, eps, T, o = _problem(2, 3, 3, 2, zero=True)
    Ps, Ns = o.species(0), o.species(1)
    assert np.all(np.diff(o.p_idx) >= 0)
    for i in range(1, o.dim):
        if o.p_idx[i] == o.p_idx[i - 1]:
            assert o.n_idx[i] > o.n_idx[i - 1]
    assert np.all(Ps["twoM"][o.p_idx] + Ns["twoM"][o.n_idx] == 0)
    assert np.all(Ps["q"][o.p_idx] + Ns["q"][o.n_idx] <= 2)
    assert sorted(_states_of(o)) == sorted(brute.basis(sp, 3, 3, 2, 0))


# ---------------------------------------------------------------- pattern

def test_difference_equals_popcount_of_xor():
    sp, eps, T, o = _problem(3, 4, 2, 3, zero=True)
    s = o.species(0)
    rng = np.random.default_rng(0)
    n = len(s["occ"])
    for _ in range(500):
        a, b = rng.integers(0, n, 2)
        x = s["bits"][a] ^ s["bits"][b]
        pc = sum(bin(int(w)).count("1") for w in x)
        d = o.count_difference(0, int(a), int(b))
        assert d == pc and d % 2 == 0


def test_pattern_config0_dense_brute_force():
    """nnz of the 4p+4n N<=1 space: all pairs within 4 differences."""
    sp, eps, T, o = _problem(1, 4, 4, -1, seed=0)
    states = [frozenset(s) for s in _states_of(o)]
    rp, cols, vals, ab = o.csr()
    nnz_by_d = [0, 0, 0, 0, 0]
    for i in range(o.dim):
        ref = [j for j in range(o.dim) if len(states[i] ^ states[j]) <= 4]
        assert list(cols[rp[i]:rp[i + 1]]) == ref
        for j in ref:
            nnz_by_d[len(states[i] ^ states[j])] += 1
    assert rp[-1] == 88462
    assert nnz_by_d == [1014, 0, 7056, 0, 80392]
    # pattern is structural: independent of the interaction
    _, _, _, o2 = _problem(1, 4, 4, -1, seed=5)
    assert np.array_equal(o2.csr()[0], rp)


def test_row_slab_pattern_brute_force_and_thread_count():
    """The count -> scan -> fill of a row slab (the oracle's bounded CPU
    baseline): every slab row holds exactly the columns within 4 differing
    s.p. states (brute-force set differences), and the slab is the same on
    one thread and on all of them."""
    import oracle
    sp, eps, T, o = _problem(1, 4, 4, -1, seed=0)
    states = [frozenset(s) for s in _states_of(o)]
    i0, i1 = 37, 311
    prev = oracle.set_threads(0)
    try:
        runs = []
        for th in (1, prev):
            assert oracle.set_threads(th) == th
            runs.append(o.csr_rows(i0, i1))
    finally:
        oracle.set_threads(prev)
    (rp, cols, vals), (rp2, cols2, vals2) = runs
    assert np.array_equal(rp, rp2) and np.array_equal(cols, cols2) and np.array_equal(vals, vals2)
    assert len(rp) == i1 - i0 + 1 and rp[0] == 0
    for k, i in enumerate(range(i0, i1)):
        ref = [j for j in range(o.dim) if len(states[i] ^ states[j]) <= 4]
        assert list(cols[rp[k]:rp[k + 1]]) == ref
    assert len(o.csr_rows(5, 5)[1]) == 0


# ---------------------------------------------------------------- values

@pytest.mark.parametrize("nsh,Z,N,nmax", [(1, 2, 2, -1), (1, 3, 2, -1), (1, 2, 1, -1), (1, 1, 3, -1),
                                          (2, 2, 2, 2), (2, 1, 2, 1), (1, 2, 0, -1), (1, 0, 3, -1)])
def test_values_equal_brute_force(nsh, Z, N, nmax):
    sp, eps, T, o = _problem(nsh, Z, N, nmax, seed=3)
    states, Hb = brute.hamiltonian(sp, Z, N, nmax, (Z + N) % 2, eps, T)
    idx = {s: i for i, s in enumerate(states)}
    perm = np.array([idx[s] for s in _states_of(o)], dtype=int)
    rp, cols, vals, ab = o.csr()
    Ho = oracle.dense_from_csr(rp, cols, vals, o.dim)
    assert np.allclose(Ho, Hb[np.ix_(perm, perm)], rtol=0, atol=1e-12)
    # brute force has no entries outside the oracle's structural pattern
    mask = np.zeros_like(Ho, dtype=bool)
    for i in range(o.dim):
        mask[i, cols[rp[i]:rp[i + 1]]] = True
    assert not np.any(Hb[np.ix_(perm, perm)][~mask])


def test_values_config0_columns_brute_force():
    """Columns of the 4p+4n N<=1 H against brute force on a sample of kets."""
    sp, eps, T, o = _problem(1, 4, 4, -1, seed=0)
    states = _states_of(o)
    index = {s: i for i, s in enumerate(states)}
    V = {k: np.asarray(T[k], np.float64) for k in T}
    for j in range(0, o.dim, 97):
        col = {}
        for coef, ops in brute._terms(o.S, eps, V, states[j]):
            sgn, out = brute.apply_string(ops, states[j])
            if sgn:
                col[index[out]] = col.get(index[out], 0.0) + sgn * coef
        cols, vals, ab, d = o.row(j)   # H is symmetric: row j == column j
        got = dict(zip(cols.tolist(), vals.tolist()))
        for i, v in col.items():
            assert abs(got.get(i, 0.0) - v) < 1e-12
        assert set(k for k, v in col.items() if v != 0) <= set(got)


def test_closed_form_zero_interaction():
    """V = 0: H is diagonal and its levels are sums of eps (320..400 MeV)."""
    sp, eps, T, o = _problem(1, 4, 4, -1, zero=True)
    rp, cols, vals, ab = o.csr()
    H = oracle.dense_from_csr(rp, cols, vals, o.dim)
    assert np.count_nonzero(H - np.diag(np.diag(H))) == 0
    levels = {}
    for s in brute.basis(sp, 4, 4, -1, 0):
        e = sum(float(eps[m % 8]) for m in s)
        levels[e] = levels.get(e, 0) + 1
    assert levels == {320.0: 51, 340.0: 248, 360.0: 416, 380.0: 248, 400.0: 51}
    w = oracle.lowest_dense(H, o.dim)
    ref = np.sort(np.concatenate([[e] * c for e, c in levels.items()]))
    assert np.allclose(w, ref, atol=1e-10)
    assert np.allclose(oracle.lowest_dense(H, 5), [320.0] * 5)


def test_closed_form_two_like_particles():
    """2 protons, no neutrons: H_(cd),(ab) = (eps_a+eps_b) delta + V^pp_cdab, a<b, c<d."""
    sp = synth.ho_sp_table(2)
    S = len(sp["N"])
    eps = synth.sp_energies(sp, 20.0)
    T = synth.tbme_tables(sp, 9, np.float64)
    o = oracle.OracleProblem(sp, 2, 0, -1, 0, eps, T)
    pairs = [tuple(int(x) for x in o.species(0)["occ"][p]) for p in o.p_idx]
    V = T["pp"].reshape(S, S, S, S)
    ref = np.array([[V[c, d, a, b] + ((eps[a] + eps[b]) if (a, b) == (c, d) else 0.0)
                     for (a, b) in pairs] for (c, d) in pairs])
    rp, cols, vals, ab = o.csr()
    assert np.allclose(oracle.dense_from_csr(rp, cols, vals, o.dim), ref, atol=1e-13)


def test_closed_form_proton_neutron_pair():
    """1 proton + 1 neutron: H_(c,d),(a,b) = (eps_a+eps_b) delta + V^pn_cdab."""
    sp = synth.ho_sp_table(2)
    S = len(sp["N"])
    eps = synth.sp_energies(sp, 20.0)
    T = synth.tbme_tables(sp, 4, np.float64)
    o = oracle.OracleProblem(sp, 1, 1, -1, 0, eps, T)
    P, Nn = o.species(0)["occ"], o.species(1)["occ"]
    st = [(int(P[o.p_idx[i]][0]), int(Nn[o.n_idx[i]][0])) for i in range(o.dim)]
    V = T["pn"].reshape(S, S, S, S)
    ref = np.array([[V[c, d, a, b] + ((eps[a] + eps[b]) if (a, b) == (c, d) else 0.0)
                     for (a, b) in st] for (c, d) in st])
    rp, cols, vals, ab = o.csr()
    assert np.allclose(oracle.dense_from_csr(rp, cols, vals, o.dim), ref, atol=1e-13)


def test_invariants_symmetry_linearity_trace():
    sp, eps, T, o = _problem(1, 3, 3, -1, seed=2)
    rp, cols, vals, ab = o.csr()
    H = oracle.dense_from_csr(rp, cols, vals, o.dim)
    assert np.array_equal(H, H.T)
    Tm = {k: -v for k, v in T.items()}
    om = oracle.OracleProblem(sp, 3, 3, -1, 0, eps, Tm)
    Hm = oracle.dense_from_csr(*om.csr()[:3], om.dim)
    _, _, _, oz = _problem(1, 3, 3, -1, zero=True)
    H0 = oracle.dense_from_csr(*oz.csr()[:3], oz.dim)
    assert np.allclose(H + Hm, 2 * H0, atol=1e-12)
    w = oracle.lowest_dense(H, o.dim)
    assert abs(w.sum() - np.trace(H)) < 1e-9
    # absums bound every value
    assert np.all(np.abs(vals) <= ab + 1e-12)


def test_nmax_truncation_is_a_projection():
    """The Nmax-cut H is the sub-block of the uncut H on the kept states."""
    sp, eps, T, o = _problem(2, 2, 2, 2, seed=6)
    _, _, _, full = _problem(2, 2, 2, -1, seed=6)
    st_cut = _states_of(o)
    st_full = {s: i for i, s in enumerate(_states_of(full))}
    sel = np.array([st_full[s] for s in st_cut])
    Hc = oracle.dense_from_csr(*o.csr()[:3], o.dim)
    Hf = oracle.dense_from_csr(*full.csr()[:3], full.dim)
    assert np.array_equal(Hc, Hf[np.ix_(sel, sel)])


# ---------------------------------------------------------------- scan, SpMM, eigenvalues

@pytest.mark.parametrize("n", [0, 1, 2, 7, 8, 1000, 4097])
def test_exclusive_scan(n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 3000, n)
    y = oracle.exclusive_scan(x)
    assert y[0] == 0 and len(y) == n + 1
    assert np.array_equal(y[1:], np.cumsum(x))


def test_spmm_matches_dense_product():
    sp, eps, T, o = _problem(1, 4, 4, -1, seed=1)
    rp, cols, vals, ab = o.csr()
    H = oracle.dense_from_csr(rp, cols, vals, o.dim)
    X = np.random.default_rng(1).standard_normal((o.dim, 8))
    assert np.allclose(oracle.spmm(rp, cols, vals, X), H @ X, atol=1e-10)


def test_sparse_lowest_matches_dense():
    sp, eps, T, o = _problem(2, 3, 3, 2, seed=8)
    rp, cols, vals, ab = o.csr()
    H = oracle.dense_from_csr(rp, cols, vals, o.dim)
    wd = oracle.lowest_dense(H, 6)
    ws = oracle.lowest_sparse(rp, cols, vals, o.dim, 6)
    assert np.allclose(wd, ws, atol=1e-8)
    # Rayleigh quotients bound the lowest eigenvalue from above
    X = np.random.default_rng(2).standard_normal((o.dim, 4))
    rq = np.einsum("ij,ij->j", X, H @ X) / np.einsum("ij,ij->j", X, X)
    assert np.all(rq >= wd[0] - 1e-9)


# ---- count benchmark (Sec. 2.1, Listing 2) -------------------------------------

def _all_subsets(S, N):
    import itertools
    return np.array(list(itertools.combinations(range(S), N)), np.uint16)


@pytest.mark.parametrize("S,N,max_diff,expect", [
    (10, 4, 4, 1 + 4 * 6 + 6 * 15),             # k <= 2 moved particles: sum C(N,k) C(S-N,k)
    (10, 4, 6, 1 + 4 * 6 + 6 * 15 + 4 * 20),
    (10, 4, 0, 1),
    (9, 3, 4, 1 + 3 * 6 + 3 * 15)])
def test_count_pairs_closed_form_all_subsets(S, N, max_diff, expect):
    """Over every N-subset of S states, each state has sum_k C(N,k) C(S-N,k)
    partners with at most k moved particles (2k differing states)."""
    mbs = _all_subsets(S, N)
    c = oracle.count_pairs(mbs, max_diff=max_diff)
    assert np.all(c == expect)


def test_count_pairs_brute_force_sets():
    import synth
    mbs = synth.e1_states(300, N=8, S=128, r=0.9, seed=5)   # denser than the benchmark
    sets = [set(x.tolist()) for x in mbs]
    ref = np.array([sum(len(a ^ b) <= 4 for b in sets) for a in sets])
    assert ref.sum() > 2 * len(sets)          # the case has off-diagonal pairs
    assert np.array_equal(oracle.count_pairs(mbs), ref)
    rows = np.array([7, 0, 299, 7])
    assert np.array_equal(oracle.count_pairs(mbs, rows=rows), ref[rows])


def test_count_pairs_duplicates_and_singletons():
    mbs = np.array([[0, 1, 2, 3], [0, 1, 2, 3], [0, 1, 2, 4], [10, 11, 12, 13]], np.uint16)
    assert oracle.count_pairs(mbs).tolist() == [3, 3, 3, 1]
    assert oracle.count_pairs(mbs[:0]).tolist() == []


# ---- observables (Fig. 1, observables step) ------------------------------------------

def _operator(n_shell, Z, N, nmax, seed, twoM=None):
    """Oracle problem of the two-body operator with the TBMEs of `seed` and
    no one-body part (oracle Slater-Condon rules), and its CSR."""
    sp = synth.ho_sp_table(n_shell)
    T = synth.tbme_tables(sp, seed, np.float64)
    if twoM is None:
        twoM = (Z + N) % 2
    o = oracle.OracleProblem(sp, Z, N, nmax, twoM, np.zeros(len(sp["N"])), T)
    return o, o.csr()


def test_expectation_values_dense_and_unit_vectors():
    o, (rp, col, val, ab) = _operator(1, 2, 2, -1, 77)
    dense = oracle.dense_from_csr(rp, col, val, o.dim)
    X = np.random.default_rng(1).standard_normal((o.dim, 3))
    a = oracle.expectation_values(rp, col, val, X)
    assert np.allclose(a, np.einsum("iv,ij,jv->v", X, dense, X), rtol=1e-13, atol=1e-12)
    for i in (0, o.dim // 2, o.dim - 1):     # unit vector: the diagonal element
        e = np.zeros(o.dim)
        e[i] = 1.0
        assert oracle.expectation_values(rp, col, val, e)[0] == o.element(i, i)[0]


def test_transition_elements_dense_units_and_polarisation():
    """x^T O y against the dense operator and against single elements
    (unit vectors pick O_ij); the polarisation identity ties it to the
    expectation values, x^T O y = (a(x + y) - a(x - y)) / 4 for a symmetric
    O; a non-symmetric CSR catches swapped X and Y."""
    o, (rp, col, val, ab) = _operator(1, 2, 2, -1, 78)
    dense = oracle.dense_from_csr(rp, col, val, o.dim)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((o.dim, 4))
    Y = rng.standard_normal((o.dim, 4))
    t = oracle.expectation_values(rp, col, val, X, Y)
    assert np.allclose(t, np.einsum("iv,ij,jv->v", X, dense, Y), rtol=1e-13, atol=1e-12)
    pol = (oracle.expectation_values(rp, col, val, X + Y) - oracle.expectation_values(rp, col, val, X - Y)) / 4
    assert np.allclose(t, pol, rtol=1e-12, atol=1e-12)
    nz = [(i, int(col[e])) for i in range(o.dim) for e in range(rp[i], rp[i + 1]) if col[e] != i]
    for i, j in nz[:: max(1, len(nz) // 5)]:
        ei = np.zeros(o.dim); ei[i] = 1.0
        ej = np.zeros(o.dim); ej[j] = 1.0
        assert oracle.expectation_values(rp, col, val, ei, ej)[0] == o.element(i, j)[0]
    with pytest.raises(ValueError):
        oracle.expectation_values(rp, col, val, X, Y[:, :2])
    A = np.triu(rng.standard_normal((6, 6)))          # not symmetric
    arp = np.concatenate([[0], np.cumsum((A != 0).sum(1))]).astype(np.int64)
    acol = np.nonzero(A)[1].astype(np.int64)
    x, y = rng.standard_normal((6, 2)), rng.standard_normal((6, 2))
    ta = oracle.expectation_values(arp, acol, A[A != 0], x, y)
    assert np.allclose(ta, np.einsum("iv,ij,jv->v", x, A, y), rtol=1e-13)
    assert not np.allclose(ta, np.einsum("iv,ij,jv->v", y, A, x))


def test_operator_has_no_one_body_part_and_scales():
    """The same TBMEs with eps = 0: H(seed) - O(seed) is the one-body
    diagonal; a scaled vector scales the value quadratically."""
    _, _, _, oh = _problem(1, 2, 2, -1, seed=4)
    _, (rp, col, val, _) = _operator(1, 2, 2, -1, 4)
    hrp, hcol, hval, _ = oh.csr()
    assert np.array_equal(rp, hrp) and np.array_equal(col, hcol)
    diff = oracle.dense_from_csr(hrp, hcol, hval, oh.dim) - oracle.dense_from_csr(rp, col, val, oh.dim)
    assert np.allclose(diff - np.diag(np.diag(diff)), 0.0, atol=1e-12)
    x = np.random.default_rng(2).standard_normal(oh.dim)
    a1 = oracle.expectation_values(rp, col, val, x)[0]
    assert np.isclose(oracle.expectation_values(rp, col, val, 3 * x)[0], 9 * a1, rtol=1e-12)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_seeded_oracle_matches_flat_tables(dtype):
    """The oracle's on-demand TBME draws (no S**4 tables) give bit for bit the
    matrix of the flat tables written by the input generator: same draws, same
    antisymmetric completion, same float32 rounding."""
    sp = synth.ho_sp_table(2)
    eps = synth.sp_energies(sp, 20.0)
    T = synth.tbme_tables(sp, 17, dtype)
    a = oracle.OracleProblem(sp, 2, 3, 2, 1, eps, T)
    b = oracle.OracleProblem(sp, 2, 3, 2, 1, eps, seed=17, round_f32=dtype == np.float32)
    ra, ca, va, aa = a.csr()
    rb, cb, vb, ab = b.csr()
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb)
    assert np.array_equal(va, vb) and np.array_equal(aa, ab)
    c = oracle.OracleProblem(sp, 2, 3, 2, 1, eps, seed=18, round_f32=dtype == np.float32)
    assert not np.array_equal(va, c.csr()[2])


def test_seeded_oracle_two_body_elements_above_128_states():
    """S = 168 (HO shells N <= 6): with one proton and one neutron, the
    element between (a, b) and (c, d) (a != c, b != d) is the single pn draw
    V_cdab; with two protons, a < b and c < d all different, it is the pp
    draw V_cdab with its sign.  Pair
    indices here reach P = a S + b > 2**14 and states above 127."""
    sp = synth.ho_sp_table(6)
    S = len(sp["N"])
    assert S == 168
    eps = synth.sp_energies(sp, 20.0)
    rng = np.random.default_rng(3)
    o = oracle.OracleProblem(sp, 1, 1, -1, 0, eps, seed=21, round_f32=False)
    P, Nn = o.species(0)["occ"][:, 0], o.species(1)["occ"][:, 0]
    hi = np.nonzero((P[o.p_idx] >= 128) & (Nn[o.n_idx] >= 128))[0]
    rows = np.concatenate([rng.choice(o.dim, 20, replace=False), rng.choice(hi, 20, replace=False)])
    for i in rows:
        for j in rng.choice(o.dim, 10, replace=False):
            a, b = int(P[o.p_idx[j]]), int(Nn[o.n_idx[j]])
            c, d = int(P[o.p_idx[i]]), int(Nn[o.n_idx[i]])
            if (a, b) == (c, d) or a == c or b == d:
                continue
            v, _ = o.element(i, j)
            Pi, Pj = c * S + d, a * S + b
            ref = synth.tbme_gaussian(21, synth.CH_PN, min(Pi, Pj), max(Pi, Pj))
            assert v == float(ref), (i, j)
    o2 = oracle.OracleProblem(sp, 2, 0, -1, 0, eps, seed=21, round_f32=True)
    occ = o2.species(0)["occ"]
    for i in rng.choice(o2.dim, 30, replace=False):
        for j in rng.choice(o2.dim, 30, replace=False):
            (c, d), (a, b) = occ[o2.p_idx[i]], occ[o2.p_idx[j]]
            if len({a, b, c, d}) < 4:
                continue
            v, _ = o2.element(i, j)
            Pi, Pj = int(d) * (int(d) - 1) // 2 + int(c), int(b) * (int(b) - 1) // 2 + int(a)
            ref = np.float32(synth.tbme_gaussian(21, synth.CH_PP, min(Pi, Pj), max(Pi, Pj)))
            assert v == float(ref), (i, j)   # <cd|H|ab> = V_cdab, a < b, c < d
