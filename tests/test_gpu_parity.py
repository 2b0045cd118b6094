"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bit-exact: species lists, basis, species connectivity, row counts, scan,
nonzero pattern (column indices).  Values: per element
|h - h64| <= rel * max(|h64|, sum |terms|) with rel = 1e-6 (FP32) or 1e-12
(FP64).  Eigenvalues: |l - l64| <= 1e-5 * max(|l64|, 1).
"""

import numpy as np
import pytest

import oracle
from helpers import (EIG_REL, REL32, REL64, golden, gpu_problem, inputs, oracle_problem, preset_inputs,
                     value_bound)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = [
    # (n_shell, Z, N, nmax) -- ragged sizes, odd A, empty species, Nmax 0
    (1, 2, 2, -1), (1, 3, 2, -1), (1, 2, 0, -1), (1, 0, 3, -1), (2, 3, 3, 2),
    (2, 2, 3, 1), (3, 2, 2, 0), (3, 3, 2, 2), (1, 1, 1, -1), (2, 4, 2, 2),
]


def _species_eq(o, g, s):
    a, b = o.species(s), g.species(s)
    assert np.array_equal(a["bits"], b["bits"])
    assert np.array_equal(a["q"], b["q"]) and np.array_equal(a["twoM"], b["twoM"])


@pytest.mark.parametrize("case", SMALL + ["c0", "c2_sub"])
def test_basis_bit_exact(case):
    inp = preset_inputs(case) if isinstance(case, str) else inputs(*case, seed=3)
    o, g = oracle_problem(inp), gpu_problem(inp)
    assert g.enumerate_basis() == o.dim
    _species_eq(o, g, 0)
    _species_eq(o, g, 1)
    p, n = g.basis()
    assert np.array_equal(p, o.p_idx) and np.array_equal(n, o.n_idx)


def _species_pairs(o, s):
    """Oracle reference of the kept species pairs (difference <= 2, or 4 with equal 2M)."""
    sp = o.species(s)
    occ, m = sp["occ"], sp["twoM"]
    n = len(occ)
    out = []
    for i in range(n):
        row = []
        for j in range(n):
            d = o.count_difference(s, i, j)
            if d <= 2 or (d == 4 and m[i] == m[j]):
                row.append((j, d))
        out.append(row)
    return out


@pytest.mark.parametrize("case", [(1, 4, 4, -1), (2, 3, 3, 2), (3, 2, 3, 1)])
def test_species_connectivity_bit_exact(case):
    inp = inputs(*case, seed=1)
    o, g = oracle_problem(inp), gpu_problem(inp)
    g.species_filter()
    for s in (0, 1):
        ptr, idx, d = g.species_conn(s)
        ref = _species_pairs(o, s)
        assert len(ptr) == len(ref) + 1
        for i, row in enumerate(ref):
            got = list(zip(idx[ptr[i]:ptr[i + 1]].tolist(), d[ptr[i]:ptr[i + 1]].tolist()))
            assert got == row


@pytest.mark.parametrize("case", SMALL + ["c0", "c2_sub"])
def test_row_counts_bit_exact(case):
    inp = preset_inputs(case) if isinstance(case, str) else inputs(*case, seed=2)
    o, g = oracle_problem(inp), gpu_problem(inp)
    dim = g.enumerate_basis()
    cnt = torch.zeros(max(dim, 1), dtype=torch.int32, device="cuda")
    nnz = g.count_nnz(cnt)
    ref = o.row_counts()
    assert nnz == int(ref.sum())
    assert np.array_equal(cnt.cpu().numpy()[:dim], ref)


@pytest.mark.parametrize("n", [0, 1, 31, 4095, 4096, 4097, 123457, 3_000_001])
def test_exclusive_scan_bit_exact(n):
    import paper_2110_10765_gb300 as ci
    rng = np.random.default_rng(n)
    x = rng.integers(0, 2000, n).astype(np.int32)
    xd = torch.from_numpy(x).cuda() if n else torch.zeros(1, dtype=torch.int32, device="cuda")
    y = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
    ci.exclusive_scan(xd[:n] if n else xd[:0], y)
    assert np.array_equal(y.cpu().numpy(), oracle.exclusive_scan(x))


@pytest.mark.parametrize("n", [1, 8, 4097, 123457])
@pytest.mark.parametrize("shift", [(1, 0), (0, 1), (3, 1)])
def test_exclusive_scan_unaligned(n, shift):
    """Counts or offsets off a 16-byte boundary take the one-load-per-item
    path (and the no-allocation variant the same), with identical results."""
    import paper_2110_10765_gb300 as ci
    sx, sy = shift
    x = np.random.default_rng(n + sx).integers(0, 2000, n).astype(np.int32)
    xb = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
    xb[sx:sx + n] = torch.from_numpy(x).cuda()
    yb = torch.full((n + 3,), -7, dtype=torch.int64, device="cuda")
    ci.exclusive_scan(xb[sx:sx + n], yb[sy:sy + n + 1])
    assert np.array_equal(yb[sy:sy + n + 1].cpu().numpy(), oracle.exclusive_scan(x))
    if sy:
        assert int(yb[0]) == -7
    yb.fill_(-7)
    check = ci.exclusive_scan_noalloc if hasattr(ci, "exclusive_scan_noalloc") else None
    if check is not None:
        check(xb[sx:sx + n], yb[sy:sy + n + 1])
        assert np.array_equal(yb[sy:sy + n + 1].cpu().numpy(), oracle.exclusive_scan(x))


def test_exclusive_scan_large_total_int64():
    import paper_2110_10765_gb300 as ci
    n = 3_000_000
    x = np.full(n, 1500, np.int32)  # total 4.5e9 > 2^31
    y = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ci.exclusive_scan(torch.from_numpy(x).cuda(), y)
    assert int(y[-1]) == 1500 * n and int(y[n // 2]) == 1500 * (n // 2)


def _check_matrix(o, M, rel, rows=None):
    rp, col, val, _ = M.export()
    if rows is None:
        orp, ocol, oval, oab = o.csr()
        assert np.array_equal(rp, orp)
        assert np.array_equal(col.astype(np.int64), ocol)
        err = np.abs(val.astype(np.float64) - oval)
        assert np.all(err <= value_bound(oval, oab, rel)), err.max()
        return rp, col, val
    for i in rows:
        ocol, oval, oab, _ = o.row(i)
        s, e = rp[i], rp[i + 1]
        assert np.array_equal(col[s:e].astype(np.int64), ocol), i
        err = np.abs(val[s:e].astype(np.float64) - oval)
        assert np.all(err <= value_bound(oval, oab, rel)), (i, err.max())
    return rp, col, val


@pytest.mark.parametrize("case", SMALL)
@pytest.mark.parametrize("vtype", ["f32", "f64"])
def test_build_H_small(case, vtype):
    inp = inputs(*case, seed=5, dtype=np.float64 if vtype == "f64" else np.float32)
    o, g = oracle_problem(inp), gpu_problem(inp)
    M = g.build_H(vtype)
    assert M.dim == o.dim
    _check_matrix(o, M, REL64 if vtype == "f64" else REL32)


def _sliced_inputs(S, Z, N, nmax, twoM, seed, dtype):
    """The first S states of the HO table up to shell 4: S = 63, 64, 65 put
    the highest state on either side of the 64-bit word boundary."""
    import synth
    sp = {k: v[:S].copy() for k, v in synth.ho_sp_table(4).items()}
    return dict(sp=sp, Z=Z, N=N, nmax=nmax, twoM=twoM, eps=synth.sp_energies(sp, 20.0),
                tables=synth.tbme_tables(sp, seed, dtype))


@pytest.mark.parametrize("S", [63, 64, 65])
@pytest.mark.parametrize("case", [(1, 1, -1, 0), (1, 2, 5, 3), (2, 2, 4, 0)])
def test_word_boundary_states(S, case):
    """Bit 63 and bit 64 of the determinant strings: basis, pattern and FP64
    values against the oracle, and the SpMM."""
    inp = _sliced_inputs(S, *case, seed=8, dtype=np.float64)
    o, g = oracle_problem(inp), gpu_problem(inp)
    assert g.enumerate_basis() == o.dim
    _species_eq(o, g, 0)
    _species_eq(o, g, 1)
    M = g.build_H("f64")
    rp, col, val = _check_matrix(o, M, REL64)
    X = np.random.default_rng(1).standard_normal((o.dim, 8))
    Y = torch.empty((o.dim, 8), dtype=torch.float64, device="cuda")
    M.apply_H(torch.from_numpy(X).cuda(), Y)
    orp, ocol, oval, oab = o.csr()
    ref = oracle.spmm(orp, ocol, oval, X)
    bound = oracle.spmm(orp, ocol, np.maximum(np.abs(oval), oab), np.abs(X))
    assert np.all(np.abs(Y.cpu().numpy() - ref) <= 1e-11 * bound + 1e-300)


@pytest.mark.parametrize("case", [(16, 0, -1, 0), (16, 1, 2, 1), (15, 2, 2, 1), (16, 16, 0, 0), (16, 2, 1, 0)])
def test_maximum_particle_number(case):
    """16 nucleons of a species (the ABI's maximum) in the 20 states of the
    shells N <= 2: hole-like determinants, long phase strings."""
    Z, N, nmax, twoM = case
    inp = inputs(2, Z, N, nmax, seed=9, dtype=np.float64, twoM=twoM)
    o, g = oracle_problem(inp), gpu_problem(inp)
    assert g.enumerate_basis() == o.dim
    _species_eq(o, g, 0)
    _species_eq(o, g, 1)
    M = g.build_H("f64")
    rows = None if o.dim < 5000 else np.random.default_rng(0).choice(o.dim, 300, replace=False)
    _check_matrix(o, M, REL64, rows)


def test_build_H_config0_fp64():
    inp = preset_inputs("c0")
    o, g = oracle_problem(inp), gpu_problem(inp)
    M = g.build_H("f64")
    assert (M.dim, M.nnz) == (1014, 88462)
    _check_matrix(o, M, REL64)


def test_build_H_nmax2_subspace_fp32():
    inp = preset_inputs("c2_sub")
    o, g = oracle_problem(inp), gpu_problem(inp)
    M = g.build_H("f32")
    assert M.nnz == golden()["c2_sub"]["nnz"]
    _check_matrix(o, M, REL32)


def _sha256_i64(a):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i8").tobytes()).hexdigest()


def _boundary_rows(o):
    """First and last row of every (2M, q) group of the proton list: the
    rows where a proton 2M block or a q prefix of the cut begins or ends."""
    sp = o.species(0)
    key = sp["twoM"].astype(np.int64)[o.p_idx] * 1024 + sp["q"].astype(np.int64)[o.p_idx]
    edges = np.flatnonzero(np.diff(key)) + 1
    starts = np.concatenate([[0], edges])
    ends = np.concatenate([edges - 1, [o.dim - 1]])
    return set(starts.tolist()) | set(ends.tolist())


@pytest.mark.parametrize("case", ["c0", "c2_sub", "c1"])
def test_build_H_full_pattern_digest(case):
    """The whole structural pattern (row_ptr and every column index) against
    SHA-256 digests of the oracle's full CSR, bit for bit; c1 is the
    benchmark workload at full size (172,684 rows, 102,601,752 nonzeros)."""
    inp = preset_inputs(case)
    g = gpu_problem(inp)
    M = g.build_H("f64" if case == "c0" else "f32")
    gd = golden()[case]
    assert (M.dim, M.nnz) == (gd["dim"], gd["nnz"])
    rp, col, _, _ = M.export()
    assert _sha256_i64(rp) == gd["row_ptr_sha256"]
    assert _sha256_i64(col) == gd["col_sha256"]


def test_build_H_config1_full_size_sampled_rows():
    """Nmax=4, 70 states per species (two-word bit strings): values and
    patterns of 2,000+ rows against the oracle, among them the first and
    last row of every (2M, q) group of the proton list."""
    inp = preset_inputs("c1")
    o, g = oracle_problem(inp), gpu_problem(inp)
    M = g.build_H("f32")
    gd = golden()["c1"]
    assert (M.dim, M.nnz) == (gd["dim"], gd["nnz"])
    edge = _boundary_rows(o)
    rng = np.random.default_rng(11)
    rows = set(edge) | {0, M.dim - 1}
    while len(rows) < 2000 + len(edge):
        rows.add(int(rng.integers(0, M.dim)))
    rows = sorted(rows)
    rp, col, val = _check_matrix(o, M, REL32, rows)
    # structural symmetry and value symmetry on sampled rows
    for i in rows[::50]:
        for j, v in zip(col[rp[i]:rp[i + 1]].tolist(), val[rp[i]:rp[i + 1]].tolist()):
            seg = col[rp[j]:rp[j + 1]]
            k = np.searchsorted(seg, i)
            assert k < len(seg) and seg[k] == i
            assert abs(val[rp[j] + k] - v) <= 1e-5 * max(abs(v), 1.0)


def test_seeded_tables_match_synth_tables():
    """The device TBME generator reproduces synth's tables bit for bit."""
    inp = inputs(2, 3, 2, 2, seed=77)
    g_tab = gpu_problem(inp)
    g_seed = gpu_problem(inp, seed=77)
    A = g_tab.build_H("f32").export()
    B = g_seed.build_H("f32").export()
    assert np.array_equal(A[0], B[0]) and np.array_equal(A[1], B[1]) and np.array_equal(A[2], B[2])


def _rand_block(dim, nvec, dtype, seed=0):
    return np.random.default_rng(seed).standard_normal((dim, nvec)).astype(dtype)


@pytest.mark.parametrize("nvec", [1, 3, 8])
def test_apply_H_small_full(nvec):
    inp = inputs(2, 3, 3, 2, seed=4)
    o, g = oracle_problem(inp), gpu_problem(inp)
    M = g.build_H("f32")
    rp, cols, vals, ab = o.csr()
    X = _rand_block(o.dim, nvec, np.float32)
    Y = torch.empty((o.dim, nvec), dtype=torch.float32, device="cuda")
    M.apply_H(torch.from_numpy(X).cuda(), Y)
    torch.cuda.synchronize()
    ref = oracle.spmm(rp, cols, vals, X.astype(np.float64))
    # FP32 accumulation: bound by sum |H_ij X_j| * 1e-6 per row
    bound = 1e-6 * oracle.spmm(rp, cols, np.abs(vals), np.abs(X.astype(np.float64))) + 1e-30
    assert np.all(np.abs(Y.cpu().numpy() - ref) <= bound)


def test_apply_H_config0_fp64():
    inp = preset_inputs("c0")
    o, g = oracle_problem(inp), gpu_problem(inp)
    M = g.build_H("f64")
    rp, cols, vals, ab = o.csr()
    X = _rand_block(o.dim, 8, np.float64, 1)
    Y = torch.empty((o.dim, 8), dtype=torch.float64, device="cuda")
    M.apply_H(torch.from_numpy(X).cuda(), Y)
    ref = oracle.spmm(rp, cols, vals, X)
    bound = 1e-12 * oracle.spmm(rp, cols, np.abs(vals), np.abs(X)) + 1e-300
    assert np.all(np.abs(Y.cpu().numpy() - ref) <= bound)


def test_apply_H_config1_sampled_rows():
    inp = preset_inputs("c1")
    o, g = oracle_problem(inp), gpu_problem(inp)
    M = g.build_H("f32")
    X = _rand_block(M.dim, 8, np.float32, 2)
    Y = torch.empty((M.dim, 8), dtype=torch.float32, device="cuda")
    M.apply_H(torch.from_numpy(X).cuda(), Y)
    Yh = Y.cpu().numpy()
    X64 = X.astype(np.float64)
    for i in np.random.default_rng(3).integers(0, M.dim, 60):
        c, v, ab, _ = o.row(int(i))
        ref = v @ X64[c]
        bound = 1e-6 * (np.abs(v) @ np.abs(X64[c]))
        assert np.all(np.abs(Yh[i] - ref) <= bound + 1e-30)


def test_lowest_eigs_config0_fp64():
    inp = preset_inputs("c0")
    g = gpu_problem(inp)
    M = g.build_H("f64")
    ev, info = M.lowest_eigs(k=5)
    ref = np.array(golden()["c0"]["lowest"])
    assert np.all(np.abs(ev - ref) <= 1e-9 * np.maximum(np.abs(ref), 1))


def test_lowest_eigs_degenerate_closed_form():
    """Zero interaction: lowest five levels are all 320 MeV (51-fold).  The
    Krylov space of a diagonal H with few distinct levels runs out, so a
    block turns rank deficient: the device block QR hands it to the host's
    rank-revealing path (deflation and random completion)."""
    inp = inputs(1, 4, 4, -1, zero=True, dtype=np.float64)
    M = gpu_problem(inp).build_H("f64")
    ev, info = M.lowest_eigs(k=5)
    assert np.allclose(ev, 320.0, rtol=0, atol=1e-8)
    assert info["host_qr"] >= 1


def test_lowest_eigs_nmax2_subspace_fp32():
    inp = preset_inputs("c2_sub")
    M = gpu_problem(inp).build_H("f32")
    evecs = torch.zeros((M.dim, 10), dtype=torch.float64, device="cuda")
    ev, info = M.lowest_eigs(k=10, evecs=evecs)
    ref = np.array(golden()["c2_sub"]["lowest"])
    assert np.all(np.abs(ev - ref) <= EIG_REL * np.maximum(np.abs(ref), 1)), ev - ref
    V = evecs.cpu().numpy()
    assert np.allclose(V.T @ V, np.eye(10), atol=1e-6)


def test_lowest_eigs_config1_fp32():
    inp = preset_inputs("c1")
    M = gpu_problem(inp).build_H("f32")
    ev, info = M.lowest_eigs(k=5)
    ref = np.array(golden()["c1"]["lowest"])
    assert np.all(np.abs(ev - ref) <= EIG_REL * np.maximum(np.abs(ref), 1)), ev - ref
    assert max(info["residual"]) <= 1e-4 * info["hnorm_est"]
    assert info["host_qr"] == 0   # every block step orthonormalised on the device
    assert 0 <= info["qr_one_pass"] <= info["iterations"]


@pytest.mark.parametrize("case", [(1, 2, 2, -1), (2, 2, 1, 1), (1, 1, 1, -1)])
def test_lowest_eigs_small_dense_path(case):
    inp = inputs(*case, seed=9, dtype=np.float64)
    o = oracle_problem(inp)
    M = gpu_problem(inp).build_H("f64")
    k = min(3, o.dim)
    ev, info = M.lowest_eigs(k=k, max_basis=32, block=4) if o.dim >= 3 else M.lowest_eigs(k=1, block=1,
                                                                                              max_basis=16)
    ref = oracle.lowest_dense(oracle.dense_from_csr(*o.csr()[:3], o.dim), len(ev))
    assert np.allclose(ev, ref, atol=1e-9)


def test_config2_full_size_sampled_rows_and_precision():
    """Nmax=6 (dim 2,680,018, 3.2e9 nonzeros): sampled rows against the oracle
    (pattern bit-exact, values within the FP32 bound), structural symmetry on
    them, and the lowest 10 eigenvalues of the FP32 H against the FP64 GPU
    run (the precision study of the workload)."""
    import torch
    inp = preset_inputs("c2")
    o, g = oracle_problem(inp), gpu_problem(inp)
    M = g.build_H("f32")
    assert M.dim == golden()["c2"]["dim"]
    rp = torch.empty(M.dim + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(M.nnz, dtype=torch.int32, device="cuda")
    val = torch.empty(M.nnz, dtype=torch.float32, device="cuda")
    M.export_device(rp, col, val)
    rph = rp.cpu().numpy()
    assert rph[-1] == M.nnz
    rng = np.random.default_rng(21)
    rows = sorted(set(rng.integers(0, M.dim, 12).tolist()) | {0, M.dim - 1})
    for i in rows:
        ocol, oval, oab, _ = o.row(i)
        c = col[rph[i]:rph[i + 1]].cpu().numpy()
        v = val[rph[i]:rph[i + 1]].cpu().numpy()
        assert np.array_equal(c.astype(np.int64), ocol), i
        assert np.all(np.abs(v.astype(np.float64) - oval) <= value_bound(oval, oab, REL32)), i
        for j in c[:: max(1, len(c) // 16)].tolist():      # the transposed entry exists
            seg = col[rph[j]:rph[j + 1]].cpu().numpy()
            k = np.searchsorted(seg, i)
            assert k < len(seg) and seg[k] == i
    del rp, col, val
    ev32, info32 = M.lowest_eigs(k=10)
    del M
    ev64, info64 = g.build_H("f64").lowest_eigs(k=10)
    assert np.all(np.abs(ev32 - ev64) <= EIG_REL * np.maximum(np.abs(ev64), 1)), ev32 - ev64


def _bf16_rn(x32):
    """Round float32 values to bfloat16 bits, to nearest even (finite input)."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def _bf16_to_f64(h16):
    return (h16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("case", ["small", "c2_sub"])
def test_build_H_bf16_rowscale(case):
    """BF16 storage (the precision-study option): per row, scale = max |v|
    of the FP32 row and the stored value is bf16(v * (1/scale)) rounded to
    nearest even; bit-exact against the FP32 build."""
    inp = inputs(2, 3, 2, 2, seed=5) if case == "small" else preset_inputs("c2_sub")
    g = gpu_problem(inp)
    M32 = g.build_H("f32")
    Mb = g.build_H("bf16")
    rp, col, v32, _ = M32.export()
    rpb, colb, v16, scale = Mb.export()
    assert np.array_equal(rp, rpb) and np.array_equal(col, colb)
    for r in range(M32.dim):
        row = v32[rp[r]:rp[r + 1]]
        m = np.float32(np.max(np.abs(row))) if len(row) else np.float32(0)
        sc = m if m > 0 else np.float32(1)
        assert scale[r] == sc
        inv = np.float32(1) / sc
        assert np.array_equal(v16[rp[r]:rp[r + 1]], _bf16_rn(row * inv)), r


def test_apply_and_eigs_bf16_rowscale():
    """SpMM of the BF16 form against its own values in FP64, and the lowest
    eigenvalues within the perturbation bound of the BF16 rounding (Weyl:
    |d lambda| <= ||dH||_2 <= max row sum of |dH|, |dH_rj| <= 2^-9 scale_r)."""
    import torch
    inp = preset_inputs("c2_sub")
    g = gpu_problem(inp)
    Mb = g.build_H("bf16")
    rp, col, v16, scale = Mb.export()
    vals = _bf16_to_f64(v16) * np.repeat(scale.astype(np.float64), np.diff(rp))
    X = np.random.default_rng(4).standard_normal((Mb.dim, 8)).astype(np.float32)
    Y = torch.empty((Mb.dim, 8), dtype=torch.float32, device="cuda")
    Mb.apply_H(torch.from_numpy(X).cuda(), Y)
    ref = oracle.spmm(rp, col, vals, X.astype(np.float64))
    absref = oracle.spmm(rp, col, np.abs(vals), np.abs(X.astype(np.float64)))
    assert np.all(np.abs(Y.cpu().numpy() - ref) <= 1e-6 * absref + 1e-30)
    ev, info = Mb.lowest_eigs(k=10)
    exact = np.array(golden()["c2_sub"]["lowest"])
    bound = np.max(np.diff(rp) * scale.astype(np.float64)) * 2.0 ** -9
    assert np.all(np.abs(ev - exact) <= bound + 1e-5 * np.abs(exact)), (np.abs(ev - exact).max(), bound)


def _sp128():
    import synth
    sp6 = synth.ho_sp_table(6)                  # 168 states: the first 128 (shells 0..5 and part of 6)
    return {k: v[:128].copy() for k, v in sp6.items()}


def test_maximum_sp_states_seeded_tables():
    """S = 128 (two 64-bit words, both full) with TBMEs from the
    seeded generator (no flat tables): one proton and one neutron, no Nmax
    cut, so every basis pair is within four differences.  The matrix is
    symmetric, dense, and the solver agrees with LAPACK on it."""
    import synth
    sp = _sp128()
    eps = synth.sp_energies(sp, 20.0)
    inp = dict(sp=sp, Z=1, N=1, nmax=-1, twoM=0, eps=eps)
    g = gpu_problem(inp, seed=12)
    dim = g.enumerate_basis()
    assert g.species(0)["bits"].shape[1] == 2
    assert int(g.species(0)["bits"][:, 1].max()) >> 63 == 1        # state 127 occurs
    M = g.build_H("f64")
    assert M.nnz == dim * dim
    rp, col, val, _ = M.export()
    H = oracle.dense_from_csr(rp, col.astype(np.int64), val, dim)
    assert np.array_equal(H, H.T)
    ev, info = M.lowest_eigs(k=5)
    ref = np.linalg.eigvalsh(H)[:5]
    assert np.allclose(ev, ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def _sp_first(n_shell, S):
    import synth
    return {k: v[:S].copy() for k, v in synth.ho_sp_table(n_shell).items()}


@pytest.mark.parametrize("case", [(6, 168, 2, 2, 6, 0), (7, 240, 2, 1, 7, 1), (8, 256, 1, 2, 8, 1),
                                  (7, 200, 1, 1, -1, 0)])
def test_sp_states_above_128(case):
    """S = 168, 200, 240, 256 s.p. states (three and four 64-bit words; HO
    shells up to N = 8) with TBMEs drawn by the counter-based generator on
    both sides: species lists bit-exact, the whole CSR pattern bit-exact,
    FP64 and FP32 values within their bounds, the SpMM, and the lowest
    eigenvalues against the oracle's Lanczos."""
    n_shell, S, Z, N, nmax, twoM = case
    sp = _sp_first(n_shell, S)
    import synth
    eps = synth.sp_energies(sp, 20.0)
    o = oracle.OracleProblem(sp, Z, N, nmax, twoM, eps, seed=31, round_f32=False)   # exact draws
    g = gpu_problem(dict(sp=sp, Z=Z, N=N, nmax=nmax, twoM=twoM, eps=eps), seed=31)
    assert g.enumerate_basis() == o.dim > 0
    W = (S + 63) // 64
    for s in (0, 1):
        _species_eq(o, g, s)
        assert g.species(s)["bits"].shape[1] == W
    occ = np.concatenate([o.species(0)["occ"].ravel(), o.species(1)["occ"].ravel()])
    assert occ.max() >= 64 * (W - 1)                        # the top word is in use
    M = g.build_H("f64")
    rp, col, val = _check_matrix(o, M, REL64)
    M32 = g.build_H("f32")
    _check_matrix(o, M32, REL32)
    X = np.random.default_rng(2).standard_normal((o.dim, 8))
    Y = torch.empty((o.dim, 8), dtype=torch.float64, device="cuda")
    M.apply_H(torch.from_numpy(X).cuda(), Y)
    orp, ocol, oval, oab = o.csr()
    ref = oracle.spmm(orp, ocol, oval, X)
    bound = oracle.spmm(orp, ocol, np.maximum(np.abs(oval), oab), np.abs(X))
    assert np.all(np.abs(Y.cpu().numpy() - ref) <= 1e-11 * bound + 1e-300)
    ev, info = M.lowest_eigs(k=4)
    ref_ev = oracle.lowest_sparse(orp, ocol, oval, o.dim, 4)
    assert np.allclose(ev, ref_ev, rtol=0, atol=1e-8 * max(1.0, np.abs(ref_ev).max()))


def test_maximum_sp_states_zero_interaction_closed_form():
    """S = 128 with zero TBMEs (device tables): the levels of one proton and
    one neutron are eps_a + eps_b over the pairs with m_a + m_b = 0."""
    import synth
    sp = _sp128()
    eps = synth.sp_energies(sp, 20.0)
    S = 128
    zeros = {k: torch.zeros(S ** 4, dtype=torch.float32, device="cuda") for k in ("pp", "nn", "pn")}
    inp = dict(sp=sp, Z=1, N=1, nmax=-1, twoM=0, eps=eps, tables=zeros)
    g = gpu_problem(inp)
    M = g.build_H("f32")
    ev, info = M.lowest_eigs(k=5)
    m = np.asarray(sp["twom"])
    levels = np.sort([eps[a] + eps[b] for a in range(S) for b in range(S) if m[a] + m[b] == 0])
    assert np.allclose(ev, levels[:5], rtol=0, atol=1e-4)
    del zeros
