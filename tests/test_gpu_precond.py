"""Many-body basis orbitals and the block-diagonal LOBPCG preconditioner
(Sec. 2) on the GPU against the oracle: group indices bit-exact, the
preconditioned block within the FP32 storage bound of the inverses, and
LOBPCG eigenvalues against the oracle's."""

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import EIG_REL, golden, gpu_problem, inputs, oracle_problem, preset_inputs

pytestmark = pytest.mark.gpu

P = oracle.precond


def _oracle_groups(inp, labels):
    o = oracle_problem(inp)
    blk, nb = P.orbital_blocks(o.species(0)["occ"], o.species(1)["occ"], o.p_idx, o.n_idx, labels)
    return o, blk, nb


@pytest.mark.parametrize("case", [(2, 2, 3, 2, 1), (2, 3, 3, -1, 0), (3, 2, 2, 3, 0), (2, 4, 1, 2, 3),
                                  (2, 0, 3, 2, 1), (1, 2, 2, -1, 0)])
def test_orbital_blocks_bit_exact(case):
    n_shell, Z, N, nmax, twoM = case
    inp = inputs(n_shell, Z, N, nmax, seed=1, twoM=twoM)
    labels = synth.sp_orbitals(inp["sp"])
    o, ref, nref = _oracle_groups(inp, labels)
    blk, nb = gpu_problem(inp).orbital_blocks(labels)
    assert nb == nref and np.array_equal(blk.cpu().numpy(), ref)


def test_orbital_blocks_config0_and_label_extremes():
    inp = preset_inputs("c0")
    g = gpu_problem(inp)
    S = len(inp["sp"]["N"])
    for labels in (synth.sp_orbitals(inp["sp"]), np.arange(S, dtype=np.int32), np.zeros(S, np.int32)):
        o, ref, nref = _oracle_groups(inp, labels)
        blk, nb = g.orbital_blocks(labels)
        assert nb == nref and np.array_equal(blk.cpu().numpy(), ref)


def _apply_case(inp, sigma_of, labels=None, nvec=5, seed=0):
    o = oracle_problem(inp)
    rp, col, val, _ = o.csr()
    H = oracle.dense_from_csr(rp, col, val, o.dim)
    labels = synth.sp_orbitals(inp["sp"]) if labels is None else labels
    ref_blk, nb = P.orbital_blocks(o.species(0)["occ"], o.species(1)["occ"], o.p_idx, o.n_idx, labels)
    sigma = sigma_of(H)
    R = np.random.default_rng(seed).standard_normal((o.dim, nvec))
    Wr, shr, Wabs = P.block_precond(rp, col, val, ref_blk, nb, sigma, R)
    # sub-blocks whose shifted matrix is close to singular decide their shift
    # by rounding: compare only the others
    ok = np.ones(o.dim, bool)
    for rows in P.sub_blocks(ref_blk, nb):
        A = H[np.ix_(rows, rows)]
        lam = np.linalg.eigvalsh(A - sigma * np.eye(len(rows)))
        scale = np.abs(A).sum(1).max() + abs(sigma)
        if np.min(np.abs(lam)) < 1e-6 * scale:
            ok[rows] = False
    g = gpu_problem(inp)
    M = g.build_H("f64")
    blk, nbg = g.orbital_blocks(labels)
    W, sh = M.block_precond_apply((blk, nbg), sigma, torch.from_numpy(R).cuda())
    W, sh = W.cpu().numpy(), sh.cpu().numpy()
    assert ok.mean() > 0.9
    assert np.allclose(sh[ok], shr[ok], rtol=1e-12, atol=1e-12 * abs(sigma))
    err = np.abs(W - Wr)[ok]
    assert np.all(err <= 2e-5 * Wabs[ok] + 1e-300), np.max(err / Wabs[ok])
    return sh, shr, sigma


@pytest.mark.parametrize("case", [(2, 2, 3, 2, 1), (2, 3, 3, 3, 0), (2, 4, 1, 2, 3)])
def test_block_precond_below_spectrum(case):
    n_shell, Z, N, nmax, twoM = case
    inp = inputs(n_shell, Z, N, nmax, seed=2, twoM=twoM, dtype=np.float64)
    sh, shr, sigma = _apply_case(inp, lambda H: np.linalg.eigvalsh(H)[0] - 1.0)
    assert np.all(sh == sigma)                # interlacing: no block needs the fallback


@pytest.mark.parametrize("case", [(2, 2, 3, 2, 1), (2, 3, 3, 3, 0), (3, 2, 2, 2, 0)])
def test_block_precond_inside_spectrum(case):
    n_shell, Z, N, nmax, twoM = case
    inp = inputs(n_shell, Z, N, nmax, seed=3, twoM=twoM, dtype=np.float64)
    sh, shr, sigma = _apply_case(inp, lambda H: float(np.median(np.diag(H))), nvec=8, seed=1)
    assert np.any(sh < sigma) and np.any(sh == sigma)


def test_block_precond_large_groups_and_one_row_groups():
    inp = inputs(1, 2, 2, -1, seed=4, dtype=np.float64)          # dim 190
    _apply_case(inp, lambda H: np.linalg.eigvalsh(H)[0] - 0.5, labels=np.zeros(8, np.int32), nvec=3)
    _apply_case(inp, lambda H: float(np.median(np.diag(H))), labels=np.arange(8, dtype=np.int32), nvec=1)


def test_block_precond_fp32_matrix():
    """An FP32 H: the blocks are gathered from the FP32 values (the oracle
    takes the FP64 build), so compare with the FP32 value bound added."""
    inp = inputs(2, 2, 3, 2, seed=5, twoM=1)
    o = oracle_problem(inp)
    rp, col, val, _ = o.csr()
    labels = synth.sp_orbitals(inp["sp"])
    ref_blk, nb = P.orbital_blocks(o.species(0)["occ"], o.species(1)["occ"], o.p_idx, o.n_idx, labels)
    H = oracle.dense_from_csr(rp, col, val, o.dim)
    sigma = np.linalg.eigvalsh(H)[0] - 2.0
    R = np.random.default_rng(6).standard_normal((o.dim, 4))
    Wr, shr, Wabs = P.block_precond(rp, col, val, ref_blk, nb, sigma, R)
    g = gpu_problem(inp)
    M = g.build_H("f32")
    W, sh = M.block_precond_apply(g.orbital_blocks(labels), sigma, torch.from_numpy(R).cuda())
    assert np.all(sh.cpu().numpy() == sigma)
    assert np.allclose(W.cpu().numpy(), Wr, rtol=0, atol=1e-4 * np.max(Wabs))


def test_lobpcg_block_precond_config0():
    inp = preset_inputs("c0")
    g = gpu_problem(inp)
    M = g.build_H("f64")
    blocks = g.orbital_blocks(synth.sp_orbitals(inp["sp"]))
    ev, info = M.lowest_eigs(k=5, method="lobpcg", blocks=blocks)
    ref = np.array(golden()["c0"]["lowest"])
    assert np.all(np.abs(ev - ref) <= 1e-8 * np.maximum(np.abs(ref), 1)), ev - ref
    assert max(info["residual"]) <= 1e-8 * info["hnorm_est"]


def test_lobpcg_block_precond_config1_fewer_iterations():
    inp = preset_inputs("c1")
    g = gpu_problem(inp)
    M = g.build_H("f32")
    blocks = g.orbital_blocks(synth.sp_orbitals(inp["sp"]))
    ev, info = M.lowest_eigs(k=5, method="lobpcg", blocks=blocks)
    ref = np.array(golden()["c1"]["lowest"])
    assert np.all(np.abs(ev - ref) <= EIG_REL * np.maximum(np.abs(ref), 1)), ev - ref
    ev_d, info_d = M.lowest_eigs(k=5, method="lobpcg")
    print("iterations: block", info["iterations"], "diagonal", info_d["iterations"])
    assert info["iterations"] <= info_d["iterations"]


@pytest.mark.parametrize("case", [(1, 2, 2, -1), (2, 2, 1, 1), (2, 3, 2, 2)])
def test_lobpcg_block_precond_small_against_dense(case):
    inp = inputs(*case, seed=9, dtype=np.float64)
    o = oracle_problem(inp)
    g = gpu_problem(inp)
    M = g.build_H("f64")
    k = min(3, o.dim)
    ev, info = M.lowest_eigs(k=k, block=4, method="lobpcg", blocks=g.orbital_blocks(synth.sp_orbitals(inp["sp"])))
    ref = oracle.lowest_dense(oracle.dense_from_csr(*o.csr()[:3], o.dim), k)
    assert np.allclose(ev, ref, atol=1e-8)


def test_block_precond_invalid():
    import paper_2110_10765_gb300 as ci
    inp = inputs(2, 2, 3, 2, seed=5, twoM=1)
    g = gpu_problem(inp)
    M = g.build_H("f64")
    blk, nb = g.orbital_blocks(synth.sp_orbitals(inp["sp"]))
    R = torch.zeros((M.dim, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(ci.CIError):
        M.block_precond_apply((blk, nb - 1), 0.0, R)                  # an index outside 0..nblocks-1
    with pytest.raises(ci.CIError):
        M.block_precond_apply((blk.cpu(), nb), 0.0, R)                # host row_block
    with pytest.raises(ci.CIError):
        M.block_precond_apply((blk, nb), float("nan"), R)
    with pytest.raises(ci.CIError):
        M.lowest_eigs(k=3, method="lobpcg", blocks=(blk, 0))
    with pytest.raises(ci.CIError):
        g.orbital_blocks(-np.ones(len(inp["sp"]["N"]), np.int32))
    with pytest.raises(ValueError):
        M.lowest_eigs(k=3, blocks=(blk, nb))                          # blocks with Lanczos


def test_lobpcg_block_precond_bf16_rowscale():
    """BF16 values with row scales: the blocks are gathered from the scaled
    values (not exactly symmetric); LOBPCG still reaches the lowest
    eigenvalues within the Weyl bound of the BF16 rounding, and refining
    with the FP64 H recovers the FP64 values."""
    inp = preset_inputs("c2_sub")
    g = gpu_problem(inp)
    Mb = g.build_H("bf16")
    rp, col, v16, scale = Mb.export()
    blocks = g.orbital_blocks(synth.sp_orbitals(inp["sp"]))
    E = torch.zeros((Mb.dim, 8), dtype=torch.float64, device="cuda")
    ev, info = Mb.lowest_eigs(k=8, method="lobpcg", blocks=blocks, evecs=E)   # default tol for BF16: 4e-3
    exact = np.array(golden()["c2_sub"]["lowest"])[:8]
    bound = np.max(np.diff(rp) * scale.astype(np.float64)) * 2.0 ** -9
    assert np.all(np.abs(ev - exact) <= bound + 1e-5 * np.abs(exact)), (np.abs(ev - exact).max(), bound)
    evr, rn = g.refine_eigs(E, iters=2)
    assert np.all(evr >= exact - 1e-9)          # Ritz values of the exact operator bound from above
    assert np.max(np.abs(evr - exact)) < np.max(np.abs(ev - exact))
