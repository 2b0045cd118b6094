"""Half-stored symmetric H (Fig. 2, optional FMA: one stored element updates
both outputs) against the oracle: the stored triangle exactly, the SpMM
within the FP32 / FP64 element bounds, and the eigensolvers on it."""

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import EIG_REL, REL32, golden, gpu_problem, inputs, oracle_problem, preset_inputs

pytestmark = pytest.mark.gpu


def _upper_ref(rp, col, val):
    keep = col >= np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    urp = np.concatenate([[0], np.cumsum(np.add.reduceat(keep.astype(np.int64), rp[:-1])
                                         if len(col) else np.zeros(len(rp) - 1, np.int64))])
    return urp, col[keep], val[keep]


@pytest.mark.parametrize("case,vt", [((2, 2, 3, 2), "f32"), ((2, 3, 2, -1), "f64"), ((1, 2, 2, -1), "bf16")])
def test_upper_triangle_exact(case, vt):
    inp = inputs(*case, seed=1, dtype=np.float64 if vt == "f64" else np.float32)
    M = gpu_problem(inp).build_H(vt)
    U = M.upper()
    assert U.nnz == (M.nnz + M.dim) // 2 and U.dim == M.dim and U.vtype == M.vtype
    rp, col, val, rs = M.export()
    urp, ucol, uval, urs = U.export()
    wrp, wcol, wval = _upper_ref(rp, col.astype(np.int64), val)
    assert np.array_equal(urp, wrp) and np.array_equal(ucol, wcol) and np.array_equal(uval, wval)
    if rs is not None:
        assert np.array_equal(rs, urs)


def _spmm_check(inp, vt, nvec, rel):
    o = oracle_problem(inp)
    rp, col, val, ab = o.csr()
    M = gpu_problem(inp).build_H(vt).upper()
    dt = torch.float64 if vt == "f64" else torch.float32
    X = np.random.default_rng(2).standard_normal((o.dim, nvec))
    Y = torch.empty((o.dim, nvec), dtype=dt, device="cuda")
    M.apply_H(torch.from_numpy(X).to(dt).cuda(), Y)
    Xr = X.astype(np.float32).astype(np.float64) if vt != "f64" else X
    ref = oracle.spmm(rp, col, val, Xr)
    bound = oracle.spmm(rp, col, np.maximum(np.abs(val), ab), np.abs(Xr))
    err = np.abs(Y.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= rel * bound + 1e-300), np.max(err / bound)


@pytest.mark.parametrize("nvec", [8, 3, 1])
def test_upper_spmm_fp32(nvec):
    # rounding of the elements (1e-6) plus FP32 accumulation in any order
    _spmm_check(inputs(2, 2, 3, 2, seed=3), "f32", nvec, 4 * REL32)


@pytest.mark.parametrize("nvec", [8, 5])
def test_upper_spmm_fp64(nvec):
    _spmm_check(inputs(2, 3, 2, -1, seed=4, dtype=np.float64), "f64", nvec, 1e-11)


def test_upper_spmm_config0():
    _spmm_check(preset_inputs("c0"), "f32", 8, 4 * REL32)


def test_upper_spmm_bf16_matches_full_storage():
    """Same stored values and scales: the two storages differ only in the
    order of the FP32 sums."""
    inp = inputs(2, 2, 3, 2, seed=5)
    M = gpu_problem(inp).build_H("bf16")
    U = M.upper()
    X = torch.randn((M.dim, 8), device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    Yf, Yu = torch.empty_like(X), torch.empty_like(X)
    M.apply_H(X, Yf)
    U.apply_H(X, Yu)
    rp, col, val, rs = M.export()
    absH = np.abs(val.astype(np.float32)) * np.repeat(rs, np.diff(rp))
    bound = oracle.spmm(rp, col.astype(np.int64), absH.astype(np.float64), np.abs(X.cpu().numpy()).astype(np.float64))
    assert np.all(np.abs((Yf - Yu).cpu().numpy()) <= 1e-5 * bound + 1e-30)


def test_upper_lanczos_config1():
    M = gpu_problem(preset_inputs("c1")).build_H("f32").upper()
    ev, info = M.lowest_eigs(k=5)
    ref = np.array(golden()["c1"]["lowest"])
    assert np.all(np.abs(ev - ref) <= EIG_REL * np.maximum(np.abs(ref), 1)), ev - ref


def test_upper_lobpcg_block_precond_config0():
    inp = preset_inputs("c0")
    g = gpu_problem(inp)
    M = g.build_H("f64").upper()
    ev, info = M.lowest_eigs(k=5, method="lobpcg", blocks=g.orbital_blocks(synth.sp_orbitals(inp["sp"])))
    ref = np.array(golden()["c0"]["lowest"])
    assert np.all(np.abs(ev - ref) <= 1e-8 * np.maximum(np.abs(ref), 1)), ev - ref


def test_upper_block_precond_equals_full():
    """The preconditioner mirrors the stored triangle: same blocks, same
    inverses as from the full matrix."""
    inp = inputs(2, 2, 3, 2, seed=6, dtype=np.float64, twoM=1)
    g = gpu_problem(inp)
    M = g.build_H("f64")
    U = M.upper()
    blocks = g.orbital_blocks(synth.sp_orbitals(inp["sp"]))
    R = torch.randn((M.dim, 4), dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(2))
    sigma = -50.0
    Wf, sf = M.block_precond_apply(blocks, sigma, R)
    Wu, su = U.block_precond_apply(blocks, sigma, R)
    assert torch.equal(sf, su) and torch.equal(Wf, Wu)


def test_upper_invalid_and_empty():
    import paper_2110_10765_gb300 as ci
    M = gpu_problem(inputs(1, 2, 2, -1, seed=1)).build_H("f32")
    with pytest.raises(ci.CIError):
        M.upper().upper()
    E = gpu_problem(inputs(1, 2, 2, 0, seed=1, twoM=9)).build_H("f32")   # no state with 2M = 9
    assert E.dim == 0 and E.upper().nnz == 0
