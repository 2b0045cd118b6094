"""The reorthogonalisation products of the block Lanczos solver (Sec. 2,
Fig. 1 eigensolve) through ci_basis_product: the tensor-core form (exact
products of 8-bit digit planes on tcgen05) and the FP64 CUDA-core form,
both against an extended-precision product of the same FP64 inputs, on
ragged row counts, every column count up to 64 and vector scales from 1e-8
to 1e8; then the whole Lanczos solve with either form."""

import numpy as np
import pytest
import torch

import oracle
from helpers import EIG_REL, golden, gpu_problem, preset_inputs

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _basis(n, na, rng):
    q, _ = np.linalg.qr(rng.standard_normal((n, na)))
    return q


def _vectors(n, rng, scales=(1e-8, 1e-3, 1.0, 3.0, 1e2, 1e5, 1e8, 0.5)):
    return rng.standard_normal((n, 8)) * np.array(scales)[None, :]


def _tn_ref(A, B):
    return np.einsum("ku,kv->uv", A.astype(np.longdouble), B.astype(np.longdouble))


@pytest.mark.parametrize("n", [1, 63, 129, 5000, 20001])
@pytest.mark.parametrize("na", [1, 8, 17, 37, 64])
def test_tn_tensor_cores_fp64_accuracy(n, na):
    import paper_2110_10765_gb300 as ci
    rng = np.random.default_rng(n * 131 + na)
    A = _basis(max(n, na), na, rng)[:n] if n >= na else rng.uniform(-1, 1, (n, na))
    B = _vectors(n, rng)
    ref = _tn_ref(A, B)
    bound = 8 * U * _tn_ref(np.abs(A), np.abs(B)) + n * 2.0 ** -58 * np.abs(A).max() * np.abs(B).max(axis=0)
    Ad = torch.zeros((n, 64), dtype=torch.float64, device="cuda")   # the solver's basis row stride
    Ad[:, :na] = torch.from_numpy(A)
    Bd = torch.from_numpy(B).cuda()
    for method in ("tc", "fp64"):
        C = torch.full((na, 8), float("nan"), dtype=torch.float64, device="cuda")
        ci.basis_product("tn", Ad[:, :na], Bd, C, method=method)
        err = np.abs(C.cpu().numpy().astype(np.longdouble) - ref)
        assert np.all(err <= bound), (method, float(np.max(err / bound)))


@pytest.mark.parametrize("n", [1, 127, 128, 129, 20000])
@pytest.mark.parametrize("na", [3, 16, 33, 64])
@pytest.mark.parametrize("beta", [1.0, 0.0])
def test_nn_tensor_cores_fp64_accuracy(n, na, beta):
    import paper_2110_10765_gb300 as ci
    rng = np.random.default_rng(n * 17 + na)
    A = _basis(max(n, na), na, rng)[:n] if n >= na else rng.uniform(-1, 1, (n, na))
    Cm = rng.standard_normal((na, 8)) * np.array([1e-6, 1e-2, 1, 10, 1e3, 1e6, 2.0, 0.25])[None, :]
    B0 = _vectors(n, rng)
    AC = np.einsum("ku,uv->kv", A.astype(np.longdouble), Cm.astype(np.longdouble))
    ref = beta * B0.astype(np.longdouble) - AC
    absAC = np.einsum("ku,uv->kv", np.abs(A), np.abs(Cm))
    bound = 8 * U * (beta * np.abs(B0) + absAC) + na * 2.0 ** -58 * np.abs(Cm).max(axis=0)[None, :]
    Ad = torch.zeros((n, 64), dtype=torch.float64, device="cuda")
    Ad[:, :na] = torch.from_numpy(A)
    Cd = torch.from_numpy(Cm).cuda()
    for method in ("tc", "fp64"):
        Bd = torch.from_numpy(B0).cuda() if beta else torch.full((n, 8), float("nan"), dtype=torch.float64,
                                                                  device="cuda")
        ci.basis_product("nn", Ad[:, :na], Bd, Cd, alpha=-1.0, beta=beta, method=method)
        err = np.abs(Bd.cpu().numpy().astype(np.longdouble) - ref)
        assert np.all(err <= bound), (method, float(np.max(err / bound)))


@pytest.mark.parametrize("na", [5, 40, 64])
def test_tensor_core_products_long_rows(na):
    """400,003 rows: every SM's share of A^T B spans several 1024-row
    accumulation segments, and W = W - A C runs through the stage ring and
    both accumulators many times per SM."""
    import paper_2110_10765_gb300 as ci
    n = 400_003
    rng = np.random.default_rng(na)
    A = rng.uniform(-1, 1, (n, na)) / np.sqrt(n)
    B = _vectors(n, rng)
    Ad = torch.zeros((n, 64), dtype=torch.float64, device="cuda")
    Ad[:, :na] = torch.from_numpy(A)
    Bd = torch.from_numpy(B).cuda()
    C = torch.full((na, 8), float("nan"), dtype=torch.float64, device="cuda")
    ci.basis_product("tn", Ad[:, :na], Bd, C, method="tc")
    ref = _tn_ref(A, B)
    bound = 8 * U * _tn_ref(np.abs(A), np.abs(B)) + n * 2.0 ** -58 * np.abs(A).max() * np.abs(B).max(axis=0)
    err = np.abs(C.cpu().numpy().astype(np.longdouble) - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    Cm = rng.standard_normal((na, 8))
    W = torch.from_numpy(B).cuda()
    ci.basis_product("nn", Ad[:, :na], W, torch.from_numpy(Cm).cuda(), alpha=-1.0, beta=1.0, method="tc")
    rows = np.concatenate([np.arange(300), rng.choice(n, 3000, replace=False), np.arange(n - 300, n)])
    AC = np.einsum("ku,uv->kv", A[rows].astype(np.longdouble), Cm.astype(np.longdouble))
    refw = B[rows].astype(np.longdouble) - AC
    bw = 8 * U * (np.abs(B[rows]) + np.abs(A[rows]) @ np.abs(Cm)) + na * 2.0 ** -58 * np.abs(Cm).max(axis=0)[None, :]
    errw = np.abs(W.cpu().numpy()[rows].astype(np.longdouble) - refw)
    assert np.all(errw <= bw), float(np.max(errw / bw))


@pytest.mark.parametrize("col0", [0, 1])
def test_tn_tensor_cores_strided_operands(col0):
    """A^T B with B a column slice of a wider array (odd row stride) and A
    starting at an odd or even column of its own wider array."""
    import paper_2110_10765_gb300 as ci
    n, na = 7001, 21
    rng = np.random.default_rng(7 + col0)
    A = rng.uniform(-1, 1, (n, na)) / np.sqrt(n)
    Bw = rng.standard_normal((n, 9))
    Ad = torch.zeros((n, 40), dtype=torch.float64, device="cuda")
    Ad[:, col0:col0 + na] = torch.from_numpy(A)
    Bd = torch.from_numpy(Bw).cuda()
    C = torch.full((na, 8), float("nan"), dtype=torch.float64, device="cuda")
    ci.basis_product("tn", Ad[:, col0:col0 + na], Bd[:, 1:9], C, method="tc")
    ref = _tn_ref(A, Bw[:, 1:9])
    bound = 8 * U * _tn_ref(np.abs(A), np.abs(Bw[:, 1:9])) + n * 2.0 ** -58 * np.abs(Bw).max()
    err = np.abs(C.cpu().numpy().astype(np.longdouble) - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_tensor_core_product_range_and_shapes():
    import paper_2110_10765_gb300 as ci
    A = torch.zeros((300, 64), dtype=torch.float64, device="cuda")
    A[:, :8] = 0.1
    A[17, 3] = 2.5                       # outside |a| < 2: refused, nothing faults
    B = torch.ones((300, 8), dtype=torch.float64, device="cuda")
    C = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ci.CIError):
        ci.basis_product("tn", A[:, :8], B, C, method="tc")
    A[17, 3] = 1.0
    ci.basis_product("tn", A[:, :8], B, C, method="tc")
    import math
    ref = math.fsum([0.1] * 299 + [1.0])
    assert np.allclose(C[3].cpu().numpy(), ref, rtol=1e-15, atol=0)
    with pytest.raises(ci.CIError):     # nb != 8
        ci.basis_product("tn", A[:, :8], B[:, :5], torch.zeros((8, 5), dtype=torch.float64, device="cuda"),
                         method="tc")
    with pytest.raises(ci.CIError):     # na > 64
        ci.basis_product("tn", torch.zeros((10, 80), dtype=torch.float64, device="cuda"), B[:10], C, method="tc")
    # the same call after the refusals still works (the context is intact)
    ci.basis_product("tn", A[:, :8], B, C, method="tc")


@pytest.mark.parametrize("case,vt", [("c0", "f64"), ("c2_sub", "f64"), ("c2_sub", "f32"), ("c1", "f32")])
def test_lanczos_tensor_core_products_match_fp64_products(case, vt):
    """The block Lanczos solve with the tensor-core reorthogonalisation
    products gives the golden eigenvalues and agrees with the FP64
    CUDA-core form: to 1e-9 with an FP64 H; with an FP32 H both sit at the
    FP32 matrix's level (its SpMM rounds each product), 1e-7 relative."""
    inp = preset_inputs(case)
    M = gpu_problem(inp).build_H(vt)
    gd = golden()[case]
    k = gd["k"]
    ev_tc, info_tc = M.lowest_eigs(k=k)
    ev_64, info_64 = M.lowest_eigs(k=k, fp64_products=True)
    ref = np.array(gd["lowest"])
    assert np.all(np.abs(ev_tc - ref) <= EIG_REL * np.maximum(np.abs(ref), 1)), ev_tc - ref
    agree = 1e-9 if vt == "f64" else 1e-7
    assert np.all(np.abs(ev_tc - ev_64) <= agree * np.maximum(np.abs(ev_64), 1)), ev_tc - ev_64
    assert max(info_tc["residual"]) <= 10 * max(max(info_64["residual"]), 1e-12 * info_64["hnorm_est"])
