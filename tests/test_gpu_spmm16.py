"""The 16-vector product (LOBPCG's H [X P], Fig. 2 optional FMA with two
8-vector blocks side by side) against two 8-vector products of the same
halves and against the oracle's FP64 product: FP32 and BF16-row-scale H,
rows of every length (the kernel's tail loop), through ci_apply_H."""

import numpy as np
import pytest
import torch

import oracle
from helpers import REL32, gpu_problem, inputs, oracle_problem, preset_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["c2_sub", (2, 2, 3, 2), (1, 1, 1, -1)])
@pytest.mark.parametrize("vt", ["f32", "bf16"])
def test_spmm16_matches_two_8_vector_products(case, vt):
    inp = preset_inputs(case) if isinstance(case, str) else inputs(*case, seed=6)
    o = oracle_problem(inp)
    M = gpu_problem(inp).build_H(vt)
    rng = np.random.default_rng(16)
    X = rng.standard_normal((M.dim, 16)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Y16 = torch.full((M.dim, 16), float("nan"), device="cuda")
    M.apply_H(Xd, Y16)
    halves = []
    for h in range(2):
        Xh = Xd[:, 8 * h:8 * h + 8].contiguous()
        Yh = torch.empty_like(Xh)
        M.apply_H(Xh, Yh)
        halves.append(Yh)
    Y8 = torch.cat(halves, dim=1).cpu().numpy().astype(np.float64)
    Y = Y16.cpu().numpy().astype(np.float64)
    rp, col, val, ab = o.csr()
    absH = oracle.spmm(rp, col, np.maximum(np.abs(val), ab), np.abs(X.astype(np.float64)))
    # same stored values, another summation order: FP32 rounding only
    nmax = int(np.max(np.diff(rp)))
    assert np.all(np.abs(Y - Y8) <= 2 * nmax * 2.0 ** -24 * absH + 1e-30), np.max(np.abs(Y - Y8) / (absH + 1e-30))
    # against the FP64 product of the oracle's H: the element bound of the
    # stored values (FP32: 1e-6; BF16 with row scale: 2^-9) plus accumulation
    ref = oracle.spmm(rp, col, val, X.astype(np.float64))
    rel = REL32 if vt == "f32" else 2.0 ** -8
    assert np.all(np.abs(Y - ref) <= (rel + 2 * nmax * 2.0 ** -24) * absH + 1e-30)


def test_spmm16_rejects_other_shapes():
    import paper_2110_10765_gb300 as ci
    inp = inputs(1, 2, 2, -1, seed=1, dtype=np.float64)
    M = gpu_problem(inp).build_H("f64")
    X = torch.zeros((M.dim, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(ci.CIError):
        M.apply_H(X, torch.empty_like(X))
    M32 = gpu_problem(inputs(1, 2, 2, -1, seed=1)).build_H("f32")
    X = torch.zeros((M32.dim, 12), device="cuda")
    with pytest.raises(ci.CIError):
        M32.apply_H(X, torch.empty_like(X))
