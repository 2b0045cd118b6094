"""Refinement of Ritz pairs found with an FP32 H by the FP64 Hamiltonian
applied on the fly: the refined eigenvalues against the FP64 oracle's."""

import numpy as np
import pytest
import torch

from helpers import golden, gpu_problem, inputs, preset_inputs

pytestmark = pytest.mark.gpu


def _fp32_then_refine(inp, k, iters, **kw):
    g = gpu_problem(inp)
    M = g.build_H("f32")
    E = torch.zeros((M.dim, k), dtype=torch.float64, device="cuda")
    ev32, info = M.lowest_eigs(k=k, evecs=E, **kw)
    ev, rn = g.refine_eigs(E, iters=iters)
    return g, M, E, ev32, ev, rn


def test_refine_config0_recovers_fp64_digits():
    ref = np.array(golden()["c0"]["lowest"])
    g, M, E, ev32, ev, rn = _fp32_then_refine(preset_inputs("c0"), 5, 2, tol=1e-7)
    e32 = np.max(np.abs(ev32 - ref))
    e64 = np.max(np.abs(ev - ref))
    print("config 0: FP32 error", e32, "refined", e64, "residuals", rn)
    assert e64 <= 1e-8 * np.max(np.abs(ref))
    assert e64 < e32 / 10
    V = E.cpu().numpy()
    assert np.allclose(V.T @ V, np.eye(5), atol=1e-10)


def test_refine_config1_recovers_fp64_digits():
    ref = np.array(golden()["c1"]["lowest"])
    g, M, E, ev32, ev, rn = _fp32_then_refine(preset_inputs("c1"), 5, 2)
    e32 = np.max(np.abs(ev32 - ref))
    e64 = np.max(np.abs(ev - ref))
    print("config 1: FP32 error", e32, "refined", e64, "residuals", rn)
    assert e64 <= 1e-7 * np.max(np.abs(ref))
    assert e64 < e32 / 10


def test_refine_degenerate_closed_form():
    """Zero interaction: the lowest level 320 MeV is 51-fold; the refined
    Ritz values are 320 to FP64 rounding (their error is quadratic in the
    vectors' residual components on the higher levels, which one step only
    reduces)."""
    inp = inputs(1, 4, 4, -1, zero=True)
    g, M, E, ev32, ev, rn = _fp32_then_refine(inp, 5, 1)
    assert np.allclose(ev, 320.0, rtol=0, atol=1e-10)
    assert np.all(rn <= 1e-4)


@pytest.mark.parametrize("k,iters", [(1, 0), (3, 1), (12, 1)])
def test_refine_sizes(k, iters):
    inp = inputs(2, 3, 3, 2, seed=4)
    g = gpu_problem(inp)
    M64 = g.build_H("f64")
    ref, _ = M64.lowest_eigs(k=k, block=8 if k <= 8 else 8, max_basis=64 if k <= 8 else 96, tol=1e-11)
    M = g.build_H("f32")
    E = torch.zeros((M.dim, k), dtype=torch.float64, device="cuda")
    M.lowest_eigs(k=k, evecs=E, max_basis=64 if k <= 8 else 96)
    ev, rn = g.refine_eigs(E, iters=iters)
    assert np.all(np.abs(ev - ref) <= 1e-7 * np.maximum(np.abs(ref), 1)), ev - ref


def test_refine_invalid():
    import paper_2110_10765_gb300 as ci
    g = gpu_problem(inputs(1, 2, 2, -1, seed=1))
    dim = g.enumerate_basis()
    with pytest.raises(ci.CIError):
        g.refine_eigs(torch.zeros((dim, 17), dtype=torch.float64, device="cuda"))
    with pytest.raises(ci.CIError):
        g.refine_eigs(torch.zeros((dim, 2), dtype=torch.float64))                 # host vectors
    with pytest.raises(ci.CIError):
        g.refine_eigs(torch.zeros((dim, 2), dtype=torch.float64, device="cuda"))  # dependent (zero) vectors
