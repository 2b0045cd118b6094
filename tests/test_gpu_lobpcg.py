"""LOBPCG (Fig. 1, eigensolve: the paper names LOBPCG beside Lanczos) against
the oracle's eigenvalues."""

import numpy as np
import pytest
import torch

import oracle
from helpers import EIG_REL, golden, gpu_problem, inputs, oracle_problem, preset_inputs

pytestmark = pytest.mark.gpu


def test_lobpcg_config0_fp64():
    M = gpu_problem(preset_inputs("c0")).build_H("f64")
    ev, info = M.lowest_eigs(k=5, method="lobpcg")
    ref = np.array(golden()["c0"]["lowest"])
    assert np.all(np.abs(ev - ref) <= 1e-8 * np.maximum(np.abs(ref), 1)), ev - ref
    assert max(info["residual"]) <= 1e-8 * info["hnorm_est"]


def test_lobpcg_nmax2_subspace_fp32_vectors():
    M = gpu_problem(preset_inputs("c2_sub")).build_H("f32")
    E = torch.zeros((M.dim, 6), dtype=torch.float64, device="cuda")
    ev, info = M.lowest_eigs(k=6, block=8, method="lobpcg", evecs=E)
    ref = np.array(golden()["c2_sub"]["lowest"])[:6]
    assert np.all(np.abs(ev - ref) <= EIG_REL * np.maximum(np.abs(ref), 1)), ev - ref
    V = E.cpu().numpy()
    assert np.allclose(V.T @ V, np.eye(6), atol=1e-6)


def test_lobpcg_config1_fp32():
    M = gpu_problem(preset_inputs("c1")).build_H("f32")
    ev, info = M.lowest_eigs(k=5, method="lobpcg")
    ref = np.array(golden()["c1"]["lowest"])
    assert np.all(np.abs(ev - ref) <= EIG_REL * np.maximum(np.abs(ref), 1)), ev - ref


def test_lobpcg_degenerate_closed_form():
    """Zero interaction: the lowest level (320 MeV) is 51-fold."""
    inp = inputs(1, 4, 4, -1, zero=True, dtype=np.float64)
    M = gpu_problem(inp).build_H("f64")
    ev, info = M.lowest_eigs(k=5, method="lobpcg")
    assert np.allclose(ev, 320.0, rtol=0, atol=1e-8)


@pytest.mark.parametrize("case", [(1, 2, 2, -1), (2, 2, 1, 1), (2, 3, 2, 2)])
def test_lobpcg_small_against_dense(case):
    inp = inputs(*case, seed=9, dtype=np.float64)
    o = oracle_problem(inp)
    M = gpu_problem(inp).build_H("f64")
    k = min(3, o.dim)
    ev, info = M.lowest_eigs(k=k, block=4, method="lobpcg")
    ref = oracle.lowest_dense(oracle.dense_from_csr(*o.csr()[:3], o.dim), k)
    assert np.allclose(ev, ref, atol=1e-8)


def test_lobpcg_invalid():
    import paper_2110_10765_gb300 as ci
    M = gpu_problem(preset_inputs("c0")).build_H("f64")
    with pytest.raises(ci.CIError):
        M.lowest_eigs(k=6, block=4, method="lobpcg")
