"""Kernel tracing: every launch counted, CUDA-event durations on every launch
or on a sample of them."""

import numpy as np
import pytest
import torch

from helpers import gpu_problem, inputs

pytestmark = pytest.mark.gpu


def _spmm_runs(M, n):
    X = torch.randn((M.dim, 8), device="cuda")
    Y = torch.empty_like(X)
    for _ in range(n):
        M.apply_H(X, Y)
    torch.cuda.synchronize()


def test_trace_counts_and_sampling():
    import paper_2110_10765_gb300 as ci
    M = gpu_problem(inputs(2, 3, 3, 2, seed=2)).build_H("f32")
    ci.trace_enable(True)
    ci.trace_read(reset=True)
    _spmm_runs(M, 10)
    full = ci.trace_read(reset=True)
    assert full["k_spmm"][0] == 10 and full["k_spmm"][1] > 0
    ci.trace_enable(True, sample=4)             # launches 1, 5, 9 timed
    _spmm_runs(M, 10)
    sampled = ci.trace_read(reset=True)
    assert sampled["k_spmm"][0] == 10 and sampled["k_spmm"][1] > 0
    mean_full, mean_sampled = full["k_spmm"][1] / 10, sampled["k_spmm"][1] / 10
    assert 0.2 < mean_sampled / mean_full < 5.0
    ci.trace_enable(False)
    _spmm_runs(M, 3)
    assert ci.trace_read(reset=True) == {}
