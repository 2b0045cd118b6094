"""Expectation values and transition elements of seeded two-body operators
(Fig. 1, observables step) evaluated on the fly on the GPU, against the
oracle's operator CSR."""

import numpy as np
import pytest

import oracle
import synth
from helpers import inputs, preset_inputs, gpu_problem

pytestmark = pytest.mark.gpu


def _oracle_values(inp, seeds, X, Y=None):
    out, bound = [], []
    for sd in seeds:
        T = synth.tbme_tables(inp["sp"], int(sd), np.float64)
        o = oracle.OracleProblem(inp["sp"], inp["Z"], inp["N"], inp["nmax"], inp["twoM"],
                                 np.zeros(len(inp["sp"]["N"])), T)
        rp, col, val, ab = o.csr()
        out.append(oracle.expectation_values(rp, col, val, X, Y))
        bound.append(oracle.expectation_values(rp, col, np.abs(val), np.abs(X), None if Y is None else np.abs(Y)))
    return np.array(out), np.array(bound)


def _check(inp, seeds, n, xseed=0, transition=False):
    import torch
    g = gpu_problem(inp)
    dim = g.enumerate_basis()
    rng = np.random.default_rng(xseed)
    X = rng.standard_normal((dim, n))
    Y = rng.standard_normal((dim, n)) if transition else None
    a = g.observables(seeds, torch.from_numpy(X).cuda(), None if Y is None else torch.from_numpy(Y).cuda())
    ref, bound = _oracle_values(inp, seeds, X, Y)
    assert a.shape == (len(seeds), n)
    assert np.all(np.abs(a - ref) <= 1e-11 * bound + 1e-300), np.max(np.abs(a - ref) / bound)


@pytest.mark.parametrize("case,n", [((1, 2, 2, -1), 8), ((1, 3, 2, -1), 3), ((2, 2, 2, 1), 5),
                                    ((2, 3, 1, 2), 1), ((2, 1, 1, -1), 8)])
def test_observables_small(case, n):
    _check(inputs(*case, seed=3), [11, 12, 13], n)


def test_observables_config0():
    _check(preset_inputs("c0"), [101, 102, 103, 104], 8, xseed=1)


def test_observables_nmax2_subspace():
    _check(preset_inputs("c2_sub"), [7, 8], 5, xseed=2)


@pytest.mark.parametrize("case,n", [((1, 2, 2, -1), 16), ((2, 2, 2, 1), 11), ((2, 3, 1, 2), 9)])
def test_observables_more_than_eight_vectors(case, n):
    _check(inputs(*case, seed=4), [21, 22], n, xseed=5)


@pytest.mark.parametrize("case,n", [((1, 2, 2, -1), 8), ((2, 2, 2, 1), 13), ((2, 3, 1, 2), 3)])
def test_transition_elements(case, n):
    _check(inputs(*case, seed=6), [31, 32, 33], n, xseed=7, transition=True)


def test_transition_elements_config0():
    _check(preset_inputs("c0"), [105, 106], 16, xseed=8, transition=True)


def test_transition_same_vectors_equal_expectation():
    """Y = X passed explicitly takes the two-buffer route and must give the
    expectation values bit for bit (same kernels, same summation order)."""
    import torch
    inp = inputs(2, 2, 2, 1, seed=6)
    g = gpu_problem(inp)
    dim = g.enumerate_basis()
    X = torch.from_numpy(np.random.default_rng(9).standard_normal((dim, 10))).cuda()
    a = g.observables([41, 42], X)
    b = g.observables([41, 42], X, X.clone())
    assert np.array_equal(a, b)


def test_observables_more_operators_than_one_chunk():
    """70 operators: the library processes them in chunks of 64."""
    _check(inputs(1, 2, 2, -1, seed=3), list(range(200, 270)), 3, xseed=4)


def test_observables_zero_vectors_and_single_operator():
    import torch
    inp = inputs(1, 2, 2, -1, seed=3)
    g = gpu_problem(inp)
    dim = g.enumerate_basis()
    a = g.observables([5], torch.zeros((dim, 4), dtype=torch.float64, device="cuda"))
    assert a.shape == (1, 4) and np.all(a == 0.0)


def test_observables_invalid():
    import torch
    import paper_2110_10765_gb300 as ci
    inp = inputs(1, 2, 2, -1, seed=3)
    g = gpu_problem(inp)
    dim = g.enumerate_basis()
    with pytest.raises(ci.CIError):
        g.observables([1], torch.zeros((dim, 17), dtype=torch.float64, device="cuda"))
    with pytest.raises(ci.CIError):
        g.observables([1], torch.zeros((dim, 2), dtype=torch.float64))       # host X
    with pytest.raises(ci.CIError):
        g.observables([], torch.zeros((dim, 2), dtype=torch.float64, device="cuda"))
    with pytest.raises(ci.CIError):                                            # host Y
        g.observables([1], torch.zeros((dim, 2), dtype=torch.float64, device="cuda"),
                      torch.zeros((dim, 2), dtype=torch.float64))
    with pytest.raises(ValueError):
        g.observables([1], torch.zeros((dim, 2), dtype=torch.float64, device="cuda"),
                      torch.zeros((dim, 3), dtype=torch.float64, device="cuda"))
