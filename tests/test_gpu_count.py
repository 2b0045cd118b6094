"""Count benchmark (Sec. 2.1, Listings 1-2) on the GPU against the oracle.

Every form of the pair test (64-state prefilter + MBS, MBS only, full bit
representation) must give the oracle's per-state counts exactly."""

import itertools

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

VARIANTS = ["hybrid", "mbs", "bits"]


def _gpu_counts(mbs, S, variant, max_diff=4):
    import torch
    import paper_2110_10765_gb300 as ci
    n = len(mbs)
    d = torch.from_numpy(mbs.view(np.int16)).cuda() if n else torch.zeros((0, mbs.shape[1]), dtype=torch.int16,
                                                                            device="cuda")
    rc = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    total = ci.count_pairs(d, S, variant, max_diff, row_counts=rc[:n] if n else None)
    return total, rc[:n].cpu().numpy()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("max_diff", [4, 6, 0])
def test_count_pairs_match_oracle(variant, max_diff):
    mbs = synth.e1_states(5003, N=8, S=128, r=0.93, seed=11)   # ragged n, denser than the benchmark
    ref = oracle.count_pairs(mbs, max_diff=max_diff)
    total, rows = _gpu_counts(mbs, 128, variant, max_diff)
    assert np.array_equal(rows, ref)
    assert total == int(ref.sum())


@pytest.mark.parametrize("variant", VARIANTS)
def test_count_pairs_closed_form(variant):
    mbs = np.array(list(itertools.combinations(range(10), 4)), np.uint16)
    total, rows = _gpu_counts(mbs, 10, variant)
    assert np.all(rows == 1 + 4 * 6 + 6 * 15)
    assert total == len(mbs) * 115


@pytest.mark.parametrize("N,S,variant", [(4, 128, "mbs"), (12, 128, "mbs"), (16, 128, "mbs"), (20, 128, "mbs"),
                                         (5, 128, "mbs"), (20, 128, "hybrid"), (12, 100, "bits"),
                                         (3, 40, "hybrid")])
def test_count_pairs_particle_numbers(N, S, variant):
    mbs = synth.e1_states(3001, N=N, S=S, r=0.9, seed=N)
    ref = oracle.count_pairs(mbs)
    total, rows = _gpu_counts(mbs, S, variant)
    assert np.array_equal(rows, ref)


@pytest.mark.parametrize("variant", VARIANTS)
def test_count_pairs_edges(variant):
    one = np.array([[1, 5, 9, 70]], np.uint16)
    assert _gpu_counts(one, 128, variant)[0] == 1
    dup = np.array([[0, 1, 2, 3], [0, 1, 2, 3], [0, 1, 2, 4], [10, 11, 12, 13]], np.uint16)
    total, rows = _gpu_counts(dup, 128, variant)
    assert rows.tolist() == [3, 3, 3, 1] and total == 10
    assert _gpu_counts(np.zeros((0, 4), np.uint16), 128, variant)[0] == 0


def test_count_pairs_benchmark_size_sampled():
    """Full benchmark size: the three forms agree on the total and on sampled
    rows, which match the oracle."""
    n = 131072
    mbs = synth.e1_states(n, N=8, S=128, seed=1)
    rows = np.unique(np.concatenate([np.random.default_rng(0).integers(0, n, 150), [0, n - 1]]))
    ref = oracle.count_pairs(mbs, rows=rows)
    totals = []
    for v in VARIANTS:
        total, rc = _gpu_counts(mbs, 128, v)
        assert np.array_equal(rc[rows], ref)
        totals.append(total)
    assert len(set(totals)) == 1 and totals[0] >= n


def test_count_pairs_invalid_args():
    import torch
    import paper_2110_10765_gb300 as ci
    d = torch.zeros((4, 4), dtype=torch.int16, device="cuda")
    with pytest.raises(ci.CIError):
        ci.count_pairs(d, 200, "bits")           # bit form needs S <= 128
    with pytest.raises(ci.CIError):
        ci.count_pairs(d, 128, 7)                # unknown variant
    with pytest.raises(ci.CIError):
        ci.count_pairs(d.cpu(), 128, "hybrid")   # host pointer
    with pytest.raises(ci.CIError):
        ci.count_pairs(d, 128, "hybrid", max_diff=-2)
