"""The motif benchmarks of Sec. 2.2-2.4 on the GPU against the oracle:
serial and parallel scans and the shared-array fill bit-exact, the
small-array reduction within its FP32 summation bound."""

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [0, 1, 7, 8, 9, 1000, 123457])
def test_serial_scan_bit_exact(n):
    import paper_2110_10765_gb300 as ci
    c = np.random.default_rng(n).integers(0, 1000, n).astype(np.int32)
    d = torch.from_numpy(c).cuda()
    o1 = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    o2 = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ci.scan_serial(d, o1)
    ci.exclusive_scan(d, o2)
    ref = oracle.exclusive_scan(c)
    assert np.array_equal(o1.cpu().numpy(), ref) and np.array_equal(o2.cpu().numpy(), ref)


@pytest.mark.parametrize("n,m,p,gap", [(1000, 512, 1, 0), (777, 100, 3, 2), (5, 0, 1, 1), (33, 31, 32, 0),
                                       (4097, 65, 2, 5)])
def test_fill_shared_bit_exact(n, m, p, gap):
    import paper_2110_10765_gb300 as ci
    cnt = m // p
    offset = np.arange(n, dtype=np.int64) * (cnt + gap)
    size = max(n * (cnt + gap), 1)
    arr = torch.full((size,), -1, dtype=torch.int32, device="cuda")
    ci.fill_shared(torch.from_numpy(offset).cuda(), m, p, arr)
    assert np.array_equal(arr.cpu().numpy(), oracle.motifs.fill_shared(offset, m, p, size))


@pytest.mark.parametrize("n,m", [(1, 8), (63, 16), (64, 64), (65, 256), (1000, 64), (300, 32), (129, 128)])
def test_array_reduction_against_oracle(n, m):
    import paper_2110_10765_gb300 as ci
    rng = np.random.default_rng(n + m)
    x = rng.standard_normal((n, m)).astype(np.float32)
    y = rng.standard_normal((n, m)).astype(np.float32)
    a = ci.array_reduction(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
    ref = oracle.motifs.array_reduction(x, y) if n <= 65 else x.astype(np.float64).sum(0) * y.astype(np.float64).sum(0)
    bound = np.abs(x).astype(np.float64).sum(0) * np.abs(y).astype(np.float64).sum(0)
    assert np.all(np.abs(a - ref) <= 1e-4 * bound + 1e-6), np.max(np.abs(a - ref) / bound)


def test_motifs_invalid():
    import paper_2110_10765_gb300 as ci
    x = torch.zeros((4, 12), dtype=torch.float32, device="cuda")
    with pytest.raises(ci.CIError):
        ci.array_reduction(x, x)                                 # m = 12
    with pytest.raises(ci.CIError):
        ci.array_reduction(x[:, :8].contiguous().cpu(), x[:, :8].contiguous())   # host x
    with pytest.raises(ci.CIError):
        ci.fill_shared(torch.zeros(3, dtype=torch.int64, device="cuda"), 8, 0,
                       torch.zeros(30, dtype=torch.int32, device="cuda"))        # p = 0
    c = torch.zeros(5, dtype=torch.int32)
    with pytest.raises(ci.CIError):
        ci.scan_serial(c, torch.zeros(6, dtype=torch.int64, device="cuda"))    # host counts
