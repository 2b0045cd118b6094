"""Pins of the oracle's motif definitions (Sec. 2.3-2.4) against closed
forms."""

import numpy as np
import pytest

import oracle

O = oracle.motifs


@pytest.mark.parametrize("m,p", [(512, 1), (100, 3), (31, 32), (0, 1), (7, 7)])
def test_fill_shared_rows_are_the_multiples_of_p(m, p):
    cnt = m // p
    offset = np.arange(5, dtype=np.int64) * (cnt + 2)            # gaps of two between the rows
    arr = O.fill_shared(offset, m, p, 5 * (cnt + 2))
    for i in range(5):
        row = arr[offset[i]: offset[i] + cnt + 2]
        assert np.array_equal(row[:cnt], np.arange(1, cnt + 1) * p)
        assert np.all(row[cnt:] == -1)                          # the gap is untouched


@pytest.mark.parametrize("n,m", [(1, 8), (5, 16), (33, 64), (7, 3)])
def test_array_reduction_is_the_product_of_column_sums(n, m):
    rng = np.random.default_rng(n * m)
    x = rng.standard_normal((n, m))
    y = rng.standard_normal((n, m))
    a = O.array_reduction(x, y)
    assert np.allclose(a, x.sum(0) * y.sum(0), rtol=1e-12, atol=1e-12)
    # linearity and the swap of x and y
    assert np.allclose(O.array_reduction(2 * x, y), 2 * a, rtol=1e-12)
    assert np.allclose(O.array_reduction(y, x), a, rtol=1e-12, atol=1e-12)
