"""The paper's motif benchmarks (Sec. 2.3-2.4) as plain definitions.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``fill_shared``: Listing 7's motif.  Row i stores every j in 1..m with
  j mod p == 0, in ascending order, at arr[offset[i]], arr[offset[i] + 1], ...
  (the listing's atomic counter, taken one j after another).
* ``array_reduction``: Eq. 2's small-array reduction in the benchmark form of
  Listings 8-9, a[k] = sum over all pairs (i, j) of x[i, k] * y[j, k], in
  FP64, by the double loop over the pairs.
"""

import numpy as np


def fill_shared(offset, m, p, size, fill=-1):
    """arr [size] int32 (untouched entries = fill) after the fill."""
    arr = np.full(size, fill, dtype=np.int32)
    for i, off in enumerate(np.asarray(offset, dtype=np.int64)):
        k = int(off)
        for j in range(1, m + 1):
            if j % p == 0:
                arr[k] = j
                k += 1
    return arr


def array_reduction(x, y):
    """a [m] float64 for x, y [n, m] (row i = the listings' column x(:, i))."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, m = x.shape
    a = np.zeros(m)
    for i in range(n):
        for j in range(n):
            a += x[i] * y[j]
    return a
