"""The allocation-free exclusive scan (ci_exclusive_scan_noalloc).

Some callers cannot allocate device memory: their memory belongs to another
caching allocator or a fixed reservation, or they run on a latency-critical
thread where cudaMalloc / cudaFree would stall on a device synchronisation.
This entry point keeps its scratch in a static device array instead.  Its
results must equal ci_exclusive_scan's, bit for bit (integer offsets), on
consecutive calls that reuse the shared array.  Collected last so that a
failure here does not hide the other tests.
"""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE = 4096          # counts per scan tile
MAX_COUNTS = 65536 * TILE


def _scan(fn, x):
    from paper_2110_10765_gb300 import _lib
    n = x.numel()
    y = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    st = getattr(_lib.lib(), fn)(C.c_void_p(x.data_ptr()), n, C.c_void_p(y.data_ptr()),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st, fn)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("sizes", [(3 * TILE + 123, 5 * TILE + 1), (1, 70001)])
def test_noalloc_scan_matches_scan_on_consecutive_calls(sizes):
    rng = np.random.default_rng(sizes[0])
    for n in sizes:   # two calls in a row: the second reuses the static array
        x = torch.from_numpy(rng.integers(0, 3000, n).astype(np.int32)).cuda()
        ref = _scan("ci_exclusive_scan", x)
        got = _scan("ci_exclusive_scan_noalloc", x)
        assert np.array_equal(got, ref)
        assert got[0] == 0 and got[-1] == int(x.sum())


def test_noalloc_scan_rejects_sizes_beyond_maximum():
    from paper_2110_10765_gb300 import _lib
    L = _lib.lib()
    st = L.ci_exclusive_scan_noalloc(C.c_void_p(16), MAX_COUNTS + 1, C.c_void_p(16), None)
    assert st == 4   # CI_ERR_CAPACITY, nothing launched
    assert b"exceeds the maximum" in L.ci_last_error()
