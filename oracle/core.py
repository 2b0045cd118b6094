"""ctypes wrapper of the FP64 C oracle (``ci_oracle.c``).  Test infrastructure.

``build_library()`` compiles ``ci_oracle.c`` with the host gcc into
``oracle/_build/`` (git-ignored) and is called lazily on first use.
"""

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ci_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libci_oracle.so")
_lib = None
_lock = threading.Lock()


def build_library(force=False):
    """Compile the C oracle (gcc, -O2, OpenMP) if missing or out of date."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("S", C.c_int), ("sp_N", C.POINTER(C.c_int)),
                ("sp_twom", C.POINTER(C.c_int)), ("eps", C.POINTER(C.c_double)),
                ("Vpp", C.POINTER(C.c_double)), ("Vnn", C.POINTER(C.c_double)),
                ("Vpn", C.POINTER(C.c_double)), ("A", C.c_int * 2),
                ("nmax", C.c_int), ("twoM", C.c_int), ("seed", C.c_uint64),
                ("round_f32", C.c_int)]


class _Species(C.Structure):
    _fields_ = [("A", C.c_int), ("n", C.c_int64), ("occ", C.POINTER(C.c_uint8)),
                ("q", C.POINTER(C.c_int)), ("twoM", C.POINTER(C.c_int))]


class _BasisView(C.Structure):
    _fields_ = [("pr", C.POINTER(_Problem)), ("sp", C.POINTER(_Species) * 2),
                ("dim", C.c_int64), ("p_idx", C.POINTER(C.c_int32)),
                ("n_idx", C.POINTER(C.c_int32))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build_library())
            P = C.POINTER
            lib.orc_species_build.argtypes = [P(_Problem), C.c_int, P(_Species)]
            lib.orc_species_free.argtypes = [P(_Species)]
            lib.orc_basis.argtypes = [P(_Problem), P(_Species), P(_Species),
                                      C.c_void_p, C.c_void_p]
            lib.orc_basis.restype = C.c_int64
            lib.orc_count_difference.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
            lib.orc_element.argtypes = [P(_Problem)] + [C.c_void_p] * 4 + [P(C.c_double)]
            lib.orc_element.restype = C.c_double
            lib.orc_row.argtypes = [P(_BasisView), C.c_int64, C.c_int64] + [C.c_void_p] * 6
            lib.orc_row.restype = C.c_int64
            lib.orc_row_counts.argtypes = [P(_BasisView), C.c_void_p]
            lib.orc_fill.argtypes = [P(_BasisView)] + [C.c_void_p] * 4
            lib.orc_row_counts_range.argtypes = [P(_BasisView), C.c_int64, C.c_int64, C.c_void_p]
            lib.orc_fill_range.argtypes = [P(_BasisView), C.c_int64, C.c_int64] + [C.c_void_p] * 4
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_set_threads.restype = C.c_int
            lib.orc_spmm.argtypes = [C.c_int64] + [C.c_void_p] * 5 + [C.c_int]
            lib.orc_exclusive_scan.argtypes = [C.c_void_p, C.c_int64, C.c_void_p]
            lib.orc_count_pairs.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_int64,
                                            C.c_void_p]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class OracleProblem:
    """One CI problem: s.p. table, particle numbers, cuts and interaction.

    ``tables`` holds the flat ``pp``, ``nn``, ``pn`` TBME tables in any float
    dtype; they are widened to float64 exactly.  Without tables, ``seed``
    draws every TBME on demand from the counter-based SplitMix64 recipe
    (each draw rounded to float32 when ``round_f32``), so that no S**4 table
    is held.  ``eps`` are the one-body energies [S].
    """

    def __init__(self, sp, Z, N, nmax, twoM, eps, tables=None, seed=None, round_f32=True):
        self.lib = _load()
        self.S = int(len(sp["N"]))
        self.sp_N = np.ascontiguousarray(sp["N"], dtype=np.int32).astype(np.intc)
        self.sp_twom = np.ascontiguousarray(sp["twom"], dtype=np.int32).astype(np.intc)
        self.eps = np.ascontiguousarray(eps, dtype=np.float64)
        self.Z, self.N, self.nmax, self.twoM = int(Z), int(N), int(nmax), int(twoM)
        if tables is not None:
            self.V = {k: np.ascontiguousarray(tables[k], dtype=np.float64) for k in ("pp", "nn", "pn")}
            for k, v in self.V.items():
                if v.size != self.S ** 4:
                    raise ValueError("table %s must have S**4 entries" % k)
            vp = [_dptr(self.V[k]) for k in ("pp", "nn", "pn")]
            seed, round_f32 = 0, False
        else:
            if seed is None:
                raise ValueError("give TBME tables or a seed")
            self.V = None
            vp = [None, None, None]
        self._pr = _Problem(self.S, _iptr(self.sp_N), _iptr(self.sp_twom), _dptr(self.eps),
                            vp[0], vp[1], vp[2],
                            (C.c_int * 2)(self.Z, self.N), self.nmax, self.twoM,
                            int(seed) & 0xFFFFFFFFFFFFFFFF, int(bool(round_f32)))
        self._sp = [_Species(), _Species()]
        for s in (0, 1):
            if self.lib.orc_species_build(C.byref(self._pr), s, C.byref(self._sp[s])) != 0:
                raise ValueError("bad particle number")
        n = self.lib.orc_basis(C.byref(self._pr), C.byref(self._sp[0]), C.byref(self._sp[1]), None, None)
        self.dim = int(n)
        self.p_idx = np.zeros(max(n, 1), dtype=np.int32)
        self.n_idx = np.zeros(max(n, 1), dtype=np.int32)
        self.lib.orc_basis(C.byref(self._pr), C.byref(self._sp[0]), C.byref(self._sp[1]),
                           _ptr(self.p_idx), _ptr(self.n_idx))
        self.p_idx = self.p_idx[:n]
        self.n_idx = self.n_idx[:n]
        self._bv = _BasisView()
        self._bv.pr = C.pointer(self._pr)
        self._bv.sp[0] = C.pointer(self._sp[0])
        self._bv.sp[1] = C.pointer(self._sp[1])
        self._bv.dim = self.dim
        self._bv.p_idx = self.p_idx.ctypes.data_as(C.POINTER(C.c_int32))
        self._bv.n_idx = self.n_idx.ctypes.data_as(C.POINTER(C.c_int32))
        self._species_cache = {}

    def __del__(self):
        try:
            for s in self._sp:
                self.lib.orc_species_free(C.byref(s))
        except Exception:
            pass

    # -- species lists -------------------------------------------------
    def species(self, s):
        """dict with ``occ`` [n, A] uint8, ``q``, ``twoM``, ``bits`` [n, W] uint64."""
        if s in self._species_cache:
            return self._species_cache[s]
        sp = self._sp[s]
        n, A = int(sp.n), int(sp.A)
        occ = (np.ctypeslib.as_array(sp.occ, shape=(n * A,)).reshape(n, A).copy()
               if n * A else np.zeros((n, A), np.uint8))
        q = np.ctypeslib.as_array(sp.q, shape=(n,)).copy() if n else np.zeros(0, np.intc)
        m = np.ctypeslib.as_array(sp.twoM, shape=(n,)).copy() if n else np.zeros(0, np.intc)
        W = (self.S + 63) // 64
        bits = np.zeros((n, W), dtype=np.uint64)
        for i in range(n):
            for o in occ[i]:
                bits[i, o // 64] |= np.uint64(1) << np.uint64(o % 64)
        out = {"occ": occ, "q": q.astype(np.int32), "twoM": m.astype(np.int32), "bits": bits}
        self._species_cache[s] = out
        return out

    # -- matrix ----------------------------------------------------------
    def element(self, i, j):
        """(<Phi_i|H|Phi_j>, sum of |terms|)."""
        P, Nn = self.species(0)["occ"], self.species(1)["occ"]
        pb = np.ascontiguousarray(P[self.p_idx[i]]); nb = np.ascontiguousarray(Nn[self.n_idx[i]])
        pk = np.ascontiguousarray(P[self.p_idx[j]]); nk = np.ascontiguousarray(Nn[self.n_idx[j]])
        ab = C.c_double()
        v = self.lib.orc_element(C.byref(self._pr), _ptr(pb), _ptr(nb), _ptr(pk), _ptr(nk), C.byref(ab))
        return v, ab.value

    def row(self, i):
        """Row i: (cols int64, vals f64, absums f64, total difference int8)."""
        scr_p = np.zeros(max(int(self._sp[0].n), 1), np.uint8)
        scr_n = np.zeros(max(int(self._sp[1].n), 1), np.uint8)
        n = self.lib.orc_row(C.byref(self._bv), int(i), 0, None, None, None, None,
                             _ptr(scr_p), _ptr(scr_n))
        cols = np.zeros(n, np.int64); vals = np.zeros(n); ab = np.zeros(n); d = np.zeros(n, np.int8)
        self.lib.orc_row(C.byref(self._bv), int(i), n, _ptr(cols), _ptr(vals), _ptr(ab), _ptr(d),
                         _ptr(scr_p), _ptr(scr_n))
        return cols, vals, ab, d

    def row_counts(self):
        cnt = np.zeros(max(self.dim, 1), np.int64)
        self.lib.orc_row_counts(C.byref(self._bv), _ptr(cnt))
        return cnt[: self.dim]

    def csr(self, with_absums=True):
        """Full H as (row_ptr int64, cols int64, vals f64, absums f64|None)."""
        cnt = self.row_counts()
        row_ptr = exclusive_scan(cnt)
        nnz = int(row_ptr[-1])
        cols = np.zeros(max(nnz, 1), np.int64); vals = np.zeros(max(nnz, 1))
        ab = np.zeros(max(nnz, 1)) if with_absums else None
        self.lib.orc_fill(C.byref(self._bv), _ptr(row_ptr), _ptr(cols), _ptr(vals),
                          _ptr(ab) if with_absums else None)
        return row_ptr, cols[:nnz], vals[:nnz], (ab[:nnz] if with_absums else None)

    def csr_rows(self, i0, i1):
        """Rows i0 <= i < i1 of H as a CSR slab (row_ptr from 0, global
        column indices, FP64 values): the count, scan and fill of Fig. 1
        restricted to those rows."""
        i0, i1 = int(i0), int(min(i1, self.dim))
        cnt = np.zeros(max(i1 - i0, 1), np.int64)
        self.lib.orc_row_counts_range(C.byref(self._bv), i0, i1, _ptr(cnt))
        row_ptr = exclusive_scan(cnt[: i1 - i0])
        nnz = int(row_ptr[-1])
        cols = np.zeros(max(nnz, 1), np.int64); vals = np.zeros(max(nnz, 1))
        self.lib.orc_fill_range(C.byref(self._bv), i0, i1, _ptr(row_ptr), _ptr(cols), _ptr(vals), None)
        return row_ptr, cols[:nnz], vals[:nnz]

    def count_difference(self, s, a, b):
        occ = self.species(s)["occ"]
        x = np.ascontiguousarray(occ[a]); y = np.ascontiguousarray(occ[b])
        return self.lib.orc_count_difference(_ptr(x), _ptr(y), occ.shape[1])


def expectation_values(row_ptr, cols, vals, X, Y=None):
    """a[v] = sum_ij X[i, v] O_ij Y[j, v] for a CSR operator O (Fig. 1,
    observables step: Eq. 2 with the eigenvectors c_i; Y = None means Y = X,
    the expectation values, another Y gives transition elements): the rows
    of O Y, dotted with X column by column (the SpMM of ``spmm`` is the one
    product)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    if Y is None:
        Y = X
    else:
        Y = np.asarray(Y, dtype=np.float64)
        if Y.ndim == 1:
            Y = Y[:, None]
        if Y.shape != X.shape:
            raise ValueError("X and Y must have the same shape")
    OY = spmm(row_ptr, cols, vals, Y)
    return np.einsum("iv,iv->v", X, OY)


def set_threads(n=0):
    """OpenMP threads of the oracle's row loops (n <= 0 keeps the default);
    returns the count in use."""
    return int(_load().orc_set_threads(int(n)))


def count_pairs(mbs, rows=None, max_diff=4):
    """Count benchmark of Sec. 2.1 (Listing 2): for each state i in rows (all
    states by default) the number of states j of mbs [n][N] (uint16,
    ascending) that differ from it in at most max_diff s.p. states."""
    lib = _load()
    mbs = np.ascontiguousarray(mbs, dtype=np.uint16)
    n, N = mbs.shape
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(len(rows), np.int64)
    lib.orc_count_pairs(_ptr(mbs), n, N, max_diff, _ptr(rows), len(rows), _ptr(out))
    return out


def exclusive_scan(x):
    """Exclusive prefix sum with the total appended (Eq. 1), int64."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.int64)
    y = np.zeros(len(x) + 1, np.int64)
    lib.orc_exclusive_scan(_ptr(x), len(x), _ptr(y))
    return y


def spmm(row_ptr, cols, vals, X):
    """Y = H X in FP64 for a CSR H and row-major X [dim, nvec]."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    dim, nvec = X.shape
    Y = np.zeros_like(X)
    lib.orc_spmm(dim, _ptr(np.ascontiguousarray(row_ptr, np.int64)),
                 _ptr(np.ascontiguousarray(cols, np.int64)),
                 _ptr(np.ascontiguousarray(vals, np.float64)), _ptr(X), _ptr(Y), nvec)
    return Y
