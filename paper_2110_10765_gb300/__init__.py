"""GB300 (sm_103a) library for the hot path of MFDn-style configuration
interaction: bit-string basis, XOR+popcount filter, count -> scan -> fill of
the sparse Hamiltonian, SpMM and block Lanczos, behind the C ABI of
``include/mfdci.h``.

This module is the thin Python binding: the functions carry the C names
(``enumerate_basis``, ``count_nnz``, ``build_H``, ``apply_H``,
``lowest_eigs``, ...) and only marshal arguments.  Device buffers are torch
CUDA tensors (PyTorch provides memory and streams only); host arrays are
numpy arrays.
"""

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (CIError, CI_F32, CI_F64, CI_BF16_ROWSCALE, CI_TBME_TABLES,
                   CI_TBME_SEED, check, lib)

__all__ = ["Problem", "Matrix", "Batch", "Queue", "basis_product", "exclusive_scan", "count_pairs", "COUNT_VARIANTS", "trace_enable", "trace_read", "CIError", "CI_F32", "CI_F64",
           "CI_BF16_ROWSCALE", "VTYPES", "lib", "current_stream"]

VTYPES = {"f32": CI_F32, "f64": CI_F64, "bf16": CI_BF16_ROWSCALE}


def current_stream():
    """cudaStream_t of torch's current stream, as an int (0 = default)."""
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


def _stream(stream):
    if stream is None:
        return C.c_void_p(current_stream())
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(int(stream.cuda_stream))
    return C.c_void_p(int(stream))


def _ptr(x):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(x.data_ptr())


class Problem:
    """A CI problem (``ci_problem``).

    sp: dict with int arrays ``N``, ``twom`` (HO shell and 2m of each s.p.
    state); eps: one-body energies; tables: dict ``pp``/``nn``/``pn`` of flat
    S**4 numpy arrays or torch tensors (float32 or float64), or None with
    ``seed`` to draw the TBMEs on the device.
    """

    def __init__(self, sp, Z, N, nmax, twoM, eps, tables=None, seed=None):
        L = lib()
        S = len(sp["N"])
        self._keep = []
        spN = np.ascontiguousarray(sp["N"], dtype=np.int32)
        spm = np.ascontiguousarray(sp["twom"], dtype=np.int32)
        e = np.ascontiguousarray(eps, dtype=np.float64)
        self._keep += [spN, spm, e]
        d = _lib.ProblemDesc()
        d.n_sp = S
        d.sp_N = spN.ctypes.data_as(C.POINTER(C.c_int32))
        d.sp_twom = spm.ctypes.data_as(C.POINTER(C.c_int32))
        d.sp_energy = e.ctypes.data_as(C.POINTER(C.c_double))
        d.Z, d.N, d.nmax, d.twoM = int(Z), int(N), int(nmax), int(twoM)
        if tables is not None:
            d.tbme_source = CI_TBME_TABLES
            arrs = []
            for k in ("pp", "nn", "pn"):
                t = tables[k]
                if isinstance(t, np.ndarray):
                    t = np.ascontiguousarray(t)
                    dt = t.dtype
                else:
                    dt = np.dtype(str(t.dtype).replace("torch.", ""))
                if dt not in (np.float32, np.float64):
                    raise ValueError("TBME tables must be float32 or float64")
                arrs.append(t)
            d.tbme_dtype = CI_F32 if dt == np.float32 else CI_F64
            d.v_pp, d.v_nn, d.v_pn = [_ptr(a) for a in arrs]
            self._keep += arrs
        else:
            if seed is None:
                raise ValueError("give TBME tables or a seed")
            d.tbme_source = CI_TBME_SEED
            d.tbme_dtype = CI_F32
            d.tbme_seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        h = C.c_void_p()
        check(L.ci_problem_create(C.byref(d), C.byref(h)), "ci_problem_create")
        self._h = h
        self.S = S
        self._keep = []  # the library copied what it keeps

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ci_problem_destroy(h)
            self._h = None

    # -- Fig. 1, basis step ---------------------------------------------------
    def enumerate_basis(self, stream=None):
        dim = C.c_int64()
        check(lib().ci_enumerate_basis(self._h, C.byref(dim), _stream(stream)), "ci_enumerate_basis")
        return dim.value

    def species(self, s):
        n, w = C.c_int64(), C.c_int32()
        check(lib().ci_species_size(self._h, s, C.byref(n), C.byref(w)), "ci_species_size")
        bits = np.zeros((n.value, w.value), np.uint64)
        q = np.zeros(n.value, np.int32)
        m = np.zeros(n.value, np.int32)
        check(lib().ci_get_species(self._h, s, _ptr(bits), _ptr(q), _ptr(m), n.value), "ci_get_species")
        return {"bits": bits, "q": q, "twoM": m}

    def basis(self):
        dim = self.enumerate_basis()
        p = np.zeros(max(dim, 1), np.int32)
        n = np.zeros(max(dim, 1), np.int32)
        check(lib().ci_get_basis(self._h, _ptr(p), _ptr(n), dim), "ci_get_basis")
        return p[:dim], n[:dim]

    # -- Fig. 1, tile filter ------------------------------------------------
    def species_filter(self, stream=None):
        check(lib().ci_species_filter(self._h, _stream(stream)), "ci_species_filter")

    def species_conn(self, s):
        n, w = C.c_int64(), C.c_int32()
        check(lib().ci_species_size(self._h, s, C.byref(n), C.byref(w)), "ci_species_size")
        ptr = np.zeros(n.value + 1, np.int64)
        total = C.c_int64()
        check(lib().ci_get_species_conn(self._h, s, _ptr(ptr), None, None, 0, C.byref(total)),
              "ci_get_species_conn")
        idx = np.zeros(max(total.value, 1), np.int32)
        d = np.zeros(max(total.value, 1), np.int8)
        check(lib().ci_get_species_conn(self._h, s, _ptr(ptr), _ptr(idx), _ptr(d), total.value,
                                        C.byref(total)), "ci_get_species_conn")
        return ptr, idx[: total.value], d[: total.value]

    # -- Fig. 1, count step ------------------------------------------------
    def count_nnz(self, row_cnt=None, stream=None):
        nnz = C.c_int64()
        check(lib().ci_count_nnz(self._h, C.byref(nnz), _ptr(row_cnt), _stream(stream)), "ci_count_nnz")
        return nnz.value

    # -- Fig. 1, observables step ----------------------------------------------
    def observables(self, op_seeds, X, Y=None, stream=None):
        """a[k, v] = X[:, v]^T O_k Y[:, v] (numpy [m, n]) for the seeded
        two-body operators op_seeds; X and Y are device float64 tensors
        [dim, n] (n <= 16), Y = None meaning Y = X (expectation values)."""
        seeds = np.ascontiguousarray(np.asarray(op_seeds, dtype=np.uint64).reshape(-1))
        n = 1 if X.dim() == 1 else int(X.shape[1])
        if Y is not None and tuple(Y.shape) != tuple(X.shape):
            raise ValueError("X and Y must have the same shape")
        a = np.zeros((len(seeds), n), np.float64)
        check(lib().ci_observables(self._h, _ptr(seeds), len(seeds), _ptr(X), None if Y is None else _ptr(Y), n,
                                   _ptr(a), _stream(stream)), "ci_observables")
        return a

    def refine_eigs(self, evecs, iters=1, stream=None):
        """Refine the Ritz pairs in evecs (device float64 [dim, k], k <= 16,
        overwritten) with the FP64 H applied on the fly: (evals, residuals),
        numpy, ascending (``ci_refine_eigs``)."""
        k = 1 if evecs.dim() == 1 else int(evecs.shape[1])
        ev = np.zeros(k, np.float64)
        rn = np.zeros(k, np.float64)
        check(lib().ci_refine_eigs(self._h, k, int(iters), _ptr(evecs), _ptr(ev), _ptr(rn), _stream(stream)),
              "ci_refine_eigs")
        return ev, rn

    def orbital_blocks(self, sp_orbital, stream=None):
        """Many-body basis orbitals: (device int32 tensor [dim] of group
        indices, number of groups) for the s.p. orbital labels sp_orbital."""
        import torch
        lab = np.ascontiguousarray(np.asarray(sp_orbital, dtype=np.int32))
        nb = C.c_int64()
        dim = self.enumerate_basis(stream)
        blk = torch.empty(dim, dtype=torch.int32, device="cuda")
        check(lib().ci_orbital_blocks(self._h, _ptr(lab), _ptr(blk), C.byref(nb), _stream(stream)),
              "ci_orbital_blocks")
        return blk, nb.value

    # -- Fig. 1, offsets and fill -----------------------------------------------
    def build_H(self, vtype="f32", stream=None):
        h = C.c_void_p()
        check(lib().ci_build_H(self._h, VTYPES.get(vtype, vtype), C.byref(h), _stream(stream)), "ci_build_H")
        return Matrix(h)


class Matrix:
    """A library-owned CSR Hamiltonian (``ci_matrix``)."""

    def __init__(self, handle):
        self._h = handle
        dim, nnz, vt = C.c_int64(), C.c_int64(), C.c_int32()
        check(lib().ci_matrix_info(handle, C.byref(dim), C.byref(nnz), C.byref(vt)), "ci_matrix_info")
        self.dim, self.nnz, self.vtype = dim.value, nnz.value, vt.value
        self.half = False

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ci_matrix_destroy(h)
            self._h = None

    @property
    def value_dtype(self):
        return {CI_F32: np.float32, CI_F64: np.float64, CI_BF16_ROWSCALE: np.uint16}[self.vtype]

    def export(self, stream=None):
        """Host copies (row_ptr int64, col int32, val, row_scale or None)."""
        rp = np.zeros(self.dim + 1, np.int64)
        col = np.zeros(max(self.nnz, 1), np.int32)
        val = np.zeros(max(self.nnz, 1), self.value_dtype)
        rs = np.zeros(max(self.dim, 1), np.float32) if self.vtype == CI_BF16_ROWSCALE else None
        check(lib().ci_matrix_export(self._h, _ptr(rp), _ptr(col), _ptr(val), _ptr(rs), _stream(stream)),
              "ci_matrix_export")
        return rp, col[: self.nnz], val[: self.nnz], rs

    def export_device(self, row_ptr, col, val, row_scale=None, stream=None):
        check(lib().ci_matrix_export(self._h, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(row_scale),
                                     _stream(stream)), "ci_matrix_export")

    def upper(self, stream=None):
        """A new half-stored copy (upper triangle, ``ci_matrix_upper``)."""
        h = C.c_void_p()
        check(lib().ci_matrix_upper(self._h, C.byref(h), _stream(stream)), "ci_matrix_upper")
        m = Matrix(h)
        m.half = True
        return m

    def block_precond_apply(self, blocks, sigma, R, stream=None):
        """W = T R with the block-diagonal preconditioner of LOBPCG over the
        groups blocks = (row_block, nblocks) and shift sigma; R a device
        float64 tensor [dim, nvec] (nvec <= 8).  Returns (W, row_shift)."""
        import torch
        nvec = 1 if R.dim() == 1 else int(R.shape[1])
        W = torch.empty_like(R)
        shift = torch.empty(self.dim, dtype=torch.float64, device=R.device)
        check(lib().ci_block_precond_apply(self._h, _ptr(blocks[0]), int(blocks[1]), float(sigma), _ptr(R), _ptr(W),
                                           nvec, _ptr(shift), _stream(stream)), "ci_block_precond_apply")
        return W, shift

    # -- Fig. 2, optional FMA -------------------------------------------------------
    def apply_H(self, X, Y, stream=None):
        """Y = H X for device tensors [dim, nvec] (nvec 1..8 or 16)."""
        nvec = 1 if X.dim() == 1 else int(X.shape[1])
        check(lib().ci_apply_H(self._h, _ptr(X), _ptr(Y), nvec, _stream(stream)), "ci_apply_H")

    # -- Fig. 1, eigensolve ------------------------------------------------------
    def lowest_eigs(self, k=5, block=8, max_basis=0, max_iter=0, tol=0.0, seed=1, reorth_passes=0,
                    check_every=0, evecs=None, stream=None, allow_unconverged=False, method="lanczos",
                    blocks=None, fp64_products=False):
        """Lowest k eigenvalues (numpy, ascending) and the solve info dict.

        evecs: optional device float64 tensor [dim, k] for the eigenvectors.
        method: "lanczos" (ci_lowest_eigs) or "lobpcg" (ci_lowest_eigs_lobpcg).
        blocks: for LOBPCG, (row_block device int32 tensor, nblocks) from
        ``Problem.orbital_blocks`` for the block-diagonal preconditioner;
        None for the diagonal one.
        fp64_products: reorthogonalisation products on the FP64 CUDA cores
        instead of the tensor cores (ci_eig_opts.fp64_products)."""
        o = _lib.EigOpts(k, block, max_basis, max_iter, tol, seed, reorth_passes, check_every, int(fp64_products))
        ev = np.zeros(k, np.float64)
        info = _lib.EigInfo()
        if method == "lanczos":
            if blocks is not None:
                raise ValueError("blocks is a LOBPCG option")
            st = lib().ci_lowest_eigs(self._h, C.byref(o), _ptr(ev), _ptr(evecs), C.byref(info), _stream(stream))
        elif method == "lobpcg":
            rb, nb = (None, 0) if blocks is None else (_ptr(blocks[0]), int(blocks[1]))
            st = lib().ci_lowest_eigs_lobpcg(self._h, C.byref(o), rb, nb, _ptr(ev), _ptr(evecs), C.byref(info),
                                             _stream(stream))
        else:
            raise ValueError(f"unknown method {method!r}")
        if not (allow_unconverged and st == _lib.CI_ERR_NOT_CONVERGED):
            check(st, "ci_lowest_eigs" if method == "lanczos" else "ci_lowest_eigs_lobpcg")
        out = {"iterations": info.iterations, "restarts": info.restarts, "converged": info.converged,
               "basis_size": info.basis_size, "hnorm_est": info.hnorm_est,
               "residual": list(info.residual)[:k], "seconds": info.seconds, "host_qr": info.host_qr,
               "qr_one_pass": info.qr_one_pass,
               "status": st}
        return ev, out


class Batch:
    """Many problems built and solved together (``ci_batch_*``).

    problems: list of ``Problem`` (kept alive by this object); k: int or a
    list of per-problem eigenpair counts.
    """

    def __init__(self, problems, k=5, max_basis=64, tol=1e-7, max_iter=400, check_every=4, seed=1):
        self.problems = list(problems)
        n = len(self.problems)
        ks = [int(k)] * n if np.isscalar(k) else [int(x) for x in k]
        self._k = ks
        arr = (C.c_void_p * n)(*[p._h.value for p in self.problems])
        karr = (C.c_int32 * n)(*ks)
        o = _lib.EigOpts(0, 8, max_basis, max_iter, tol, seed, 0, check_every)
        h = C.c_void_p()
        check(lib().ci_batch_create(C.cast(arr, C.POINTER(C.c_void_p)), n, C.cast(karr, C.c_void_p), C.byref(o),
                                    C.byref(h)), "ci_batch_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ci_batch_destroy(h)
            self._h = None

    def run(self, stream=None):
        check(lib().ci_batch_run(self._h, _stream(stream)), "ci_batch_run")

    def result(self, i, allow_unconverged=False):
        k = self._k[i]
        ev = np.zeros(k)
        info = _lib.EigInfo()
        st = lib().ci_batch_result(self._h, i, _ptr(ev), C.byref(info))
        if not (allow_unconverged and st == _lib.CI_ERR_NOT_CONVERGED):
            check(st, "ci_batch_result")
        return ev, {"iterations": info.iterations, "converged": info.converged,
                    "residual": list(info.residual)[:k], "status": st}

    def stats(self):
        b, s, st, nnz = C.c_double(), C.c_double(), C.c_int32(), C.c_int64()
        check(lib().ci_batch_stats(self._h, C.byref(b), C.byref(s), C.byref(st), C.byref(nnz)), "ci_batch_stats")
        return {"build_s": b.value, "solve_s": s.value, "steps": st.value, "nnz": nnz.value}

    def tuning(self):
        """Launch shape picked by the autotuner (``ci_batch_tuning``)."""
        tm, sm, ms = C.c_int32(), C.c_int32(), C.c_double()
        check(lib().ci_batch_tuning(self._h, C.byref(tm), C.byref(sm), C.byref(ms)), "ci_batch_tuning")
        return {"tile_ctas_per_sm": tm.value, "spmm_ctas_per_sm": sm.value, "best_step_ms": ms.value}


def _desc(sp, Z, N, nmax, twoM, eps, keep, tables=None, seed=None):
    """Fill a ProblemDesc; arrays it points to are appended to keep."""
    spN = np.ascontiguousarray(sp["N"], dtype=np.int32)
    spm = np.ascontiguousarray(sp["twom"], dtype=np.int32)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    keep += [spN, spm, e]
    d = _lib.ProblemDesc()
    d.n_sp = len(spN)
    d.sp_N = spN.ctypes.data_as(C.POINTER(C.c_int32))
    d.sp_twom = spm.ctypes.data_as(C.POINTER(C.c_int32))
    d.sp_energy = e.ctypes.data_as(C.POINTER(C.c_double))
    d.Z, d.N, d.nmax, d.twoM = int(Z), int(N), int(nmax), int(twoM)
    if tables is not None:
        arrs = [np.ascontiguousarray(tables[k]) for k in ("pp", "nn", "pn")]
        keep += arrs
        d.tbme_source = CI_TBME_TABLES
        d.tbme_dtype = CI_F32 if arrs[0].dtype == np.float32 else CI_F64
        d.v_pp, d.v_nn, d.v_pn = [_ptr(a) for a in arrs]
    else:
        d.tbme_source = CI_TBME_SEED
        d.tbme_dtype = CI_F32
        d.tbme_seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return d


class Queue:
    """Solve queue with continuous batching (``ci_queue_*``)."""

    def __init__(self, mem_budget=0, max_slots=256, max_basis=64, max_iter=400, tol=1e-7, max_tiles=0):
        d = _lib.QueueDesc(int(mem_budget), max_slots, max_basis, max_iter, max_tiles, tol)
        h = C.c_void_p()
        check(lib().ci_queue_create(C.byref(d), C.byref(h)), "ci_queue_create")
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ci_queue_destroy(h)
            self._h = None

    __del__ = close

    def submit(self, sp, Z, N, nmax, twoM, eps, k, seed=None, tables=None):
        keep = []
        r = _lib.Request(_desc(sp, Z, N, nmax, twoM, eps, keep, tables, seed), int(k))
        t = C.c_uint64()
        check(lib().ci_submit(self._h, C.byref(r), C.byref(t)), "ci_submit")
        return t.value

    def poll(self, ticket):
        """(status, result dict); status 6 (CI_NOT_READY) while running."""
        r = _lib.Result()
        st = lib().ci_poll(self._h, ticket, C.byref(r))
        res = {"status": r.status, "k": r.k, "iterations": r.iterations, "dim": r.dim, "nnz": r.nnz,
               "evals": np.array(r.evals[: r.k]), "residual": np.array(r.residual[: r.k]),
               "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done, "latency_s": r.latency_s}
        return st, res

    def cancel(self, ticket):
        check(lib().ci_cancel(self._h, ticket), "ci_cancel")

    def stats(self):
        a, b, c, d, m = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_size_t()
        check(lib().ci_queue_stats(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(m)),
              "ci_queue_stats")
        return {"submitted": a.value, "admitted": b.value, "completed": c.value, "steps": d.value,
                "mem_used": m.value}


def trace_enable(on=True, sample=1):
    """Count every library kernel launch and bracket every `sample`-th launch
    of each kernel with CUDA events (ci_trace_enable)."""
    check(lib().ci_trace_enable((max(int(sample), 1)) if on else 0), "ci_trace_enable")


def trace_read(reset=True):
    """{kernel name: (launches, total ms)} since the last reset (ci_trace_read)."""
    n = C.c_int32()
    check(lib().ci_trace_read(None, 0, C.byref(n), 0), "ci_trace_read")
    buf = (_lib.TraceEntry * max(n.value, 1))()
    check(lib().ci_trace_read(buf, n.value, C.byref(n), 1 if reset else 0), "ci_trace_read")
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(n.value)}


COUNT_VARIANTS = {"hybrid": 0, "mbs": 1, "bits": 2}


def count_pairs(mbs, S, variant="hybrid", max_diff=4, row_counts=None, stream=None):
    """Count benchmark of Sec. 2.1 (Listing 2) on the device.

    mbs: device uint16-compatible tensor [n, N] (torch.int16 / uint16 bits),
    each row the ascending occupied s.p. states of one state.  Returns the
    total number of pairs within max_diff differing states; row_counts
    (device int64 [n]) receives the per-state counts."""
    n, N = (int(mbs.shape[0]), int(mbs.shape[1])) if mbs.dim() == 2 else (0, 1)
    total = C.c_int64()
    check(lib().ci_count_pairs(_ptr(mbs), n, N, int(S), COUNT_VARIANTS.get(variant, variant), int(max_diff),
                               C.byref(total), _ptr(row_counts), _stream(stream)), "ci_count_pairs")
    return total.value


def basis_product(op, A, B, Cm, alpha=-1.0, beta=1.0, method="tc", stream=None):
    """ci_basis_product on float64 device tensors: op "tn" writes
    Cm = A^T B ([na, nb]); op "nn" updates B = beta B + alpha A Cm.  method
    "tc" (tensor cores, exact digit-plane products) or "fp64" (CUDA cores).
    A, B are [n, cols] row-major (their row strides are the leading
    dimensions)."""
    import torch
    opc = {"tn": 0, "nn": 1}[op]
    mc = {"fp64": 0, "tc": 1}[method]
    n, na = int(A.shape[0]), int(A.shape[1])
    nb = int(B.shape[1])
    for t in (A, B):
        if t.dim() != 2 or t.stride(1) != 1 or t.dtype != torch.float64 or not t.is_cuda:
            raise ValueError("A and B must be float64 CUDA matrices with unit column stride")
    check(lib().ci_basis_product(opc, mc, n, C.c_void_p(A.data_ptr()), int(A.stride(0)), na,
                                 C.c_void_p(B.data_ptr()), int(B.stride(0)), nb, _ptr(Cm), float(alpha), float(beta),
                                 _stream(stream)), "ci_basis_product")


def exclusive_scan(counts, offsets, stream=None):
    """Eq. 1 on the device: int32 counts [n] -> int64 offsets [n+1]."""
    check(lib().ci_exclusive_scan(_ptr(counts), int(counts.numel()), _ptr(offsets), _stream(stream)),
          "ci_exclusive_scan")


def exclusive_scan_noalloc(counts, offsets, stream=None):
    """The same scan without device allocation (ci_exclusive_scan_noalloc)."""
    check(lib().ci_exclusive_scan_noalloc(_ptr(counts), int(counts.numel()), _ptr(offsets), _stream(stream)),
          "ci_exclusive_scan_noalloc")


# -- motif benchmarks of Sec. 2.2-2.4 ----------------------------------------
def scan_serial(counts, offsets, stream=None):
    """Listing 5's serial prefix sum on the device (one thread):
    int32 counts [n] -> int64 offsets [n+1] (ci_scan_serial)."""
    check(lib().ci_scan_serial(_ptr(counts), int(counts.numel()), _ptr(offsets), _stream(stream)), "ci_scan_serial")


def fill_shared(offset, m, p, arr, stream=None):
    """Listing 7's shared-array fill: row i stores j = p, 2p, ... <= m at
    arr[offset[i]:] (ci_fill_shared); offset device int64 [n], arr device int32."""
    check(lib().ci_fill_shared(_ptr(offset), int(offset.numel()), int(m), int(p), _ptr(arr), _stream(stream)),
          "ci_fill_shared")


def array_reduction(x, y, stream=None):
    """Eq. 2's small-array reduction a[k] = sum_ij x[i, k] y[j, k] over all
    n^2 pairs; x, y device float32 [n, m] (row i = the listings' column
    x(:, i)); returns a device float32 [m] (ci_array_reduction)."""
    import torch
    n, m = int(x.shape[0]), int(x.shape[1])
    a = torch.empty(m, dtype=torch.float32, device=x.device)
    check(lib().ci_array_reduction(_ptr(x), _ptr(y), n, m, _ptr(a), _stream(stream)), "ci_array_reduction")
    return a
