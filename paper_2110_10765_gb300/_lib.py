"""ctypes declarations of libmfdci.so (the C ABI of include/mfdci.h).

Argument marshalling only: every step of the path runs in the library.  The
library must have been built (``paper_2110_10765_gb300.build.build()``);
there is no fallback.
"""

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmfdci.so")

_lib = None
_lock = threading.Lock()

CI_OK = 0
CI_NOT_READY = 6
CI_ERR_NOT_CONVERGED = 9
CI_F32, CI_F64, CI_BF16_ROWSCALE = 0, 1, 2
CI_TBME_TABLES, CI_TBME_SEED = 0, 1


class ProblemDesc(C.Structure):
    _fields_ = [("n_sp", C.c_int32), ("sp_N", C.POINTER(C.c_int32)),
                ("sp_twom", C.POINTER(C.c_int32)), ("sp_energy", C.POINTER(C.c_double)),
                ("Z", C.c_int32), ("N", C.c_int32), ("nmax", C.c_int32), ("twoM", C.c_int32),
                ("tbme_source", C.c_int32), ("tbme_dtype", C.c_int32),
                ("v_pp", C.c_void_p), ("v_nn", C.c_void_p), ("v_pn", C.c_void_p),
                ("tbme_seed", C.c_uint64)]


class EigOpts(C.Structure):
    _fields_ = [("k", C.c_int32), ("block", C.c_int32), ("max_basis", C.c_int32),
                ("max_iter", C.c_int32), ("tol", C.c_double), ("seed", C.c_uint64),
                ("reorth_passes", C.c_int32), ("check_every", C.c_int32), ("fp64_products", C.c_int32)]


class EigInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("basis_size", C.c_int32), ("hnorm_est", C.c_double),
                ("residual", C.c_double * 32), ("seconds", C.c_double), ("host_qr", C.c_int32),
                ("qr_one_pass", C.c_int32)]


class QueueDesc(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("max_slots", C.c_int32), ("max_basis", C.c_int32),
                ("max_iter", C.c_int32), ("max_tiles", C.c_int32), ("tol", C.c_double)]


class Request(C.Structure):
    _fields_ = [("desc", ProblemDesc), ("k", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("k", C.c_int32), ("iterations", C.c_int32), ("dim", C.c_int64),
                ("nnz", C.c_int64), ("evals", C.c_double * 16), ("residual", C.c_double * 16),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("latency_s", C.c_double)]


class TraceEntry(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double)]


class CIError(RuntimeError):
    def __init__(self, status, name, msg):
        super().__init__("%s: %s" % (name, msg))
        self.status = status


_P = C.c_void_p
_I64P = C.POINTER(C.c_int64)
_SIGS = {
    "ci_last_error": (C.c_char_p, []),
    "ci_status_string": (C.c_char_p, [C.c_int]),
    "ci_version": (C.c_char_p, []),
    "ci_problem_create": (C.c_int, [C.POINTER(ProblemDesc), C.POINTER(_P)]),
    "ci_problem_destroy": (None, [_P]),
    "ci_enumerate_basis": (C.c_int, [_P, _I64P, _P]),
    "ci_species_size": (C.c_int, [_P, C.c_int32, _I64P, C.POINTER(C.c_int32)]),
    "ci_get_species": (C.c_int, [_P, C.c_int32, _P, _P, _P, C.c_int64]),
    "ci_get_basis": (C.c_int, [_P, _P, _P, C.c_int64]),
    "ci_species_filter": (C.c_int, [_P, _P]),
    "ci_get_species_conn": (C.c_int, [_P, C.c_int32, _P, _P, _P, C.c_int64, _I64P]),
    "ci_count_nnz": (C.c_int, [_P, _I64P, _P, _P]),
    "ci_exclusive_scan": (C.c_int, [_P, C.c_int64, _P, _P]),
    "ci_exclusive_scan_noalloc": (C.c_int, [_P, C.c_int64, _P, _P]),
    "ci_count_pairs": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                 C.POINTER(C.c_int64), _P, _P]),
    "ci_observables": (C.c_int, [_P, _P, C.c_int32, _P, _P, C.c_int32, _P, _P]),
    "ci_build_H": (C.c_int, [_P, C.c_int32, C.POINTER(_P), _P]),
    "ci_matrix_destroy": (None, [_P]),
    "ci_matrix_upper": (C.c_int, [_P, C.POINTER(_P), _P]),
    "ci_matrix_info": (C.c_int, [_P, _I64P, _I64P, C.POINTER(C.c_int32)]),
    "ci_matrix_export": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "ci_apply_H": (C.c_int, [_P, _P, _P, C.c_int32, _P]),
    "ci_lowest_eigs": (C.c_int, [_P, C.POINTER(EigOpts), _P, _P, C.POINTER(EigInfo), _P]),
    "ci_basis_product": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, _P, C.c_int32, C.c_int32, _P, C.c_int32,
                                   C.c_int32, _P, C.c_double, C.c_double, _P]),
    "ci_lowest_eigs_lobpcg": (C.c_int, [_P, C.POINTER(EigOpts), _P, C.c_int64, _P, _P, C.POINTER(EigInfo), _P]),
    "ci_orbital_blocks": (C.c_int, [_P, _P, _P, _I64P, _P]),
    "ci_refine_eigs": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _P, _P]),
    "ci_scan_serial": (C.c_int, [_P, C.c_int64, _P, _P]),
    "ci_fill_shared": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, _P, _P]),
    "ci_array_reduction": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, _P]),
    "ci_block_precond_apply": (C.c_int, [_P, _P, C.c_int64, C.c_double, _P, _P, C.c_int32, _P, _P]),
    "ci_batch_create": (C.c_int, [C.POINTER(_P), C.c_int32, _P, C.POINTER(EigOpts), C.POINTER(_P)]),
    "ci_batch_run": (C.c_int, [_P, _P]),
    "ci_batch_result": (C.c_int, [_P, C.c_int32, _P, C.POINTER(EigInfo)]),
    "ci_batch_stats": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32), _I64P]),
    "ci_batch_tuning": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "ci_batch_destroy": (None, [_P]),
    "ci_queue_create": (C.c_int, [C.POINTER(QueueDesc), C.POINTER(_P)]),
    "ci_submit": (C.c_int, [_P, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "ci_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(Result)]),
    "ci_cancel": (C.c_int, [_P, C.c_uint64]),
    "ci_queue_stats": (C.c_int, [_P, _I64P, _I64P, _I64P, _I64P, C.POINTER(C.c_size_t)]),
    "ci_queue_destroy": (None, [_P]),
    "ci_trace_enable": (C.c_int, [C.c_int32]),
    "ci_trace_read": (C.c_int, [C.POINTER(TraceEntry), C.c_int32, C.POINTER(C.c_int32), C.c_int32]),
}


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    "libmfdci.so is not built (%s); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first" % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                if not hasattr(L, name):
                    continue
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    """Names of _SIGS that the library exports."""
    L = lib()
    return [n for n in _SIGS if hasattr(L, n)]


def check(status, what=""):
    if status == CI_OK:
        return
    L = lib()
    name = L.ci_status_string(status).decode()
    msg = L.ci_last_error().decode()
    raise CIError(status, name, (what + ": " if what else "") + msg)
