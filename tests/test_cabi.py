"""The C-ABI library builds, loads and exports every function of mfdci.h;
argument errors come back as status codes (no GPU needed for these)."""

import ctypes as C
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mfdci.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    from paper_2110_10765_gb300 import build, _lib
    build.build()
    return _lib.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ci_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ci_enumerate_basis", "ci_count_nnz", "ci_build_H", "ci_apply_H", "ci_lowest_eigs",
              "ci_exclusive_scan", "ci_species_filter"):
        assert n in names


def test_every_declared_function_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_export(lib):
    from paper_2110_10765_gb300 import _lib
    assert set(declared_functions()) <= set(_lib._SIGS)


def test_status_strings(lib):
    assert lib.ci_status_string(0) == b"CI_OK"
    assert lib.ci_status_string(1) == b"CI_ERR_INVALID_ARG"
    assert lib.ci_version().startswith(b"mfdci")


def test_invalid_arguments_return_status(lib):
    from paper_2110_10765_gb300 import _lib
    h = C.c_void_p()
    assert lib.ci_problem_create(None, C.byref(h)) == 1
    d = _lib.ProblemDesc()
    d.n_sp = 0
    assert lib.ci_problem_create(C.byref(d), C.byref(h)) == 1
    assert b"n_sp" in lib.ci_last_error()
    d.n_sp = 200
    assert lib.ci_problem_create(C.byref(d), C.byref(h)) == 1
    assert lib.ci_exclusive_scan(None, 5, None, None) == 1
    assert lib.ci_exclusive_scan(None, -1, None, None) == 1
    assert lib.ci_apply_H(None, None, None, 8, None) == 1
    assert lib.ci_lowest_eigs(None, None, None, None, None, None) == 1
    assert lib.ci_enumerate_basis(None, None, None) == 1
    assert lib.ci_build_H(None, 0, None, None) == 1
