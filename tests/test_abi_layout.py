"""The ctypes mirrors of the C ABI's structs have the header's layout.

A C program compiled against include/mfdci.h prints sizeof and the offset of
every member the binding declares; both must equal what ctypes computes, so a
field added, dropped or reordered on one side only fails here (no GPU)."""

import os
import shutil
import subprocess
import tempfile

import ctypes as C
import pytest

from paper_2110_10765_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [
    (_lib.ProblemDesc, "ci_problem_desc"),
    (_lib.EigOpts, "ci_eig_opts"),
    (_lib.EigInfo, "ci_eig_info"),
    (_lib.QueueDesc, "ci_queue_desc"),
    (_lib.Request, "ci_request"),
    (_lib.Result, "ci_result"),
    (_lib.TraceEntry, "ci_trace_entry"),
]


def _c_layout():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mfdci.h"', "int main(void) {"]
    for cls, cname in PAIRS:
        lines.append('    printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('    printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["    return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", exe, src])
        out = subprocess.check_output([exe], text=True)
    got = {}
    for line in out.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    return got


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_struct_layouts_match_header():
    got = _c_layout()
    for cls, cname in PAIRS:
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
