"""Write tests/golden/golden.json from the FP64 oracle (and synth inputs) only.

Run:  python tests/golden/make_golden.py        (about 2-4 minutes on 8 cores)

Stored values (all computed by ``oracle``):
* dimension and nnz of the preset problems c0, c1, c2_sub, and c2's dimension;
* the lowest eigenvalues of c0 (dense LAPACK), c2_sub (dense LAPACK) and
  c1 (ARPACK on the oracle's full FP64 CSR; FP32 TBME table widened exactly);
* SHA-256 digests of the oracle's full row_ptr and column arrays (both as
  little-endian int64) for c0, c2_sub and c1: the structural pattern of
  Listing 2's count and Fig. 1's fill, compared bit for bit with the GPU's;
* for c1, the number of products H x ARPACK took and its basis size (the
  work per row of the oracle's eigensolve, which the CPU baseline samples).
"""

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def digest(a):
    """SHA-256 of an integer array as little-endian int64."""
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i8").tobytes()).hexdigest()


def make(name, need_eigs=True, dense=False):
    p = synth.preset(name)
    sp = synth.ho_sp_table(p.n_shell_max)
    eps = synth.sp_energies(sp, p.hbar_omega)
    dt = np.float64 if p.value_type == "f64" else np.float32
    T = synth.tbme_tables(sp, p.seed, dt)
    o = oracle.OracleProblem(sp, p.Z, p.N, p.nmax, p.twoM, eps, T)
    rec = {"dim": o.dim, "k": p.k, "seed": p.seed, "tbme_dtype": np.dtype(dt).name}
    if not need_eigs:
        return rec
    t = time.time()
    rp, cols, vals, _ = o.csr(with_absums=False)
    rec["nnz"] = int(rp[-1])
    rec["row_ptr_sha256"] = digest(rp)
    rec["col_sha256"] = digest(cols)
    if dense:
        w = oracle.lowest_dense(oracle.dense_from_csr(rp, cols, vals, o.dim), p.k)
        rec["method"] = "dense LAPACK eigvalsh"
    else:
        st = {}
        w = oracle.lowest_sparse(rp, cols, vals, o.dim, p.k, stats=st)
        rec["method"] = "ARPACK eigsh (which=SA, tol=1e-12)"
        rec["arpack_matvecs"] = st["matvecs"]
        rec["arpack_ncv"] = st["ncv"]
    rec["lowest"] = [float(x) for x in w]
    rec["seconds"] = round(time.time() - t, 1)
    print(name, rec, flush=True)
    return rec


def main():
    out = {
        "c0": make("c0", dense=True),
        "c2_sub": make("c2_sub", dense=True),
        "c1": make("c1"),
        "c2": make("c2", need_eigs=False),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
