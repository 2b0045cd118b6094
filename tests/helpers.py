"""Shared builders for the parity tests: one seeded problem, two sides.

The inputs (s.p. table, one-body energies, TBME tables) come from ``synth``;
``oracle_problem`` and ``gpu_problem`` build the FP64 oracle and the CUDA
library's problem from the same inputs.
"""

import json
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "golden.json")

# FP32 values: |h32 - h64| <= REL32 * max(|h64|, sum |terms|) (per element).
REL32 = 1e-6
# FP64 values: the same bound with 1e-12.
REL64 = 1e-12
# eigenvalues: |l - l64| <= EIG_REL * max(|l64|, 1)
EIG_REL = 1e-5


def inputs(n_shell, Z, N, nmax, seed=0, dtype=np.float32, zero=False, twoM=None, hw=20.0):
    sp = synth.ho_sp_table(n_shell)
    eps = synth.sp_energies(sp, hw)
    S = len(sp["N"])
    T = synth.tbme_tables_zero(S, dtype) if zero else synth.tbme_tables(sp, seed, dtype)
    if twoM is None:
        twoM = (Z + N) % 2
    return dict(sp=sp, Z=Z, N=N, nmax=nmax, twoM=twoM, eps=eps, tables=T)


def preset_inputs(name):
    p = synth.preset(name)
    dt = np.float64 if p.value_type == "f64" else np.float32
    return inputs(p.n_shell_max, p.Z, p.N, p.nmax, seed=p.seed, dtype=dt, twoM=p.twoM, hw=p.hbar_omega)


def oracle_problem(inp):
    import oracle
    return oracle.OracleProblem(inp["sp"], inp["Z"], inp["N"], inp["nmax"], inp["twoM"], inp["eps"],
                                inp["tables"])


def gpu_problem(inp, seed=None):
    import paper_2110_10765_gb300 as ci
    if seed is not None:
        return ci.Problem(inp["sp"], inp["Z"], inp["N"], inp["nmax"], inp["twoM"], inp["eps"], seed=seed)
    return ci.Problem(inp["sp"], inp["Z"], inp["N"], inp["nmax"], inp["twoM"], inp["eps"], tables=inp["tables"])


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def value_bound(h64, absum, rel):
    return rel * np.maximum(np.abs(h64), absum) + 1e-300
