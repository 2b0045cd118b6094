"""FP64 CPU oracle of the configuration-interaction hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product library never calls it, and it shares no code,
header, table or helper with the CUDA path; inputs come from ``synth``.

Parts (each pinned by the ``-m "not gpu"`` tests against something other
than itself):

* ``ci_oracle.c`` (plain C, FP64): species determinant lists, product basis,
  difference counts, Slater-Condon matrix elements, rows / CSR of H, FP64
  SpMM, the exclusive scan of Eq. 1 and the per-state counts of the count
  benchmark (Sec. 2.1);
* ``brute.py`` (pure Python): H built by applying every second-quantised
  operator term to every basis state, for tiny spaces;
* ``eig.py``: lowest eigenvalues by LAPACK (dense) or ARPACK (sparse), the
  plain definition of "lowest k eigenvalues";
* ``precond.py``: many-body basis orbitals and the block-diagonal
  preconditioner of LOBPCG (dense solves per block);
* ``motifs.py``: the shared-array fill and small-array reduction motifs of
  Sec. 2.3-2.4 (plain loops).
"""

from .core import (OracleProblem, build_library, count_pairs, exclusive_scan, expectation_values, set_threads,
                   spmm)
from .eig import lowest_dense, lowest_sparse, dense_from_csr
from . import brute, motifs, precond

__all__ = ["OracleProblem", "build_library", "count_pairs", "exclusive_scan", "expectation_values", "set_threads", "spmm",
           "lowest_dense", "lowest_sparse", "dense_from_csr", "brute", "motifs", "precond"]
