"""Lowest eigenvalues of the oracle's H.  Test infrastructure.

The lowest k eigenvalues of a real symmetric matrix have a plain
definition; the oracle evaluates it with LAPACK (dense, ``numpy.linalg``)
for dimensions up to a few thousand and with ARPACK's implicitly restarted
Lanczos (``scipy.sparse.linalg.eigsh``, smallest algebraic) above that.
Both are pinned in the tests by closed forms (zero interaction: sums of
one-body energies; two particles: the TBME block) and the trace.
"""

import numpy as np


def dense_from_csr(row_ptr, cols, vals, dim):
    H = np.zeros((dim, dim))
    for i in range(dim):
        s, e = row_ptr[i], row_ptr[i + 1]
        H[i, cols[s:e]] = vals[s:e]
    return H


def lowest_dense(H, k):
    """Sorted lowest k eigenvalues of a dense symmetric matrix (LAPACK)."""
    w = np.linalg.eigvalsh(np.asarray(H, dtype=np.float64))
    return np.sort(w)[:k]


def lowest_sparse(row_ptr, cols, vals, dim, k, tol=1e-12, stats=None):
    """Sorted lowest k eigenvalues of a sparse symmetric CSR (ARPACK).  With
    a dict ``stats``, the number of products H x ARPACK asked for goes to
    stats["matvecs"] and its basis size to stats["ncv"]."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spl
    H = sps.csr_matrix((np.asarray(vals, np.float64), np.asarray(cols, np.int64),
                        np.asarray(row_ptr, np.int64)), shape=(dim, dim))
    ncv = max(2 * k + 1, 40)
    count = [0]

    def matvec(x):
        count[0] += 1
        return H @ x

    op = spl.LinearOperator((dim, dim), matvec=matvec, dtype=np.float64)
    v0 = np.ones(dim) / np.sqrt(dim)
    w = spl.eigsh(op, k=k, which="SA", tol=tol, v0=v0, return_eigenvectors=False, ncv=ncv)
    if stats is not None:
        stats["matvecs"] = count[0]
        stats["ncv"] = ncv
    return np.sort(w)[:k]
