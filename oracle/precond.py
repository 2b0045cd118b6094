"""Many-body basis orbitals and the block-diagonal preconditioner of LOBPCG
(Sec. 2): basis states that put every nucleon into the same single-particle
orbitals, differing only in the magnetic substates, form one many-body
basis orbital, and the diagonal blocks of H over these groups give the
eigensolver's preconditioner.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definitions followed here (the paper names the preconditioner but not its
form, so these are this project's reading, stated with the library's API):

* group of a basis state = (sorted orbital labels of its protons, sorted
  orbital labels of its neutrons); groups are numbered 0, 1, ... in order of
  first appearance by row;
* every group's member rows, ascending, are cut into ceil(c / 128) nearly
  equal consecutive sub-blocks (``numpy.array_split``);
* T = blockdiag_b (H_bb - sigma_b I)^-1 over the sub-blocks, sigma_b = sigma
  when H_bb - sigma I is positive definite, else min(sigma, g_b) - eta_b with
  g_b = min_i (H_ii - sum_{j != i} |H_ij|) (Gershgorin) and
  eta_b = 1e-3 max(max_i sum_j |H_ij|, |sigma|).
"""

import numpy as np
import scipy.sparse as sps

SUB_MAX = 128


def orbital_blocks(occ_p, occ_n, p_idx, n_idx, sp_orbital):
    """(group index [dim] int32, number of groups) of the basis rows whose
    proton determinant is occ_p[p_idx[r]] and neutron determinant
    occ_n[n_idx[r]] (occupied s.p. states), for orbital labels sp_orbital."""
    lab = np.asarray(sp_orbital)
    ids = {}
    out = np.empty(len(p_idx), np.int32)
    for r in range(len(p_idx)):
        key = (tuple(sorted(lab[occ_p[p_idx[r]]].tolist())), tuple(sorted(lab[occ_n[n_idx[r]]].tolist())))
        out[r] = ids.setdefault(key, len(ids))
    return out, len(ids)


def sub_blocks(block, nblocks, sub_max=SUB_MAX):
    """Member rows of every sub-block, groups in index order."""
    block = np.asarray(block)
    subs = []
    for g in range(nblocks):
        rows = np.nonzero(block == g)[0]
        if len(rows):
            subs.extend(np.array_split(rows, -(-len(rows) // sub_max)))
    return subs


def block_shift(A, sigma):
    """sigma_b of one sub-block A = H_bb (dense, symmetric)."""
    n = A.shape[0]
    try:
        np.linalg.cholesky(A - sigma * np.eye(n))
        return float(sigma)
    except np.linalg.LinAlgError:
        absrow = np.abs(A).sum(axis=1)
        d = np.diag(A)
        g = np.min(d - (absrow - np.abs(d)))
        eta = 1e-3 * max(absrow.max(), abs(sigma), 1e-300)
        return float(min(sigma, g) - eta)


def block_precond(row_ptr, cols, vals, block, nblocks, sigma, R, sub_max=SUB_MAX):
    """W = T R for R [dim, nvec], with the shift of every row and the bound
    |T| |R| (elementwise), from the CSR of H."""
    R = np.asarray(R, dtype=np.float64)
    if R.ndim == 1:
        R = R[:, None]
    dim = len(row_ptr) - 1
    H = sps.csr_matrix((np.asarray(vals, np.float64), np.asarray(cols), np.asarray(row_ptr)), shape=(dim, dim))
    W = np.zeros_like(R)
    Wabs = np.zeros_like(R)
    shift = np.zeros(dim)
    for rows in sub_blocks(block, nblocks, sub_max):
        A = H[rows][:, rows].toarray()
        s = block_shift(A, sigma)
        inv = np.linalg.inv(A - s * np.eye(len(rows)))
        W[rows] = inv @ R[rows]
        Wabs[rows] = np.abs(inv) @ np.abs(R[rows])
        shift[rows] = s
    return W, shift, Wabs
