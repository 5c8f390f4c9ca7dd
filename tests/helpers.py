"""Format conversions used by the tests (no preconditioner arithmetic)."""
import numpy as np


def bsr_dense(row_ptr, col_idx, vals):
    N = len(row_ptr) - 1
    nb = vals.shape[1]
    A = np.zeros((N * nb, N * nb))
    for i in range(N):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            j = col_idx[e]
            A[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = vals[e]
    return A


def csr_dense(row_ptr, col_idx, vals, ncols=None):
    n = len(row_ptr) - 1
    m = ncols if ncols is not None else n
    A = np.zeros((n, m))
    for i in range(n):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            A[i, col_idx[e]] += vals[e]
    return A


def diag_blocks(sysm, vals=None):
    """Diagonal block of every cell, shape (N, nb, nb)."""
    v = sysm.vals if vals is None else vals
    out = np.empty((sysm.n_cells, sysm.nb, sysm.nb))
    for i in range(sysm.n_cells):
        for e in range(sysm.row_ptr[i], sysm.row_ptr[i + 1]):
            if sysm.col_idx[e] == i:
                out[i] = v[e]
    return out


def operator_matrix(apply, n):
    """Dense matrix of a linear operator given by its action on unit vectors."""
    M = np.empty((n, n))
    e = np.zeros(n)
    for k in range(n):
        e[k] = 1.0
        M[:, k] = apply(e)
        e[k] = 0.0
    return M


def stored_factor_form(bilu, strip):
    """The block ILU(0) factors of the oracle (``OracleSolver.bilu()``) in the
    form the library stores them (``mss_bilu_factors``): the same L and U
    blocks in colour-major positions, except that an upper block coupling two
    cells of one strip holds U_qq^{-1} U_qj; plus U_qq^{-1} per position.
    strip: cells per strip of the ordering (1 for point multicolour). Format
    conversion only: the inverses are numpy's."""
    perm, rp, ci, v = bilu["perm"], bilu["row_ptr"], bilu["col_idx"], bilu["vals"]
    n = perm.size
    rows = np.repeat(np.arange(n), np.diff(rp))
    dpos = np.flatnonzero(ci == rows)
    assert dpos.size == n
    fdinv = np.linalg.inv(v[dpos])
    fv = v.copy()
    if strip > 1:
        sid = perm // strip
        m = (ci > rows) & (sid[ci] == sid[rows])
        fv[m] = np.einsum("kij,kjl->kil", fdinv[rows[m]], v[m])
    return fv, fdinv
