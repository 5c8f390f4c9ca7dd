"""Pins of the oracle's static condensation (Sec. 3, Eqs. global and reduced)
against the global system itself, assembled densely on tiny grids:
* solving the condensed system and recovering the secondary unknowns gives
  the dense solution of J delta = -r;
* A and b equal the dense Schur complement J11 - J12 J22^-1 J21 and
  -r1 + J12 J22^-1 r2 formed from the global matrix's partition;
* with no secondary unknowns A = J11 and b = -r1 exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1912_04385_gb300 import synthetic as sy


def _global_dense(f):
    """Dense J of Eq. global, unknowns ordered [all primary | all secondary],
    each cell-interleaved; and r in the same order."""
    N, n1, n2 = f.n_cells, f.n1, f.n2
    n = N * (n1 + n2)
    J = np.zeros((n, n))
    o2 = N * n1
    for i in range(N):
        for e in range(f.row_ptr[i], f.row_ptr[i + 1]):
            j = f.col_idx[e]
            J[i * n1:(i + 1) * n1, j * n1:(j + 1) * n1] = f.j11[e]
            J[o2 + i * n2:o2 + (i + 1) * n2, j * n1:(j + 1) * n1] = f.j21[e]
        J[i * n1:(i + 1) * n1, o2 + i * n2:o2 + (i + 1) * n2] = f.j12[i]
        J[o2 + i * n2:o2 + (i + 1) * n2, o2 + i * n2:o2 + (i + 1) * n2] = f.j22[i]
    r = np.concatenate([f.r1, f.r2])
    return J, r


def _bsr_dense(rp, ci, blocks):
    N, nb = len(rp) - 1, blocks.shape[1]
    A = np.zeros((N * nb, N * nb))
    for i in range(N):
        for e in range(rp[i], rp[i + 1]):
            A[i * nb:(i + 1) * nb, ci[e] * nb:(ci[e] + 1) * nb] = blocks[e]
    return A


CASES = [dict(nx=5, ny=4, n1=6, n2=4), dict(nx=6, ny=3, n1=4, n2=1, j21_neighbors=True),
         dict(nx=4, ny=4, n1=5, n2=7, j21_neighbors=True, pe=100.0),
         dict(nx=3, ny=3, n1=14, n2=10, j21_neighbors=True)]


@pytest.mark.parametrize("c", CASES)
def test_condensed_solve_equals_global_solve(c):
    c = dict(c)
    f = sy.make_full_system(c.pop("nx"), c.pop("ny"), c.pop("n1"), c.pop("n2"), seed=2, **c)
    J, r = _global_dense(f)
    delta = np.linalg.solve(J, -r)
    a, b = oracle.condense(f)
    A = _bsr_dense(f.row_ptr, f.col_idx, a)
    d1 = np.linalg.solve(A, b)
    o2 = f.n_cells * f.n1
    scale = np.abs(delta).max()
    assert np.abs(d1 - delta[:o2]).max() <= 1e-9 * scale
    d2 = oracle.recover(f, d1)
    assert np.abs(d2 - delta[o2:]).max() <= 1e-9 * scale
    # the recovery is the second block row of the global system exactly
    d2x = oracle.recover(f, delta[:o2])
    assert np.abs(d2x - delta[o2:]).max() <= 1e-11 * scale


@pytest.mark.parametrize("c", CASES)
def test_condensed_matrix_is_the_schur_complement(c):
    c = dict(c)
    f = sy.make_full_system(c.pop("nx"), c.pop("ny"), c.pop("n1"), c.pop("n2"), seed=5, **c)
    J, r = _global_dense(f)
    o2 = f.n_cells * f.n1
    J11, J12, J21, J22 = J[:o2, :o2], J[:o2, o2:], J[o2:, :o2], J[o2:, o2:]
    X = J12 @ np.linalg.inv(J22)
    S = J11 - X @ J21
    a, b = oracle.condense(f)
    A = _bsr_dense(f.row_ptr, f.col_idx, a)
    assert np.abs(A - S).max() <= 1e-12 * np.abs(S).max()
    assert np.abs(b - (-r[:o2] + X @ r[o2:])).max() <= 1e-12 * np.abs(b).max()
    # the pattern is kept: nothing of S falls outside the cell graph's blocks
    mask = _bsr_dense(f.row_ptr, f.col_idx, np.ones_like(a)) != 0
    assert not np.any(S[~mask])


def test_no_secondary_unknowns_is_the_identity_map():
    f = sy.make_full_system(5, 4, 6, 0, seed=1)
    a, b = oracle.condense(f)
    assert np.array_equal(a, f.j11) and np.array_equal(b, -f.r1)
    assert oracle.recover(f, np.zeros(f.n_cells * 6)).size == 0


def test_singular_secondary_block_is_reported():
    f = sy.make_full_system(3, 3, 4, 3, seed=1)
    f.j22[4, 0, :] = 0.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.condense(f)
    assert e.value.status == oracle.oracle.ERR_SINGULAR
