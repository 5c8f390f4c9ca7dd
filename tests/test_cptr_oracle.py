"""Pins of the oracle's two-stage CPTR (Sec. 4.2, Eqs. CPTRinit, CPTR1,
CPTRM1) and of its system AMG for the 2 x 2 block B_ee.

* scaling: Z_es = 0 in every cell block, W unit lower triangular in [s, e]
  order with only the P and T rows changed, the solution unchanged;
* composition: Eq. multistageprec with two stages, and the stage operator
  acting on (P, T) only;
* exactness: with a direct first stage on an upper-block-triangular scaled
  matrix FGMRES stops after one iteration (negative control: not so on the
  standard family);
* system AMG: the C/F split is PMIS on the Frobenius-norm matrix of the
  blocks; P has no cross-unknown weights and each unknown's rows are the
  classical interpolation of that unknown's scalar matrix on the split;
  every coarse operator is the dense P^T A P; two identical uncoupled
  unknowns give two copies of the scalar hierarchy's V-cycle; the V-cycle
  reduces the error of a coupled 2D Poisson system at a size-independent
  rate.
"""
import numpy as np
import pytest

import oracle
from paper_1912_04385_gb300 import synthetic as sy
from tests.helpers import bsr_dense, csr_dense, diag_blocks, operator_matrix


@pytest.mark.parametrize("nb,p,t", [(4, 0, 1), (6, 0, 1), (5, 2, 4), (3, 1, 0), (2, 0, 1)])
def test_cptr_scaling(nb, p, t):
    s = sy.make_system(6, 5, nb, p_idx=p, t_idx=t, pe=10.0, seed=3, band=True)
    o = oracle.OracleSolver.from_system(s, scheme="cptr")
    abar, W = o.scaled()
    D = diag_blocks(s, abar)
    sidx = [k for k in range(nb) if k not in (p, t)]
    scale = np.abs(diag_blocks(s)).max(axis=(1, 2))
    if sidx:   # Z_es of Eq. CPTR1
        for e in (p, t):
            assert np.max(np.abs(D[:, e, :][:, sidx]) / scale[:, None]) < 1e-13
    for r in sidx:
        assert np.all(W[:, r, :] == np.eye(nb)[r])
    # unit lower triangular in [s, e]: the e rows change only in s columns
    for e in (p, t):
        cols = [k for k in range(nb) if k not in sidx]
        assert np.all(W[:, e, :][:, cols] == np.eye(nb)[e][cols])
    assert np.allclose(np.linalg.det(W), 1.0, atol=1e-12)
    A = bsr_dense(s.row_ptr, s.col_idx, s.vals)
    Ab = bsr_dense(s.row_ptr, s.col_idx, abar)
    assert np.allclose(np.linalg.solve(A, s.b), np.linalg.solve(Ab, o.scale_rhs(s.b)),
                       rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("stage3", [0, 1])
def test_cptr_matches_two_stage_formula(stage3):
    s = sy.make_system(5, 4, 4, pe=1.0, seed=5)
    o = oracle.OracleSolver.from_system(s, scheme="cptr", stage3=stage3, max_coarse=3)
    abar, _ = o.scaled()
    A = bsr_dense(s.row_ptr, s.col_idx, abar)
    n = A.shape[0]
    I = np.eye(n)
    M = operator_matrix(o.apply, n)
    M1 = operator_matrix(lambda r: o.stage(1, r), n)
    M2 = operator_matrix(lambda r: o.stage(2, r), n)
    ref = M1 + M2 @ (I - A @ M1)
    assert np.max(np.abs(M - ref)) <= 1e-12 * np.abs(M).max()
    assert np.max(np.abs((I - A @ M) - (I - A @ M2) @ (I - A @ M1))) <= 1e-11 * max(
        1.0, np.abs(I - A @ M).max())


def test_cptr_stage_acts_on_pressure_and_temperature_only():
    s = sy.make_system(4, 4, 5, pe=10.0, seed=2, p_idx=3, t_idx=0)
    o = oracle.OracleSolver.from_system(s, scheme="cptr", max_coarse=4)
    r = np.random.default_rng(0).standard_normal(s.n_cells * 5)
    y = o.stage(1, r).reshape(-1, 5)
    assert np.all(y[:, [1, 2, 4]] == 0.0) and np.any(y[:, 0] != 0.0) and np.any(y[:, 3] != 0.0)
    r2 = r.reshape(-1, 5).copy()
    r2[:, [1, 2, 4]] = np.random.default_rng(1).standard_normal((s.n_cells, 3))
    assert np.array_equal(o.stage(1, r2.reshape(-1)), o.stage(1, r))   # reads r_e only


@pytest.mark.parametrize("stage3,order", [(0, 0), (0, 2), (1, 0)])
def test_cptr_exact_on_triangular_family(stage3, order):
    # Abar = [A_ss A_se; 0 B_ee] with A_ss block diagonal: the residual left
    # by an exact first stage has s components only, on which the last stage
    # is exact (its factors keep zero s columns off the diagonal blocks)
    s = sy.make_system(6, 5, 5, family="triangular", pe=1.0, seed=7)
    o = oracle.OracleSolver.from_system(s, scheme="cptr", exact_sub=1, stage3=stage3,
                                        ilu_order=order)
    x, info = o.fgmres(o.scale_rhs(s.b), tol=1e-10, maxit=5)
    assert info["status"] == 0 and info["iters"] == 1
    s2 = sy.make_system(6, 5, 5, pe=1.0, seed=7)
    o2 = oracle.OracleSolver.from_system(s2, scheme="cptr", exact_sub=1, stage3=stage3,
                                         ilu_order=order)
    _, info2 = o2.fgmres(o2.scale_rhs(s2.b), tol=1e-10, maxit=50)
    assert info2["iters"] > 1


# ---- system AMG ---------------------------------------------------------------
def _coupled_poisson(nx, ny, c=(0.3, -0.2), d=(1.0, 2.0)):
    """2 x 2 blocks on the 5-point Poisson graph: block (i, j) = a_ij times
    [[d0, c0], [c1, d1]] (the scalar Poisson entries a_ij)."""
    rp, ci, v = sy.poisson_csr(nx, ny)
    K = np.array([[d[0], c[0]], [c[1], d[1]]])
    return rp, ci, v[:, None, None] * K[None]


def test_system_split_is_pmis_on_block_norms():
    s = sy.make_system(14, 11, 4, pe=10.0, sigma=1.0, seed=4)
    o = oracle.OracleSolver.from_system(s, scheme="cptr", max_coarse=10)
    abar, _ = o.scaled()
    lev = o.amg_levels(1)
    assert len(lev) >= 3
    # level 0 is B_ee in the interleaved scalar form
    rp, ci = s.row_ptr, s.col_idx
    B = abar[:, [0, 1]][:, :, [0, 1]]
    rows = np.repeat(np.arange(s.n_cells), np.diff(rp))
    q = B.reshape(-1, 4)
    f = np.sqrt(((q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1]) + q[:, 2] * q[:, 2]) + q[:, 3] * q[:, 3])
    nrm = np.where(ci == rows, f, -f)
    _, _, _, cf = oracle.pmis_rounds(rp, ci, nrm, seed=0x5eed, level=0)
    assert np.array_equal(lev[0].cf, np.repeat(cf, 2))
    # P: unknown k of point i interpolates from unknown k of C points only,
    # with the classical weights of that unknown's scalar matrix on the split
    P = lev[0].P
    for k in (0, 1):
        _, _, Pk = oracle.interp_only(rp, ci, B[:, k, k], cf=cf)
        for i in range(s.n_cells):
            a, b = P[0][2 * i + k], P[0][2 * i + k + 1]
            assert np.all(P[1][a:b] % 2 == k)
            assert np.array_equal(P[1][a:b] // 2, Pk[1][Pk[0][i]:Pk[0][i + 1]])
            assert np.array_equal(P[2][a:b], Pk[2][Pk[0][i]:Pk[0][i + 1]])


def test_system_coarse_operators_are_galerkin_products():
    rp, ci, bv = _coupled_poisson(20, 17)
    h = oracle.OracleAMG.system(rp, ci, bv, max_coarse=20)
    lev = h.levels()
    assert len(lev) >= 3
    for l in range(len(lev) - 1):
        A = csr_dense(*lev[l].A)
        nc = int(lev[l].cf.sum())
        Pd = csr_dense(*lev[l].P, ncols=nc)
        Ac = csr_dense(*lev[l + 1].A, ncols=nc)
        assert np.allclose(Ac, Pd.T @ A @ Pd, rtol=0, atol=1e-12 * np.abs(Ac).max())


def test_uncoupled_identical_unknowns_give_two_scalar_vcycles():
    # blocks a_ij I: the norms are sqrt(2)|a_ij|, so strength, split and both
    # unknowns' interpolation equal the scalar hierarchy's, and block Jacobi
    # is point Jacobi
    rp, ci, bv = _coupled_poisson(1, 300, c=(0.0, 0.0), d=(1.0, 1.0))
    sysh = oracle.OracleAMG.system(rp, ci, bv, max_coarse=8)
    sc = oracle.OracleAMG(*sy.poisson_csr(1, 300), max_coarse=8)
    assert sysh.nlev() == sc.nlev() >= 3
    rng = np.random.default_rng(3)
    b1, b2 = rng.standard_normal(300), rng.standard_normal(300)
    x = sysh.vcycle(np.stack([b1, b2], axis=1).reshape(-1)).reshape(-1, 2)
    assert np.allclose(x[:, 0], sc.vcycle(b1), rtol=0, atol=1e-12 * np.abs(x).max())
    assert np.allclose(x[:, 1], sc.vcycle(b2), rtol=0, atol=1e-12 * np.abs(x).max())


def test_system_vcycle_converges_at_a_size_independent_rate():
    rates = []
    for n in (24, 48, 96):
        rp, ci, bv = _coupled_poisson(n, n)
        h = oracle.OracleAMG.system(rp, ci, bv, max_coarse=50)
        A = None
        # error propagation e <- e - M A e from a random start, 8 cycles
        lev = h.levels()
        A = lev[0].A
        e = np.random.default_rng(n).standard_normal(2 * n * n)
        first = np.linalg.norm(e)
        for _ in range(8):
            Ae = np.zeros_like(e)
            for i in range(len(A[0]) - 1):
                Ae[i] = np.dot(A[2][A[0][i]:A[0][i + 1]], e[A[1][A[0][i]:A[0][i + 1]]])
            e = e - h.vcycle(Ae)
        rates.append((np.linalg.norm(e) / first) ** (1 / 8))
    # the scalar hierarchy's bounds on 2D Poisson (PMIS, direct classical
    # interpolation, damped Jacobi): near 0.6 at most and mild growth; a
    # wrong sign, a transposed restriction or a dropped coupling block drives
    # the rate to or above 1
    assert max(rates) < 0.72, rates
    assert rates[-1] - rates[0] < 0.2, rates


def test_cptr_trend_between_cpr_and_cptr3():
    # unit Peclet (Sec. 5.1): CPTR with system AMG needs far fewer iterations
    # than CPR
    s = sy.make_system(32, 32, 4, pe=1.0)
    it = {}
    for scheme in ("cpr", "cptr"):
        o = oracle.OracleSolver.from_system(s, scheme=scheme, max_coarse=40, restart=100)
        _, info = o.fgmres(o.scale_rhs(s.b), tol=1e-8, maxit=400, restart=100)
        assert info["status"] == 0
        it[scheme] = info["iters"]
    assert it["cptr"] * 2 < it["cpr"], it
