"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Bars (FP64 everywhere):
* index work and set-up values that feed index decisions -- the scaled
  blocks, C/F splits, interpolation operators, Galerkin coarse operators and
  the multicolour ordering -- must match bit for bit (both sides evaluate
  the same definition in the same order without FMA contraction);
* operators whose summation order differs (V-cycles with a dense coarse
  inverse versus LU, block ILU sweeps, the full preconditioner) must agree
  to 1e-12 relative in the max norm;
* FGMRES: converged iteration counts within +-1, and the solutions after the
  same number of iterations (tol = 0) within 1e-8 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1912_04385_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

APPLY_TOL = 1e-12
SOL_TOL = 1e-8
# Factors in the max norm relative to the largest entry: both sides run the
# same IKJ elimination and no-pivot Gauss-Jordan, differing only in rounding
# (FMA on the GPU, numpy's inverse for U_qq^-1 on the oracle side).
FACTOR_TOL = 1e-12


@pytest.fixture(scope="module")
def mss():
    from paper_1912_04385_gb300 import build, mss as m
    build.build()
    m.load()
    return m


def _gpu(mss, s, **kw):
    return mss.Solver().setup_system(s, **kw)


def _orc(s, **kw):
    return oracle.OracleSolver.from_system(s, **kw)


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def _n(t):
    return t.detach().cpu().numpy()


CASES = [
    dict(nx=32, ny=32, nb=4, pe=1.0),                                  # the small case
    dict(nx=37, ny=23, nb=6, pe=10.0, sigma=2.0, band=True, seed=3),   # ragged, heterogeneous
    dict(nx=29, ny=31, nb=5, pe=1000.0, sigma=1.0, band=True, seed=4, p_idx=2, t_idx=4),
    dict(nx=40, ny=1, nb=3, pe=0.1, seed=5, p_idx=1, t_idx=0),          # 1D
]


def _sys(c):
    c = dict(c)
    return sy.make_system(c.pop("nx"), c.pop("ny"), c.pop("nb"), **c)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("scheme", ["cptr3", "cpr", "ilu0", "cptr"])
def test_scaled_matrix_bit_exact(mss, case, scheme):
    s = _sys(CASES[case])
    g = _gpu(mss, s, scheme=scheme)
    o = _orc(s, scheme=scheme)
    ab_o, _ = o.scaled()
    ab_g = _n(g.scaled())
    assert np.array_equal(ab_g, ab_o)
    b = s.b
    assert np.array_equal(_n(g.scale_rhs(_t(b))), o.scale_rhs(b))


@pytest.mark.parametrize("case", range(len(CASES)))
def test_amg_hierarchy_bit_exact(mss, case):
    s = _sys(CASES[case])
    kw = dict(scheme="cptr3", amg_max_coarse=10)
    g = _gpu(mss, s, **kw)
    o = _orc(s, scheme="cptr3", max_coarse=10)
    for which in (0, 1):
        lg, lo = g.amg_levels(which), o.amg_levels(which)
        assert len(lg) == len(lo) >= 2
        for a, b in zip(lg, lo):
            for k in range(3):
                assert np.array_equal(_n(a["A"][k]), b.A[k]), (which, k)
            if b.cf is None:
                assert a["cf"] is None
                continue
            assert np.array_equal(_n(a["cf"]), b.cf)
            for k in range(3):
                assert np.array_equal(_n(a["P"][k]), b.P[k])


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("order,strip", [(2, 32), (2, 5), (3, 32), (3, 5), (0, 1)])
def test_ordering_bit_exact(mss, case, order, strip):
    s = _sys(CASES[case])
    g = _gpu(mss, s, ilu_order=order, ilu_strip=strip)
    o = _orc(s, ilu_order=order, ilu_strip=strip)
    nc, colour, perm = g.bilu_ordering()
    f = o.bilu()
    assert nc == f["ncolours"]
    assert np.array_equal(_n(colour), f["colour"])
    assert np.array_equal(_n(perm), f["perm"])


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("order,strip", [(2, 32), (2, 5), (3, 32), (0, 1)])
def test_factor_forms(mss, case, order, strip):
    # Both factorisation kernels, forced on every colour: the same bits as
    # each other, the oracle's factors element by element, and the last stage
    # (which reads them) against the oracle's.
    from tests.helpers import stored_factor_form
    s = _sys(CASES[case])
    kw = dict(ilu_order=order, ilu_strip=strip)
    gw = _gpu(mss, s, factor_form="warp", **kw)
    gl = _gpu(mss, s, factor_form="lanes", **kw)
    fw, dw = gw.bilu_factors()
    fl, dl = gl.bilu_factors()
    assert torch.equal(fw, fl) and torch.equal(dw, dl)
    o = _orc(s, **kw)
    efv, edinv = stored_factor_form(o.bilu(), strip if order in (2, 3) else 1)
    assert _rel(_n(fl), efv) < FACTOR_TOL
    assert _rel(_n(dl), edinv) < FACTOR_TOL
    r = np.random.default_rng(case).standard_normal(s.n_cells * s.nb)
    ref = o.stage(2, r)
    for g in (gw, gl):
        assert _rel(_n(g.stage(2, _t(r))), ref) < APPLY_TOL


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("scheme,stage3,smoother,order,ilu", [
    ("cptr3", 0, "jacobi", 0, 2), ("cptr3", 0, "jacobi", 0, 0), ("cptr3", 1, "jacobi", 0, 2),
    ("cptr3", 0, "chebyshev", 0, 2), ("cptr3", 0, "jacobi", 1, 2), ("cptr3", 0, "jacobi", 0, 3),
    ("cpr", 0, "jacobi", 0, 2),
    ("ilu0", 0, "jacobi", 0, 2), ("ilu0", 0, "jacobi", 0, 0)])
def test_stages_and_apply(mss, case, scheme, stage3, smoother, order, ilu):
    s = _sys(CASES[case])
    g = _gpu(mss, s, scheme=scheme, stage3=stage3, smoother=smoother, stage_order=order,
             amg_max_coarse=40, ilu_order=ilu)
    o = _orc(s, scheme=scheme, stage3=stage3, smoother=smoother, stage_order=order,
             max_coarse=40, ilu_order=ilu)
    rng = np.random.default_rng(case)
    r = rng.standard_normal(s.n_cells * s.nb)
    rt = _t(r)
    stages = [2] + ([1] if scheme != "ilu0" else []) + ([0] if scheme == "cptr3" else [])
    for which in stages:
        assert _rel(_n(g.stage(which, rt)), o.stage(which, r)) < APPLY_TOL, which
    assert _rel(_n(g.apply(rt)), o.apply(r)) < APPLY_TOL
    x = rng.standard_normal(s.n_cells * s.nb)
    assert _rel(_n(g.spmv(_t(x))), o.spmv(x)) < 1e-14


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("scheme,orthog", [("cptr3", 0), ("cptr3", 1), ("cpr", 0), ("ilu0", 0)])
def test_fgmres_iterations_and_solution(mss, case, scheme, orthog):
    s = _sys(CASES[case])
    m = 100
    g = _gpu(mss, s, scheme=scheme, restart=m, amg_max_coarse=40, orthog=orthog)
    o = _orc(s, scheme=scheme, restart=m, max_coarse=40)
    bb = o.scale_rhs(s.b)
    xo, io = o.fgmres(bb, tol=1e-8, maxit=400, restart=m)
    xg, ig = g.solve(_t(s.b), tol=1e-8, maxit=400)
    assert io["status"] == 0 and ig["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1, (ig["iters"], io["iters"])
    assert ig["rel_res_true"] <= 1e-8
    # same number of iterations, no stopping test
    k = min(io["iters"], 45)
    xo, io2 = o.fgmres(bb, tol=0.0, maxit=k, restart=m)
    xg, ig2 = g.solve(_t(s.b), tol=0.0, maxit=k)
    assert ig2["iters"] == io2["iters"] == k
    assert np.linalg.norm(_n(xg) - xo) <= SOL_TOL * np.linalg.norm(xo)


@pytest.mark.parametrize("stage3", [0, 1])
def test_triangular_family_one_iteration_on_gpu(mss, stage3):
    # Upper-block-triangular scaled matrix in [s, P, T]: with exact T and P
    # stages (a one-level hierarchy is a direct solve) the residual left for
    # the last stage has s components only, on which block ILU(0) (any
    # ordering) and block Jacobi are exact, so M^-1 = Abar^-1.
    s = sy.make_system(6, 5, 5, family="triangular", pe=1.0, seed=7)
    g = _gpu(mss, s, scheme="cptr3", stage3=stage3, amg_max_coarse=1000)
    x, info = g.solve(_t(s.b), tol=1e-10, maxit=5)
    assert info["iters"] == 1 and info["rel_res_true"] < 1e-10


def test_host_solve_matches_device_solve(mss):
    s = sy.make_system(30, 20, 6, pe=10.0, sigma=2.0, band=True, seed=9)
    g = _gpu(mss, s)
    xd, idv = g.solve(_t(s.b), tol=1e-8, maxit=300)
    h = mss.Solver()
    xh, ih = h.solve_host(s, tol=1e-8, maxit=300)
    assert ih["iters"] == idv["iters"]
    assert np.array_equal(xh, _n(xd))


@pytest.mark.parametrize("nb", [2, 3, 7, 8, 9, 10, 13, 14, 16])
def test_block_sizes(mss, nb):
    s = sy.make_system(19, 17, nb, pe=1.0, seed=nb)
    g = _gpu(mss, s, amg_max_coarse=30)
    o = _orc(s, max_coarse=30)
    r = np.random.default_rng(nb).standard_normal(s.n_cells * nb)
    assert _rel(_n(g.apply(_t(r))), o.apply(r)) < APPLY_TOL


def test_single_cell_and_column_major(mss):
    s = sy.make_system(1, 1, 4, seed=1)
    g = _gpu(mss, s)
    o = _orc(s)
    r = np.random.default_rng(0).standard_normal(4)
    assert _rel(_n(g.apply(_t(r))), o.apply(r)) < APPLY_TOL
    s2 = sy.make_system(11, 7, 5, pe=10.0, seed=2)
    vt = np.ascontiguousarray(np.transpose(s2.vals, (0, 2, 1)))
    rp = torch.from_numpy(s2.row_ptr).cuda()
    ci = torch.from_numpy(s2.col_idx).cuda()
    gc = mss.Solver().setup(rp, ci, _t(vt.reshape(-1)), 5, 0, 1, col_major=True)
    gr = _gpu(mss, s2)
    assert torch.equal(gc.scaled(), gr.scaled())


def test_error_statuses(mss):
    s = sy.make_system(6, 6, 4, seed=0)
    ci = s.col_idx.copy()
    ci[[1, 2]] = ci[[2, 1]]
    bad = sy.BlockSystem(s.row_ptr, ci, s.vals, s.b, 6, 6, 4)
    with pytest.raises(mss.MssError) as e:
        _gpu(mss, bad)
    assert e.value.status == mss.ERR_INVALID_ARG
    vals = s.vals.copy()
    vals[:] = 0.0
    with pytest.raises(mss.MssError) as e:
        _gpu(mss, sy.BlockSystem(s.row_ptr, s.col_idx, vals, s.b, 6, 6, 4))
    assert e.value.status == mss.ERR_SINGULAR_BLOCK
    g = _gpu(mss, s)
    x, info = g.solve(_t(s.b), tol=1e-14, maxit=3)
    assert info["status"] == mss.ERR_NOT_CONVERGED and info["iters"] == 3
    assert np.all(np.isfinite(_n(x)))
    nanb = s.b.copy()
    nanb[5] = np.nan
    with pytest.raises(mss.MssError) as e:
        g.solve(_t(nanb), tol=1e-8, maxit=10)
    assert e.value.status == mss.ERR_BREAKDOWN
    with pytest.raises(mss.MssError) as e:
        mss.Solver().setup_system(s, restart=500)
    assert e.value.status == mss.ERR_INVALID_ARG


@pytest.mark.parametrize("nb", [4, 6])
def test_residual_norm_entry_point(mss, nb):
    from tests.helpers import bsr_dense
    s = sy.make_system(23, 17, nb, pe=10.0, seed=31)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(s.n_cells * nb)
    A = bsr_dense(s.row_ptr, s.col_idx, s.vals)
    ref_r = np.linalg.norm(s.b - A @ x)
    ref_b = np.linalg.norm(s.b)
    g = mss.Solver()
    rp = torch.from_numpy(s.row_ptr).cuda()
    ci = torch.from_numpy(s.col_idx).cuda()
    v = _t(s.vals.reshape(-1))
    r, bn = g.residual_norm(rp, ci, v, nb, _t(s.b), _t(x))
    assert abs(r - ref_r) <= 1e-12 * ref_r
    assert abs(bn - ref_b) <= 1e-12 * ref_b
    r2, bn2 = g.residual_norm(rp, ci, v, nb, _t(s.b), _t(x))
    assert r2 == r and bn2 == bn


@pytest.mark.parametrize("scheme,smoother,precision", [("cptr3", "jacobi", "fp64"),
                                                       ("cptr3", "chebyshev", "fp64"),
                                                       ("cptr3", "mcsgs", "fp64"),
                                                       ("cpr", "jacobi", "fp64"),
                                                       ("cptr", "jacobi", "fp64")])
def test_larger_hierarchy(mss, scheme, smoother, precision):
    # a 6,144-cell system: several AMG levels above 4,096 rows, stage and
    # whole-preconditioner parity, and the FGMRES iteration bar
    s = sy.make_system(96, 64, 4, pe=10.0, sigma=2.0, band=True, seed=12)
    g = _gpu(mss, s, scheme=scheme, smoother=smoother, amg_max_coarse=100)
    o = _orc(s, scheme=scheme, smoother=smoother, max_coarse=100)
    r = np.random.default_rng(12).standard_normal(s.n_cells * s.nb)
    rt = _t(r)
    for which in ([0, 1] if scheme == "cptr3" else [1]):
        assert _rel(_n(g.stage(which, rt)), o.stage(which, r)) < APPLY_TOL, which
    assert _rel(_n(g.apply(rt)), o.apply(r)) < APPLY_TOL
    xo, io = o.fgmres(o.scale_rhs(s.b), tol=1e-8, maxit=300, restart=50)
    g2 = _gpu(mss, s, scheme=scheme, smoother=smoother, amg_max_coarse=100, restart=50)
    xg, ig = g2.solve(_t(s.b), tol=1e-8, maxit=300)
    assert abs(ig["iters"] - io["iters"]) <= 1


@pytest.mark.parametrize("driver", ["host", "graph"])
def test_zero_rhs_and_empty_matrix(mss, driver):
    # b = 0: nothing to iterate; x = 0, no iterations, status OK
    s = _sys(CASES[1])
    g = _gpu(mss, s, driver=driver, restart=100, amg_max_coarse=40)
    x, info = g.solve(_t(np.zeros_like(s.b)), tol=1e-8, maxit=50)
    assert info["status"] == 0 and info["iters"] == 0
    assert not np.any(_n(x))
    # the same handle still solves a nonzero right-hand side afterwards
    x, info = g.solve(_t(s.b), tol=1e-8, maxit=400)
    o = _orc(s, restart=100, max_coarse=40)
    xo, io = o.fgmres(o.scale_rhs(s.b), tol=1e-8, maxit=400, restart=100)
    assert info["status"] == 0 and abs(info["iters"] - io["iters"]) <= 1
    # no cells: rejected at set-up
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    e0 = torch.zeros(0, dtype=torch.int32, device="cuda")
    v0 = torch.zeros(0, dtype=torch.float64, device="cuda")
    with pytest.raises(mss.MssError) as e:
        mss.Solver().setup(z, e0, v0, 4)
    assert e.value.status == mss.ERR_INVALID_ARG


@pytest.mark.parametrize("nu", [(1, 1), (3, 1), (1, 0), (2, 3)])
def test_smoothing_counts(mss, nu):
    # other V(nu_pre, nu_post) counts: the first sweep written by the kernel
    # that forms b, extra pre-sweeps, the prolongation's target for an even or
    # odd number of post-sweeps, both on the per-level kernels (graph) and on
    # the fused coarse levels (host loop)
    s = _sys(CASES[1])
    kw = dict(scheme="cptr3", amg_max_coarse=40, nu_pre=nu[0], nu_post=nu[1])
    g = _gpu(mss, s, **kw)
    o = _orc(s, scheme="cptr3", max_coarse=40, nu_pre=nu[0], nu_post=nu[1])
    r = np.random.default_rng(11).standard_normal(s.n_cells * s.nb)
    assert _rel(_n(g.apply(_t(r))), o.apply(r)) < APPLY_TOL
    gg = _gpu(mss, s, driver="graph", **kw)
    xh, ih = g.solve(_t(s.b), tol=1e-8, maxit=400)
    xg, ig = gg.solve(_t(s.b), tol=1e-8, maxit=400)
    assert ih["status"] == 0 and ih["iters"] == ig["iters"]
    assert torch.equal(xh, xg)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (0, 1)])
def test_multicolour_gauss_seidel(mss, case, nu):
    # the paper's AMG smoother (symmetric Gauss-Seidel, Sec. 5.1) in
    # multicolour form: both AMG stages and the whole preconditioner against
    # the oracle's smoother = 3, the FGMRES iteration bar, graph = host loop
    s = _sys(CASES[case])
    kw = dict(scheme="cptr3", smoother="mcsgs", amg_max_coarse=40, nu_pre=nu[0],
              nu_post=nu[1], restart=100)
    g = _gpu(mss, s, **kw)
    o = _orc(s, scheme="cptr3", smoother="mcsgs", max_coarse=40, nu_pre=nu[0], nu_post=nu[1],
             restart=100)
    r = np.random.default_rng(case).standard_normal(s.n_cells * s.nb)
    rt = _t(r)
    for which in (0, 1):
        assert _rel(_n(g.stage(which, rt)), o.stage(which, r)) < APPLY_TOL, which
    assert _rel(_n(g.apply(rt)), o.apply(r)) < APPLY_TOL
    if nu != (2, 2):
        return
    xo, io = o.fgmres(o.scale_rhs(s.b), tol=1e-8, maxit=400, restart=100)
    xh, ih = g.solve(_t(s.b), tol=1e-8, maxit=400)
    assert io["status"] == 0 and ih["status"] == 0
    assert abs(ih["iters"] - io["iters"]) <= 1, (ih["iters"], io["iters"])
    gg = _gpu(mss, s, driver="graph", **kw)
    xg, ig = gg.solve(_t(s.b), tol=1e-8, maxit=400)
    assert ig["iters"] == ih["iters"] and torch.equal(xg, xh)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_cptr_with_system_amg(mss, case):
    # Sec. 4.2: the system AMG of B_ee bit for bit (split, P, every Galerkin
    # operator in the interleaved scalar form), the first stage, the last
    # stage and the whole two-stage operator within 1e-12, FGMRES within +-1,
    # graph = host loop
    s = _sys(CASES[case])
    kw = dict(scheme="cptr", amg_max_coarse=40, restart=100)
    g = _gpu(mss, s, **kw)
    o = _orc(s, scheme="cptr", max_coarse=40, restart=100)
    lg, lo = g.amg_levels(1), o.amg_levels(1)
    assert len(lg) == len(lo) and g.lib.mss_amg_num_levels(g.h, 0) == 0
    for a, b in zip(lg, lo):
        for k in range(3):
            assert np.array_equal(_n(a["A"][k]), b.A[k]), k
        if b.cf is not None:
            assert np.array_equal(_n(a["cf"]), b.cf)
            for k in range(3):
                assert np.array_equal(_n(a["P"][k]), b.P[k])
    r = np.random.default_rng(case).standard_normal(s.n_cells * s.nb)
    rt = _t(r)
    for which in (1, 2):
        assert _rel(_n(g.stage(which, rt)), o.stage(which, r)) < APPLY_TOL, which
    assert _rel(_n(g.apply(rt)), o.apply(r)) < APPLY_TOL
    with pytest.raises(mss.MssError):
        g.stage(0, rt)                      # CPTR has no temperature stage
    xo, io = o.fgmres(o.scale_rhs(s.b), tol=1e-8, maxit=400, restart=100)
    xh, ih = g.solve(_t(s.b), tol=1e-8, maxit=400)
    assert io["status"] == 0 and ih["status"] == 0
    assert abs(ih["iters"] - io["iters"]) <= 1, (ih["iters"], io["iters"])
    gg = _gpu(mss, s, driver="graph", **kw)
    xg, ig = gg.solve(_t(s.b), tol=1e-8, maxit=400)
    assert ig["iters"] == ih["iters"] and torch.equal(xg, xh)
    # the mixed form (BF16 hierarchy, FP32 sweeps) reaches the FP64 tolerance
    gm = _gpu(mss, s, precision="mixed", **kw)
    xm, im = gm.solve(_t(s.b), tol=1e-8, maxit=400)
    assert im["status"] == 0 and im["rel_res_true"] <= 1e-8


@pytest.mark.parametrize("nb,p,t", [(14, 0, 1), (12, 5, 2), (16, 0, 1)])
@pytest.mark.parametrize("scheme", ["cptr3", "cpr", "cptr"])
def test_paper_block_size(mss, nb, p, t, scheme):
    # the paper's primary systems have 14 unknowns per cell (Sec. 5.1): the
    # scaling bit for bit, both factorisation forms equal, every stage and
    # the whole operator within 1e-12, FGMRES within +-1
    s = sy.make_system(23, 19, nb, pe=10.0, sigma=1.0, band=True, seed=nb, p_idx=p, t_idx=t)
    kw = dict(scheme=scheme, amg_max_coarse=40, restart=100)
    g = _gpu(mss, s, **kw)
    o = _orc(s, scheme=scheme, max_coarse=40, restart=100)
    assert np.array_equal(_n(g.scaled()), o.scaled()[0])
    gw = _gpu(mss, s, factor_form="warp", **kw)
    fl, dl = g.bilu_factors()
    fw, dw = gw.bilu_factors()
    assert torch.equal(fl, fw) and torch.equal(dl, dw)
    r = np.random.default_rng(nb).standard_normal(s.n_cells * nb)
    rt = _t(r)
    stages = [2, 1] + ([0] if scheme == "cptr3" else [])
    for which in stages:
        assert _rel(_n(g.stage(which, rt)), o.stage(which, r)) < APPLY_TOL, which
    assert _rel(_n(g.apply(rt)), o.apply(r)) < APPLY_TOL
    xo, io = o.fgmres(o.scale_rhs(s.b), tol=1e-8, maxit=400, restart=100)
    xg, ig = g.solve(_t(s.b), tol=1e-8, maxit=400)
    assert io["status"] == 0 and ig["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1, (ig["iters"], io["iters"])
