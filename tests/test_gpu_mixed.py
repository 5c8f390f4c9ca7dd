"""Mixed-precision preconditioner (BF16 storage, FP32 sweeps) against the
FP64 oracle.

The mixed form changes only M^{-1}; the outer FGMRES (flexible in the
preconditioner, Sec. 5.1) stays FP64, so the bars are on the FP64 system:
* the converged solve meets the FP64 tolerance on the scaled system and on
  the unscaled one, ||b - A x|| <= 1e-6 ||b||;
* the solution agrees with the oracle's (FP64 preconditioner, driven to a
  tighter tolerance) to the accuracy the tolerance allows;
* one application differs from the oracle's FP64 application by what BF16
  storage explains (about 2^-8 per entry, a few of those through the stages)
  and not by less than FP32 rounding (the reduced path really ran);
* the operator is linear and deterministic (same bits on a repeat).
Iteration counts are reported, and may differ from the FP64 counts.
"""
import numpy as np
import pytest

import oracle
from paper_1912_04385_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sps = pytest.importorskip("scipy.sparse")


@pytest.fixture(scope="module")
def mss():
    from paper_1912_04385_gb300 import build, mss as m
    build.build()
    m.load()
    return m


CASES = [
    dict(nx=32, ny=32, nb=4, pe=1.0),
    dict(nx=37, ny=23, nb=6, pe=10.0, sigma=2.0, band=True, seed=3),
    dict(nx=29, ny=31, nb=5, pe=1000.0, sigma=1.0, band=True, seed=4, p_idx=2, t_idx=4),
    dict(nx=64, ny=48, nb=6, pe=10.0, sigma=3.0, band=True, seed=11),
]


def _sys(c):
    c = dict(c)
    return sy.make_system(c.pop("nx"), c.pop("ny"), c.pop("nb"), **c)


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def _n(t):
    return t.detach().cpu().numpy()


def _bsr(s):
    n = s.n_cells
    v = np.asarray(s.vals, np.float64).reshape(-1, s.nb, s.nb)
    return sps.bsr_matrix((v, s.col_idx, s.row_ptr), shape=(n * s.nb, n * s.nb))


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("scheme", ["cptr3", "cpr", "ilu0"])
def test_mixed_solve_meets_fp64_tolerance(mss, case, scheme):
    if scheme == "ilu0" and case == 3:
        pytest.skip("block ILU(0) alone stalls on this sigma = 3 field in FP64 too (Sec. 5.1)")
    s = _sys(CASES[case])
    kw = dict(scheme=scheme, restart=60, amg_max_coarse=40)
    g64 = mss.Solver().setup_system(s, **kw)
    gmx = mss.Solver().setup_system(s, precision="mixed", **kw)
    x64, i64 = g64.solve(_t(s.b), tol=1e-8, maxit=600)
    xmx, imx = gmx.solve(_t(s.b), tol=1e-8, maxit=600)
    assert i64["status"] == 0 and imx["status"] == 0, (i64, imx)
    assert imx["rel_res_true"] <= 1e-8
    A = _bsr(s)
    x = _n(xmx)
    assert np.linalg.norm(s.b - A @ x) <= 1e-6 * np.linalg.norm(s.b)
    # the oracle's solution, converged further
    o = oracle.OracleSolver.from_system(s, scheme=scheme, restart=60, max_coarse=40)
    xo, io = o.fgmres(o.scale_rhs(s.b), tol=1e-12, maxit=1200)
    assert io["status"] == 0
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    err64 = np.linalg.norm(_n(x64) - xo) / np.linalg.norm(xo)
    print(f"case {case} {scheme}: iters fp64 {i64['iters']} mixed {imx['iters']}, "
          f"rel err fp64 {err64:.2e} mixed {err:.2e}")
    # both stop at the same scaled-residual tolerance: the errors are alike
    assert err <= max(100 * err64, 1e-6)
    # BF16 storage must not wreck the preconditioner
    assert imx["iters"] <= 2 * i64["iters"] + 5


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("scheme,stage3,order,ilu", [
    ("cptr3", 0, 0, 2), ("cptr3", 0, 1, 2), ("cptr3", 1, 0, 2), ("cptr3", 0, 0, 0),
    ("cpr", 0, 0, 2), ("ilu0", 0, 0, 2)])
def test_mixed_apply_close_to_oracle(mss, case, scheme, stage3, order, ilu):
    s = _sys(CASES[case])
    kw = dict(scheme=scheme, stage3=stage3, stage_order=order, ilu_order=ilu)
    g = mss.Solver().setup_system(s, precision="mixed", amg_max_coarse=40, **kw)
    o = oracle.OracleSolver.from_system(s, max_coarse=40, **kw)
    rng = np.random.default_rng(100 + case)
    r = rng.standard_normal(s.n_cells * s.nb)
    y = _n(g.apply(_t(r)))
    yo = o.apply(r)
    d = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    print(f"case {case} {scheme}/{stage3}/{order}/{ilu}: mixed vs fp64 apply {d:.2e}")
    assert 1e-7 < d < 5e-2
    # linear (no state kept between applications) and deterministic
    r2 = rng.standard_normal(r.size)
    y2 = _n(g.apply(_t(r2)))
    y12 = _n(g.apply(_t(2.0 * r - 0.5 * r2)))
    lin = np.linalg.norm(y12 - (2.0 * y - 0.5 * y2)) / np.linalg.norm(y12)
    assert lin < 1e-5, lin
    assert np.array_equal(_n(g.apply(_t(r))), y)


def test_mixed_stage_apply_stays_fp64(mss):
    # the per-stage entry point is FP64 whatever the precision option
    s = _sys(CASES[1])
    g = mss.Solver().setup_system(s, precision="mixed", amg_max_coarse=40)
    o = oracle.OracleSolver.from_system(s, max_coarse=40)
    r = np.random.default_rng(5).standard_normal(s.n_cells * s.nb)
    for which in (0, 1, 2):
        a = _n(g.stage(which, _t(r)))
        b = o.stage(which, r)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_mixed_solve_deterministic_and_host_path(mss):
    s = _sys(CASES[3])
    g = mss.Solver().setup_system(s, precision="mixed")
    x1, i1 = g.solve(_t(s.b), tol=1e-8, maxit=400)
    x2, i2 = g.solve(_t(s.b), tol=1e-8, maxit=400)
    assert i1["iters"] == i2["iters"] and torch.equal(x1, x2)
    h = mss.Solver()
    xh, ih = h.solve_host(s, tol=1e-8, maxit=400, precision="mixed")
    assert ih["iters"] == i1["iters"]
    assert np.array_equal(xh, _n(x1))


def test_precision_option_checked(mss):
    s = _sys(CASES[0])
    with pytest.raises(mss.MssError) as e:
        mss.Solver().setup_system(s, precision=7)
    assert e.value.status == mss.ERR_INVALID_ARG


def test_mixed_multicolour_gauss_seidel(mss):
    # the multicolour Gauss-Seidel smoother in the mixed form (BF16 operators,
    # FP32 sweeps) still reaches the FP64 tolerance
    s = _sys(CASES[1])
    kw = dict(scheme="cptr3", smoother="mcsgs", restart=60, amg_max_coarse=40)
    g64 = mss.Solver().setup_system(s, **kw)
    gmx = mss.Solver().setup_system(s, precision="mixed", **kw)
    x64, i64 = g64.solve(_t(s.b), tol=1e-8, maxit=600)
    xmx, imx = gmx.solve(_t(s.b), tol=1e-8, maxit=600)
    assert i64["status"] == 0 and imx["status"] == 0, (i64, imx)
    assert imx["rel_res_true"] <= 1e-8 and abs(imx["iters"] - i64["iters"]) <= 2
    A = _bsr(s)
    assert np.linalg.norm(s.b - A @ _n(xmx)) <= 1e-6 * np.linalg.norm(s.b)
