"""Newton-loop reuse (Sec. 2.5): mss_update_values through the C-ABI.

* reuse "pattern": the handle after the update equals a new mss_setup with the
  new values bit for bit -- scaled matrix, both hierarchies, ordering,
  factors, one application and the whole solve, with both drivers and in the
  mixed form;
* reuse "coarsening": against the oracle's update with the kept C/F splits,
  the hierarchies bit for bit, one application within 1e-12, FGMRES
  iterations within +-1;
* errors: another pattern, no set-up, an unknown reuse mode, the old matrix
  passed to the solve.
"""
import numpy as np
import pytest

import oracle
from paper_1912_04385_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

APPLY_TOL = 1e-12


@pytest.fixture(scope="module")
def mss():
    from paper_1912_04385_gb300 import build, mss as m
    build.build()
    m.load()
    return m


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _n(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / max(float(np.max(np.abs(b))), 1e-300))


SEQ = [dict(pe=10.0, seed=3), dict(pe=40.0, seed=4), dict(pe=5.0, seed=5)]


def _seq(nx=37, ny=23, nb=6):
    out = [sy.make_system(nx, ny, nb, sigma=2.0, band=True, **c) for c in SEQ]
    for s in out[1:]:
        assert np.array_equal(s.col_idx, out[0].col_idx)
    return out


def _state(g):
    levels = [[(*(_n(x) for x in L["A"]), None if L["cf"] is None else _n(L["cf"]))
               for L in g.amg_levels(w)] for w in (0, 1)]
    fv, fd = g.bilu_factors()
    nc, colour, perm = g.bilu_ordering()
    return _n(g.scaled()), levels, _n(fv), _n(fd), nc, _n(colour), _n(perm)


def _same_state(a, b):
    assert np.array_equal(a[0], b[0])
    for la, lb in zip(a[1], b[1]):
        assert len(la) == len(lb)
        for x, y in zip(la, lb):
            for u, v in zip(x, y):
                assert (u is None and v is None) or np.array_equal(u, v)
    for k in (2, 3, 5, 6):
        assert np.array_equal(a[k], b[k])
    assert a[4] == b[4]


@pytest.mark.parametrize("driver", ["host", "graph"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_update_equals_new_setup(mss, driver, precision):
    seq = _seq()
    kw = dict(amg_max_coarse=40, restart=60, driver=driver, precision=precision)
    rp, ci = _t(seq[0].row_ptr), _t(seq[0].col_idx)
    g = mss.Solver().setup(rp, ci, _t(seq[0].vals.reshape(-1)), 6, **kw)
    x0, i0 = g.solve(_t(seq[0].b), tol=1e-8, maxit=300)   # the graph is captured here
    assert i0["status"] == 0
    r = _t(np.random.default_rng(7).standard_normal(seq[0].n_cells * 6))
    for s in seq[1:]:
        v = _t(s.vals.reshape(-1))
        g.update_values(v)
        f = mss.Solver().setup(rp, ci, v, 6, **kw)
        _same_state(_state(g), _state(f))
        assert torch.equal(g.apply(r), f.apply(r))
        xg, ig = g.solve(_t(s.b), tol=1e-8, maxit=300)
        xf, if_ = f.solve(_t(s.b), tol=1e-8, maxit=300)
        assert ig["status"] == 0 and ig["iters"] == if_["iters"]
        assert torch.equal(xg, xf)


def test_update_with_kept_coarsening_against_the_oracle(mss):
    seq = _seq()
    rp, ci = _t(seq[0].row_ptr), _t(seq[0].col_idx)
    g = mss.Solver().setup(rp, ci, _t(seq[0].vals.reshape(-1)), 6, amg_max_coarse=40,
                           restart=60)
    o = oracle.OracleSolver.from_system(seq[0], max_coarse=40, restart=60)
    for s in seq[1:]:
        g.update_values(_t(s.vals.reshape(-1)), reuse="coarsening")
        o = o.updated(s.vals, reuse=1)      # chained: the first set-up's splits
        for which in (0, 1):
            lg, lo = g.amg_levels(which), o.amg_levels(which)
            assert len(lg) == len(lo)
            for a, b in zip(lg, lo):
                for k in range(3):
                    assert np.array_equal(_n(a["A"][k]), b.A[k]), (which, k)
                if b.cf is not None:
                    assert np.array_equal(_n(a["cf"]), b.cf)
                    for k in range(3):
                        assert np.array_equal(_n(a["P"][k]), b.P[k])
        r = np.random.default_rng(3).standard_normal(s.n_cells * 6)
        assert _rel(_n(g.apply(_t(r))), o.apply(r)) < APPLY_TOL
        xg, ig = g.solve(_t(s.b), tol=1e-8, maxit=300)
        xo, io = o.fgmres(o.scale_rhs(s.b), tol=1e-8, maxit=300, restart=60)
        assert ig["status"] == 0 and io["status"] == 0
        assert abs(ig["iters"] - io["iters"]) <= 1, (ig["iters"], io["iters"])


def test_update_errors(mss):
    seq = _seq()
    rp, ci = _t(seq[0].row_ptr), _t(seq[0].col_idx)
    v0 = _t(seq[0].vals.reshape(-1))
    fresh = mss.Solver()
    with pytest.raises(mss.MssError) as e:
        fresh._Jt = (rp, ci, v0)
        fresh.update_values(v0)
    assert e.value.status == mss.ERR_NOT_SETUP
    g = mss.Solver().setup(rp, ci, v0, 6, amg_max_coarse=40)
    # another pattern of the same size: two columns of one row swapped
    ci2 = seq[0].col_idx.copy()
    row = 40
    a, b = seq[0].row_ptr[row], seq[0].row_ptr[row] + 1
    ci2[[a, b]] = ci2[[b, a]]
    with pytest.raises(mss.MssError) as e:
        g.update_values(v0, col_idx=_t(ci2))
    assert e.value.status == mss.ERR_INVALID_ARG
    with pytest.raises(KeyError):
        g.update_values(v0, reuse="everything")
    # a valid update afterwards; the solve then needs the new matrix
    v1 = _t(seq[1].vals.reshape(-1))
    old_J = g._J
    g.update_values(v1)
    x, info = g.solve(_t(seq[1].b), tol=1e-8, maxit=300)
    assert info["status"] == 0
    g._J = old_J
    with pytest.raises(mss.MssError) as e:
        g.solve(_t(seq[1].b), tol=1e-8, maxit=300)
    assert e.value.status == mss.ERR_NOT_SETUP
