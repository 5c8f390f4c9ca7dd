"""Static condensation (Sec. 3, Eqs. global and reduced) on the GPU through
the C-ABI (mss_condense, mss_recover) against the oracle, and the whole chain
condense -> set-up -> FGMRES -> recover against a dense solve of the global
system.

Bars: A, b and the recovered secondary unknowns within 1e-12 of the oracle
in the max norm relative to the largest entry (one Gauss-Jordan of J22 per
cell and short dot products: the two sides differ by rounding only); the
chain within the FGMRES tolerance times a small factor.
"""
import numpy as np
import pytest

import oracle
from paper_1912_04385_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-12


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
    b = np.asarray(b)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(np.asarray(a) - b)) / max(float(np.max(np.abs(b))), 1e-300))


def _dev(f):
    t = dict(row_ptr=_t(f.row_ptr), col_idx=_t(f.col_idx), j11=_t(f.j11.reshape(-1)),
             j21=_t(f.j21.reshape(-1)), j12=_t(f.j12.reshape(-1)), j22=_t(f.j22.reshape(-1)))
    return dict(tensors=t, n1=f.n1, n2=f.n2)


CASES = [dict(nx=37, ny=23, n1=6, n2=4, sigma=2.0, band=True, pe=10.0),
         dict(nx=29, ny=31, n1=4, n2=1, j21_neighbors=True, pe=1000.0),
         dict(nx=20, ny=17, n1=14, n2=10, j21_neighbors=True),
         dict(nx=33, ny=1, n1=5, n2=16, j21_neighbors=True, pe=0.1, coupling=0.05),
         dict(nx=19, ny=13, n1=6, n2=0)]


def _full(c, seed=3):
    c = dict(c)
    return sy.make_full_system(c.pop("nx"), c.pop("ny"), c.pop("n1"), c.pop("n2"), seed=seed,
                               **c)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_condense_and_recover_against_the_oracle(mss, case):
    f = _full(CASES[case])
    g = mss.Solver()
    fd = _dev(f)
    a, b = g.condense(fd, _t(f.r1), _t(f.r2))
    ao, bo = oracle.condense(f)
    assert _rel(_n(a).reshape(ao.shape), ao) < TOL
    assert _rel(_n(b), bo) < TOL
    d1 = np.random.default_rng(case).standard_normal(f.n_cells * f.n1)
    d2 = g.recover(fd, _t(f.r2), _t(d1))
    assert _rel(_n(d2), oracle.recover(f, d1)) < TOL


@pytest.mark.parametrize("case", [0, 1, 2, 4])
def test_condensed_solve_equals_global_solve(mss, case):
    # the whole chain of Sec. 3: condense, solve the primary system with the
    # multi-stage preconditioner, recover the secondary unknowns
    c = dict(CASES[case])
    if c["n1"] <= 8:
        c.update(nx=12, ny=9)
    else:               # 14 + 10 unknowns per cell: 56 cells keep the dense solve small
        c.update(nx=8, ny=7)
    f = _full(c, seed=8)
    g = mss.Solver()
    fd = _dev(f)
    a, b = g.condense(fd, _t(f.r1), _t(f.r2))
    g.setup(fd["tensors"]["row_ptr"], fd["tensors"]["col_idx"], a.reshape(-1), f.n1, f.p_idx,
            f.t_idx, amg_max_coarse=20, restart=100)
    d1, info = g.solve(b, tol=1e-12, maxit=400)
    assert info["status"] == 0
    d2 = g.recover(fd, _t(f.r2), d1)
    # dense global system, unknowns [primary | secondary]
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
    delta = np.linalg.solve(J, -np.concatenate([f.r1, f.r2]))
    x = np.concatenate([_n(d1), _n(d2)])
    assert np.linalg.norm(x - delta) <= 1e-8 * np.linalg.norm(delta)


def test_condense_at_benchmark_size(mss):
    # 1024 x 1024 cells, 6 primary and 4 secondary unknowns per cell
    f = sy.make_full_system(1024, 1024, 6, 4, seed=0, sigma=2.0, band=True, pe=10.0,
                            j21_neighbors=True)
    g = mss.Solver()
    fd = _dev(f)
    a, b = g.condense(fd, _t(f.r1), _t(f.r2))
    ao, bo = oracle.condense(f)
    assert _rel(_n(a).reshape(ao.shape), ao) < TOL
    assert _rel(_n(b), bo) < TOL
    del ao, bo, a, b
    d1 = np.random.default_rng(1).standard_normal(f.n_cells * 6)
    assert _rel(_n(g.recover(fd, _t(f.r2), _t(d1))), oracle.recover(f, d1)) < TOL


def test_condense_errors(mss):
    f = _full(CASES[0])
    g = mss.Solver()
    fd = _dev(f)
    # a J22 block with a zero pivot
    bad = f.j22.copy()
    bad[7, 0, :] = 0.0
    fd2 = dict(fd, tensors=dict(fd["tensors"], j22=_t(bad.reshape(-1))))
    with pytest.raises(mss.MssError) as e:
        g.condense(fd2, _t(f.r1), _t(f.r2))
    assert e.value.status == mss.ERR_SINGULAR_BLOCK
    # sizes out of range are rejected on the host
    with pytest.raises(mss.MssError) as e:
        g.condense(dict(fd, n2=17), _t(f.r1), _t(f.r2))
    assert e.value.status == mss.ERR_INVALID_ARG
    # a column index out of range is caught by the recovery kernel's check
    ci = f.col_idx.copy()
    ci[5] = f.n_cells + 3
    fd3 = dict(fd, tensors=dict(fd["tensors"], col_idx=_t(ci)))
    with pytest.raises(mss.MssError) as e:
        g.recover(fd3, _t(f.r2), _t(np.zeros(f.n_cells * f.n1)))
    assert e.value.status == mss.ERR_INVALID_ARG
    # the handle still works
    a, b = g.condense(fd, _t(f.r1), _t(f.r2))
    assert torch.isfinite(a).all()
