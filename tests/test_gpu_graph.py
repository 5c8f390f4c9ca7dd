"""The device-driven FGMRES (the whole restarted solve as one CUDA graph with
nested while-loop conditional nodes) against the host-driven loop.

Both drivers run the same kernels in the same order, so every output must be
identical bit for bit: the solution, the iteration and restart counts, both
residual estimates and the status, for every scheme, orthogonalisation,
precision, restart length and stopping reason (tolerance, maxit, zero or
non-finite right-hand side). The host-driven loop is itself held to the oracle
in test_gpu_parity.py.
"""
import numpy as np
import pytest

from paper_1912_04385_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
]


def _sys(c):
    c = dict(c)
    return sy.make_system(c.pop("nx"), c.pop("ny"), c.pop("nb"), **c)


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def _pair(mss, s, **kw):
    return (mss.Solver().setup_system(s, driver="host", **kw),
            mss.Solver().setup_system(s, driver="graph", **kw))


def _same(mss, gh, gg, b, tol, maxit):
    l0 = mss.load().mss_kernel_launches(1)
    xh, ih = gh.solve(b, tol=tol, maxit=maxit)
    lh = mss.load().mss_kernel_launches(1)
    xg, ig = gg.solve(b, tol=tol, maxit=maxit)
    lg = mss.load().mss_kernel_launches(1)
    del l0
    for k in ("iters", "restarts", "status", "rel_res_implicit", "rel_res_true"):
        assert ih[k] == ig[k], (k, ih[k], ig[k])
    assert torch.equal(xh, xg)
    # the graph's replayed launches are counted like the host loop's; the host
    # loop runs each V-cycle's coarse levels as one fused launch, the graph
    # keeps the per-level kernels, so it counts at least as many
    assert 0 < lh <= lg, (lh, lg)
    return ih


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("scheme,orthog,precision,restart", [
    ("cptr3", 0, "fp64", 30), ("cptr3", 1, "fp64", 30), ("cptr3", 0, "mixed", 30),
    ("cptr3", 0, "fp64", 4), ("cpr", 0, "fp64", 30), ("ilu0", 0, "fp64", 30)])
def test_graph_equals_host_loop(mss, case, scheme, orthog, precision, restart):
    s = _sys(CASES[case])
    gh, gg = _pair(mss, s, scheme=scheme, orthog=orthog, precision=precision, restart=restart,
                   amg_max_coarse=40)
    b = _t(s.b)
    info = _same(mss, gh, gg, b, 1e-8, 400)
    assert info["status"] == 0
    if restart == 4:
        assert info["restarts"] >= 2
    # the same graph again, another right-hand side, a maxit stop
    b2 = _t(np.random.default_rng(case).standard_normal(s.b.size))
    info = _same(mss, gh, gg, b2, 1e-14, 7)
    assert info["status"] == mss.ERR_NOT_CONVERGED and info["iters"] == 7


def test_graph_edge_cases(mss):
    s = _sys(CASES[1])
    gh, gg = _pair(mss, s, restart=10)
    b = _t(s.b)
    # maxit = 0: one empty cycle, x = 0
    info = _same(mss, gh, gg, b, 1e-8, 0)
    assert info["iters"] == 0 and info["status"] == mss.ERR_NOT_CONVERGED
    # zero right-hand side: x = 0 at once
    z = torch.zeros_like(b)
    x, info = gg.solve(z, tol=1e-8, maxit=50)
    assert info["status"] == 0 and info["iters"] == 0 and not torch.any(x)
    # tol = 0 runs exactly maxit steps across restarts
    info = _same(mss, gh, gg, b, 0.0, 25)
    assert info["iters"] == 25 and info["restarts"] == 2
    # a non-finite right-hand side is an error on both drivers
    nb = s.b.copy()
    nb[3] = np.inf
    for g in (gh, gg):
        with pytest.raises(mss.MssError) as e:
            g.solve(_t(nb), tol=1e-8, maxit=10)
        assert e.value.status == mss.ERR_BREAKDOWN
    # the graph handle still solves afterwards
    _same(mss, gh, gg, b, 1e-8, 200)


def test_graph_rebuilt_after_new_setup(mss):
    s1 = _sys(CASES[0])
    s2 = _sys(CASES[2])
    gg = mss.Solver().setup_system(s1, driver="graph")
    x1, i1 = gg.solve(_t(s1.b), tol=1e-8, maxit=200)
    gg.setup_system(s2, driver="graph")
    x2, i2 = gg.solve(_t(s2.b), tol=1e-8, maxit=200)
    gh = mss.Solver().setup_system(s2, driver="host")
    xh, ih = gh.solve(_t(s2.b), tol=1e-8, maxit=200)
    assert i2["iters"] == ih["iters"] and torch.equal(x2, xh)
    assert i1["status"] == 0 and i2["status"] == 0


def test_driver_option_checked(mss):
    s = _sys(CASES[0])
    with pytest.raises(mss.MssError) as e:
        mss.Solver().setup_system(s, driver=5)
    assert e.value.status == mss.ERR_INVALID_ARG


def test_pool_allocator_handle_and_repeated_setup(mss):
    # a handle without allocation hooks takes its memory from the library's
    # stream-ordered device pool; the set-up's worker streams always do.
    # Repeated set-ups (worker streams reused, hierarchies freed on them)
    # give the same bits.
    s = _sys(CASES[1])
    gt = mss.Solver().setup_system(s, driver="graph")
    xt, it = gt.solve(_t(s.b), tol=1e-8, maxit=300)
    gp = mss.Solver(torch_allocator=False)
    for _ in range(3):
        gp.setup_system(s, driver="graph")
        xp, ip = gp.solve(_t(s.b), tol=1e-8, maxit=300)
        assert ip["iters"] == it["iters"] and torch.equal(xp, xt)
    gp.setup_system(_sys(CASES[2]), scheme="cpr")
    x2, i2 = gp.solve(_t(_sys(CASES[2]).b), tol=1e-8, maxit=300)
    assert i2["status"] == 0


def test_grid_barrier_wait_runs_out(mss):
    # a barrier wait that nothing completes gives up at its limit, the kernel
    # returns with the error flag set, and the context stays usable
    s = _sys(CASES[0])
    g = mss.Solver().setup_system(s, amg_max_coarse=40)
    assert g.probe_wait_limit()
    x, info = g.solve(torch.from_numpy(s.b).cuda(), tol=1e-8, maxit=300)
    assert info["status"] == 0
