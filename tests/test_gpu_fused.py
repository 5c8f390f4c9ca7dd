"""The fused batch schedule: the systems of each block size solved in lock
step through multi-system launches (tiles of each system's own launch shape,
resident CTAs taking tile after tile), the whole group solve in one CUDA
graph.

Each system must come out exactly as a single handle solves it alone: same
iteration count and restart count, same status, same solution bits. That
holds for every scheme the fused schedule takes (CPTR3, CPR, ILU0), for the
graph and the host-driven group loop, with restarts, iteration limits, zero
right-hand sides, and with systems of block sizes the fused schedule does not
take mixed in (those run on the lanes). Tile shapes (autotuned or fixed) do
not change a bit.
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


def _systems(seed=0, count=9, nbs=(4, 6)):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(rng.integers(6, 45))
        ny = int(rng.integers(6, 45))
        nb = int(rng.choice(nbs))
        pe = float(10.0 ** rng.uniform(-1, 3))
        out.append(sy.make_system(nx, ny, nb, pe=pe, sigma=2.0, band=True, seed=300 + k))
    return out


def _dev(s, zero_rhs=False):
    b = torch.from_numpy(s.b).cuda()
    if zero_rhs:
        b = torch.zeros_like(b)
    return dict(row_ptr=torch.from_numpy(s.row_ptr).cuda(),
                col_idx=torch.from_numpy(s.col_idx).cuda(),
                vals=torch.from_numpy(np.ascontiguousarray(s.vals).reshape(-1)).cuda(),
                b=b, nb=s.nb, p_idx=s.p_idx, t_idx=s.t_idx)


def _alone(mss, s, b, tol, maxit, **kw):
    g = mss.Solver().setup_system(s, **kw)
    return g.solve(b, tol=tol, maxit=maxit)


def _check(mss, systems, dev, tol, maxit, opts, fused_nbs=(2, 3, 4, 5, 6, 7, 8), **kw):
    ref = [_alone(mss, s, d["b"], tol, maxit, **opts) for s, d in zip(systems, dev)]
    B = mss.Batch(lanes=3, schedule="fused", **kw)
    for rnd in range(2):
        xs, res, inf = B.solve(dev, tol=tol, maxit=maxit, **opts)
        for i, (x, r, f) in enumerate(zip(xs, res, inf)):
            xr, ir = ref[i]
            assert r["status"] == ir["status"], (i, r, ir)
            assert r["iters"] == ir["iters"], (i, r["iters"], ir["iters"])
            assert r["restarts"] == ir["restarts"], i
            assert r["rel_res_true"] == ir["rel_res_true"], i
            assert torch.equal(x, xr), i
            fused = systems[i].nb in fused_nbs
            assert f["schedule"] == (1 if fused else 0), (i, f)
            if fused:
                assert f["group"] >= 0 and f["tile_blocks"] >= 1 and f["per_sm"] >= 1
            else:
                assert f["group"] == -1
    return inf


@pytest.mark.parametrize("scheme", ["cptr3", "cpr", "ilu0"])
def test_fused_equals_single_handle(mss, scheme):
    systems = _systems(seed=1)
    dev = [_dev(s) for s in systems]
    _check(mss, systems, dev, 1e-8, 500, dict(scheme=scheme, amg_max_coarse=40))


@pytest.mark.parametrize("driver", ["graph", "host"])
def test_fused_restarts_limits_and_zero_rhs(mss, driver):
    # restart 6: several cycles per system, different counts per system;
    # maxit 40: some systems stop unconverged; one right-hand side is zero
    systems = _systems(seed=2, count=7)
    dev = [_dev(s, zero_rhs=(k == 3)) for k, s in enumerate(systems)]
    opts = dict(restart=6, driver=driver, amg_max_coarse=30)
    _check(mss, systems, dev, 1e-10, 40, opts)


def test_fused_other_block_sizes_take_the_lanes(mss):
    systems = _systems(seed=3, count=6, nbs=(4, 6, 10))
    assert any(s.nb == 10 for s in systems)
    dev = [_dev(s) for s in systems]
    _check(mss, systems, dev, 1e-8, 500, dict(amg_max_coarse=40))


def test_fused_tile_shape_changes_no_bit(mss):
    systems = _systems(seed=4, count=5)
    dev = [_dev(s) for s in systems]
    inf = _check(mss, systems, dev, 1e-8, 500, dict(orthog=1), autotune=False)
    assert all(f["tile_blocks"] == 1 and f["per_sm"] == 4 for f in inf)


def test_fused_unsupported_options_use_the_lanes(mss):
    systems = _systems(seed=5, count=4)
    dev = [_dev(s) for s in systems]
    _check(mss, systems, dev, 1e-8, 500, dict(smoother="chebyshev"), fused_nbs=())


def test_fused_degenerate_systems(mss):
    # a single cell, a few cells (the coarsest level is level 0: the V-cycle
    # is the dense coarse solve), and ordinary systems in one group
    shapes = [(1, 1), (2, 3), (5, 4), (24, 17), (31, 30)]
    systems = [sy.make_system(nx, ny, 4, pe=10.0, sigma=1.0, band=True, seed=400 + k)
               for k, (nx, ny) in enumerate(shapes)]
    dev = [_dev(s) for s in systems]
    _check(mss, systems, dev, 1e-9, 300, dict(amg_max_coarse=20))
