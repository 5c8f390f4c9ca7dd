"""Batched solves (mss_batch_*): worker lanes with their own handles and
streams, largest-first schedule, autotuned threads per CTA and driver.

Every system in a batch must come out exactly as a single handle solves it
alone (the batch changes only where and when the kernels run): same
iteration count, same solution bits, for any lane count, with or without
the autotuner, on a first run (tuning) and a second run (cached choices).
One failing system must not disturb the others.
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


def _systems(seed=0, count=10):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(rng.integers(8, 41))
        ny = int(rng.integers(8, 41))
        nb = int(rng.choice([4, 6]))
        pe = float(10.0 ** rng.uniform(-1, 3))
        out.append(sy.make_system(nx, ny, nb, pe=pe, sigma=2.0, band=True, seed=100 + k))
    return out


def _dev(s):
    return dict(row_ptr=torch.from_numpy(s.row_ptr).cuda(),
                col_idx=torch.from_numpy(s.col_idx).cuda(),
                vals=torch.from_numpy(np.ascontiguousarray(s.vals).reshape(-1)).cuda(),
                b=torch.from_numpy(s.b).cuda(), nb=s.nb, p_idx=s.p_idx, t_idx=s.t_idx)


def _alone(mss, s, **kw):
    g = mss.Solver().setup_system(s, **kw)
    return g.solve(torch.from_numpy(s.b).cuda(), tol=1e-8, maxit=500)


@pytest.mark.parametrize("lanes,autotune,precision", [(4, True, "fp64"), (1, False, "fp64"),
                                                      (3, True, "mixed")])
def test_batch_equals_single_handle(mss, lanes, autotune, precision):
    systems = _systems(seed=lanes)
    dev = [_dev(s) for s in systems]
    ref = [_alone(mss, s, precision=precision, amg_max_coarse=50) for s in systems]
    B = mss.Batch(lanes=lanes, autotune=autotune)
    for rnd in range(2):
        xs, res, inf = B.solve(dev, tol=1e-8, maxit=500, precision=precision, amg_max_coarse=50)
        for i, (x, r) in enumerate(zip(xs, res)):
            xr, ir = ref[i]
            assert r["status"] == 0, (i, r)
            assert r["iters"] == ir["iters"], (i, r["iters"], ir["iters"])
            assert torch.equal(x, xr), i
        for f in inf:
            assert f["threads"] in (64, 128, 256, 512) and f["driver"] in (0, 1)
            assert 0 <= f["lane"] < lanes and f["latency_ms"] > 0
            assert f["finish_ms"] >= f["latency_ms"] - 1e-6
    tuned = B.tuned()
    if autotune:
        keys = {(f["bucket"], s.nb) for f, s in zip(inf, systems)}
        assert {(t[0], t[1]) for t in tuned} == keys
        # second round: every system ran with its bucket's cached choice
        choice = {(t[0], t[1]): (t[2], t[3]) for t in tuned}
        for f, s in zip(inf, systems):
            assert (f["threads"], f["driver"]) == choice[(f["bucket"], s.nb)]
    else:
        assert tuned == []
        assert all(f["threads"] == 256 and f["driver"] == 0 for f in inf)


def test_batch_isolates_a_failing_system(mss):
    systems = _systems(seed=7, count=5)
    bad = systems[2]
    vals = bad.vals.copy()
    vals[:] = 0.0
    systems[2] = sy.BlockSystem(bad.row_ptr, bad.col_idx, vals, bad.b, bad.nx, bad.ny, bad.nb)
    dev = [_dev(s) for s in systems]
    B = mss.Batch(lanes=2)
    xs, res, inf = B.solve(dev, tol=1e-8, maxit=500)
    assert res[2]["status"] == mss.ERR_SINGULAR_BLOCK
    for i in (0, 1, 3, 4):
        xr, ir = _alone(mss, systems[i])
        assert res[i]["status"] == 0 and torch.equal(xs[i], xr)


def test_batch_arguments_checked(mss):
    with pytest.raises(mss.MssError):
        mss.Batch(lanes=0)
    B = mss.Batch(lanes=2)
    xs, res, inf = B.solve([], tol=1e-8, maxit=10)
    assert xs == [] and res == []
