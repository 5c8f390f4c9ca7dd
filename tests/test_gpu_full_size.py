"""The CUDA path at the benchmark size (1024 x 1024 cells, nb = 6, FGMRES(50)
to 1e-6, Pe in {0.1, 10, 1000}) in the launch configuration bench.py times.

* Element by element against the oracle on the Pe = 10 system (the oracle's
  set-up takes a few seconds at this size, one application well under one):
  the scaled matrix, both AMG hierarchies and the strip ordering bit for bit;
  the block ILU(0) factors -- here the large colours run the kernel with nb
  lanes per strip -- within the factor tolerance of the small parity cases;
  the last stage and the whole preconditioner within 1e-12.
* Converged iteration counts equal to the oracle's within +-1; the oracle's
  counts are stored in tests/golden/bench_oracle_iterations_1024.json, written
  by tests/golden/make_bench_iterations.py, which calls only the oracle (a
  full solve with the oracle takes tens of seconds per system).
* The reported true residual is what an independent FP64 evaluation on the
  host gives (scipy BSR product of the unscaled matrix, scaled by the
  library's N^-1), and y = Abar x equals N^-1 (A x).
"""
import json
from pathlib import Path

import numpy as np
import pytest

from paper_1912_04385_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sps = pytest.importorskip("scipy.sparse")

GOLDEN = Path(__file__).with_name("golden") / "bench_oracle_iterations_1024.json"


@pytest.fixture(scope="module")
def mss():
    from paper_1912_04385_gb300 import build, mss as m
    build.build()
    m.load()
    return m


APPLY_TOL = 1e-12
FACTOR_TOL = 1e-12


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / max(float(np.max(np.abs(b))), 1e-300))


def test_full_size_elementwise_parity(mss):
    import oracle
    from tests.helpers import stored_factor_form
    gold = json.loads(GOLDEN.read_text())
    s = sy.plain_at_scale(gold["grid"], pe=gold["systems"][1]["pe"], seed=0)
    rp = torch.from_numpy(s.row_ptr).cuda()
    ci = torch.from_numpy(s.col_idx).cuda()
    v = torch.from_numpy(s.vals.reshape(-1)).cuda()
    g = mss.Solver().setup(rp, ci, v, 6, 0, 1, restart=gold["restart"], driver="graph")
    o = oracle.OracleSolver.from_system(s, restart=gold["restart"])
    # scaling (Eqs. CPTR31/CPTR32)
    ab_o, _ = o.scaled()
    assert np.array_equal(g.scaled().cpu().numpy(), ab_o)
    del ab_o
    assert np.array_equal(g.scale_rhs(torch.from_numpy(s.b).cuda()).cpu().numpy(),
                          o.scale_rhs(s.b))
    # both hierarchies
    for which in (0, 1):
        lg, lo = g.amg_levels(which), o.amg_levels(which)
        assert len(lg) == len(lo) >= 3
        for a, b in zip(lg, lo):
            for k in range(3):
                assert np.array_equal(a["A"][k].cpu().numpy(), b.A[k]), (which, k)
            if b.cf is not None:
                assert np.array_equal(a["cf"].cpu().numpy(), b.cf)
                for k in range(3):
                    assert np.array_equal(a["P"][k].cpu().numpy(), b.P[k])
    # strip ordering
    f = o.bilu()
    nc, colour, perm = g.bilu_ordering()
    assert nc == f["ncolours"]
    assert np.array_equal(colour.cpu().numpy(), f["colour"])
    assert np.array_equal(perm.cpu().numpy(), f["perm"])
    # the large colours are above the size at which the library switches to
    # nb lanes per strip (4 x (32 // nb) strips per SM)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    strips = np.bincount(f["colour"][::32])
    assert strips.max() >= 4 * (32 // 6) * sms
    # factors: auto (both forms, by colour size) and forced warp form, same bits
    fv, fd = g.bilu_factors()
    efv, edinv = stored_factor_form(f, 32)
    del f
    assert _rel(fv.cpu().numpy(), efv) < FACTOR_TOL
    assert _rel(fd.cpu().numpy(), edinv) < FACTOR_TOL
    del efv, edinv
    gw = mss.Solver().setup(rp, ci, v, 6, 0, 1, restart=gold["restart"], factor_form="warp")
    fw, dw = gw.bilu_factors()
    assert torch.equal(fw, fv) and torch.equal(dw, fd)
    del gw, fw, dw, fv, fd
    # last stage and the whole preconditioner (Algorithm 2)
    r = np.random.default_rng(5).standard_normal(s.n_cells * 6)
    rt = torch.from_numpy(r).cuda()
    assert _rel(g.stage(2, rt).cpu().numpy(), o.stage(2, r)) < APPLY_TOL
    assert _rel(g.apply(rt).cpu().numpy(), o.apply(r)) < APPLY_TOL


def _bsr(s):
    n = s.n_cells
    v = np.asarray(s.vals, np.float64).reshape(-1, s.nb, s.nb)
    return sps.bsr_matrix((v, s.col_idx, s.row_ptr), shape=(n * s.nb, n * s.nb))


@pytest.mark.parametrize("k", range(3))
def test_full_size_iterations_and_residual(mss, k):
    gold = json.loads(GOLDEN.read_text())
    rec = gold["systems"][k]
    s = sy.plain_at_scale(gold["grid"], pe=rec["pe"], seed=0)
    rp = torch.from_numpy(s.row_ptr).cuda()
    ci = torch.from_numpy(s.col_idx).cuda()
    v = torch.from_numpy(s.vals.reshape(-1)).cuda()
    b = torch.from_numpy(s.b).cuda()
    g = mss.Solver().setup(rp, ci, v, 6, 0, 1, restart=gold["restart"])
    x, info = g.solve(b, tol=gold["tol"], maxit=1000)
    assert info["status"] == 0
    assert abs(info["iters"] - rec["iters"]) <= 1, (info["iters"], rec["iters"])
    assert info["rel_res_true"] <= gold["tol"]
    A = _bsr(s)
    xh = x.cpu().numpy()
    Ax = A @ xh
    # scaled residual ||N^-1 (b - A x)|| / ||N^-1 b|| through the library's N^-1
    rs = g.scale_rhs(torch.from_numpy(s.b - Ax).cuda()).cpu().numpy()
    bs = g.scale_rhs(b).cpu().numpy()
    rel = np.linalg.norm(rs) / np.linalg.norm(bs)
    assert abs(rel - info["rel_res_true"]) <= 1e-6 * info["rel_res_true"] + 1e-14
    # the operator FGMRES iterates with
    y = g.spmv(x).cpu().numpy()
    ref = g.scale_rhs(torch.from_numpy(Ax).cuda()).cpu().numpy()
    assert np.max(np.abs(y - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_full_size_graph_driver_equals_host_loop(mss):
    # the launch configuration bench.py times: the whole solve as one graph
    gold = json.loads(GOLDEN.read_text())
    rec = gold["systems"][1]
    s = sy.plain_at_scale(gold["grid"], pe=rec["pe"], seed=0)
    rp = torch.from_numpy(s.row_ptr).cuda()
    ci = torch.from_numpy(s.col_idx).cuda()
    v = torch.from_numpy(s.vals.reshape(-1)).cuda()
    b = torch.from_numpy(s.b).cuda()
    gh = mss.Solver().setup(rp, ci, v, 6, 0, 1, restart=gold["restart"])
    xh, ih = gh.solve(b, tol=gold["tol"], maxit=1000)
    del gh
    gg = mss.Solver().setup(rp, ci, v, 6, 0, 1, restart=gold["restart"], driver="graph")
    xg, ig = gg.solve(b, tol=gold["tol"], maxit=1000)
    assert ig["iters"] == ih["iters"] and abs(ig["iters"] - rec["iters"]) <= 1
    assert torch.equal(xg, xh)


def test_mixed_precision_workload_2048(mss):
    # 2048 x 2048 (25 M unknowns), sigma 3, Pe 10: the mixed form reaches the
    # FP64 tolerance on the scaled system within two iterations of FP64
    s = sy.plain_at_scale(2048, pe=10.0, seed=0, sigma=3.0)
    rp = torch.from_numpy(s.row_ptr).cuda()
    ci = torch.from_numpy(s.col_idx).cuda()
    v = torch.from_numpy(s.vals.reshape(-1)).cuda()
    b = torch.from_numpy(s.b).cuda()
    del s
    g = mss.Solver()
    g.setup(rp, ci, v, 6, 0, 1, restart=50, driver="graph")
    x64, i64 = g.solve(b, tol=1e-6, maxit=1000)
    g.setup(rp, ci, v, 6, 0, 1, restart=50, driver="graph", precision="mixed")
    xm, im = g.solve(b, tol=1e-6, maxit=1000)
    assert i64["status"] == 0 and im["status"] == 0
    assert im["rel_res_true"] <= 1e-6
    assert im["iters"] <= i64["iters"] + 2
    rel = float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64))
    assert rel < 1e-2, rel
