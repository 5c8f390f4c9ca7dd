"""The CUDA path at the benchmark size (1024 x 1024 cells, nb = 6, FGMRES(50)
to 1e-6, Pe in {0.1, 10, 1000}) in the launch configuration bench.py times.

The oracle cannot rerun these systems inside a test, so the checks are:
* converged iteration counts equal to the oracle's within +-1; the oracle's
  counts are stored in tests/golden/bench_oracle_iterations_1024.json, written
  by tests/golden/make_bench_iterations.py, which calls only the oracle;
* the reported true residual is what an independent FP64 evaluation on the
  host gives (scipy BSR product of the unscaled matrix, scaled by the
  library's N^-1 row by row on sampled cells);
* y = Abar x at full size equals N^-1 (A x) with A x from scipy (the scaling is
  linear per cell row; the scaled blocks are compared bit for bit at small
  sizes in test_gpu_parity.py).
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
