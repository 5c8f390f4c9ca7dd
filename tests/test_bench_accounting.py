"""bench.py's accounting of one preconditioner application (CPU only): the
algorithmic flops and the roofline time max(bytes / HBM, flops / FP64 peak),
on a stand-in solver that reports hierarchy sizes the way the library does."""
import sys
from pathlib import Path

import pytest

torch = pytest.importorskip("torch")
ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))
import bench  # noqa: E402


class _Levels:
    """amg_levels(which) -> [{"A": (rp, ci, v), "P": (rp, ci, v)}, ...]."""

    def __init__(self, sizes):
        self.sizes = sizes          # per hierarchy: [(n, nnz, nnzp), ..., (n_coarse, nnz, 0)]

    def amg_levels(self, which):
        out = []
        for n, nnz, nnzp in self.sizes[which]:
            out.append({"A": (torch.zeros(n + 1), torch.zeros(nnz), torch.zeros(nnz)),
                        "P": (torch.zeros(n + 1), torch.zeros(nnzp), torch.zeros(nnzp))})
        return out


class _Opts:
    nu_pre = 2
    nu_post = 2


def test_apply_flops_hand_count():
    N, nnzb, nb = 64, 64 * 5 - 2 * 8 - 2 * 8, 6
    fake = _Levels({0: [(64, 288, 100), (20, 90, 0)], 1: [(64, 300, 110), (16, 70, 0)]})
    got = bench.apply_alg_flops(N, nnzb, nb, fake, _Opts())
    # level 0: 4 A passes of 2 flops per entry plus 3 per row, P and R 2 per entry;
    # coarsest: dense GEMV
    amg = (4 * (2 * 288 + 3 * 64) + 4 * 100 + 2 * 20 * 20) \
        + (4 * (2 * 300 + 3 * 64) + 4 * 110 + 2 * 16 * 16)
    alg = bench.algorithmic(N, nnzb, nb)
    assert got == amg + 2 * nnzb + alg["bilu_fwd"]["flops"] + alg["bilu_bwd"]["flops"]
    # the sweep count enters linearly
    class One(_Opts):
        nu_pre = 1
        nu_post = 1
    assert bench.apply_alg_flops(N, nnzb, nb, fake, One()) < got


def test_precond_roofline_takes_the_slower_bound():
    # 6.8 TB at 6800 GB/s is 1000 ms; 0.5 PFLOP at 1 TFLOP/s is 500000 ms (500 s)
    r = bench.precond_roofline(bytes_apply=6.8e12, flops_apply=0.5e15, apply_ms=2000.0,
                               hbm_gbs=6800.0, fp64_tflops=1.0)
    assert r["t_hbm_ms"] == pytest.approx(1000.0) and r["t_fp64_ms"] == pytest.approx(500000.0)
    assert r["bound"] == "alu" and r["t_roofline_ms"] == pytest.approx(500000.0)
    r = bench.precond_roofline(bytes_apply=6.8e12, flops_apply=0.5e12, apply_ms=2000.0,
                               hbm_gbs=6800.0, fp64_tflops=1.0)
    assert r["t_fp64_ms"] == pytest.approx(500.0)
    assert r["bound"] == "hbm" and r["t_roofline_ms"] == pytest.approx(1000.0)
    assert r["frac"] == pytest.approx(0.5)
    r = bench.precond_roofline(bytes_apply=3.85e9, flops_apply=0.8e9, apply_ms=1.6,
                               hbm_gbs=6794.5)
    assert r["bound"] == "alu"
    assert r["t_roofline_ms"] == pytest.approx(0.8e9 / (bench.FP64_PEAK_TFLOPS * 1e12) * 1e3,
                                               rel=1e-3)
    assert 0 < r["frac"] < 1
    assert bench.precond_roofline(1.0, 1.0, 0.0, 6800.0)["frac"] is None
