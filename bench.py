#!/usr/bin/env python3
"""Benchmark: time to a 1e-6 relative residual on a 1M-cell system.

Workload: 1024 x 1024 grid, nb = 6 (P, T, 4 components), lognormal
permeability (sigma 2, correlation length 16 cells), stiff reaction band,
seed 0, one system per Peclet number in {0.1, 10, 1000}; CPTR3 preconditioned
FGMRES(50) to a relative residual of 1e-6. One step = mss_setup +
mss_fgmres_solve for each of the three systems, inputs resident in HBM
(1.5 GB of blocks per system, far above the 129 MB L2). value = mean ms per
system.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun (N > 1) every rank solves its
own replica of the workload (no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time
from pathlib import Path

# More hardware work queues than CUDA's default of 8: the batch legs run many
# streams at once (lanes, their set-up workers, the fused groups), and streams
# that share a queue wait on each other's work. Read when CUDA starts, so set
# before torch touches the device.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

PES = (0.1, 10.0, 1000.0)
METRIC = "time-to-1e-6 rel. residual (ms) at 1M cells; FGMRES iters; precond HBM GB/s"
DATA = "synthetic (seeded 5-point thermal-compositional generator; no dataset)"
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12   # 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", "--n", dest="n", type=int, default=1024,
                    help="grid side of the benchmark systems (--n is an alias)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--restart", type=int, default=50)
    ap.add_argument("--maxit", type=int, default=1000)
    ap.add_argument("--driver", default="graph", choices=["host", "graph"],
                    help="FGMRES driver: host loop, or the whole solve as one CUDA graph")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="preconditioner precision of the main leg (the bench line is fp64)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--mixed-n", type=int, default=2048,
                    help="grid of the mixed-precision comparison (0: skip)")
    ap.add_argument("--batch", type=int, default=64,
                    help="systems in the batched-solve comparison (0: skip)")
    ap.add_argument("--batch-lanes", type=int, default=8)
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-condense", action="store_true",
                    help="skip the static-condensation leg")
    ap.add_argument("--no-schemes", action="store_true",
                    help="skip the CPTR and CPR legs")
    ap.add_argument("--no-newton", action="store_true",
                    help="skip the Newton-loop reuse leg")
    ap.add_argument("--no-smoothers", action="store_true",
                    help="skip the multicolour Gauss-Seidel legs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    return ap.parse_args()


def leg_steps(a, cap):
    """Timed steps of an auxiliary leg: the run's step count, at most cap (the
    headline keeps the run's count; the legs around it must not multiply the
    run's length)."""
    return max(1, min(a.steps, cap))


def workload_config(a):
    return {"workload": f"cptr3-fgmres{a.restart}-{a.n}x{a.n}-nb6", "grid": [a.n, a.n], "nb": 6,
            "cells": a.n * a.n, "pe": list(PES), "sigma": 2.0, "corr_len": 16, "band": True,
            "seed": 0, "tol": a.tol, "scheme": "CPTR3 (T AMG, P AMG, strip-coloured BILU0, strips of 32)",
            "restart": a.restart, "driver": a.driver,
            "l2": "inputs 1.5 GB per system >> 129 MB L2 (no flush needed)"}


def systems(a):
    from paper_1912_04385_gb300 import synthetic as sy
    return [sy.plain_at_scale(a.n, pe=pe, seed=0) for pe in PES]


# ---- clocks -----------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, enabled, device):
        self.p = None
        self.device = device
        self.path = Path(tempfile.gettempdir()) / f"mss_bench_clocks_rank{device}.csv"
        if not enabled:
            return
        try:
            self.path.parent.mkdir(exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={device}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in self.path.read_text().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in load for k, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": float(np.median([r[0] for r in load])),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "samples_under_load": len(load)}


# ---- algorithmic bytes / flops of the traced kernels --------------------------
def algorithmic(N, nnzb, nb):
    """Per-call algorithmic bytes and flops (FP64 values, int32 indices)."""
    nl = (nnzb - N) // 2          # strictly lower (= upper) blocks, symmetric pattern
    B = nb * nb * 8
    vec = N * nb * 8
    spmv = dict(bytes=nnzb * (B + 4) + (N + 1) * 4 + 2 * vec, flops=2 * nnzb * nb * nb)
    # forward: L blocks, column slices [t|p], indices, r, w (write), x_T, v_P
    fwd = dict(bytes=nl * (B + 4) + nnzb * (2 * nb * 8 + 4) + 3 * N * 4 + 2 * vec + 2 * N * 8,
               flops=2 * (nl * nb * nb + nnzb * 2 * nb))
    # backward: U blocks, diagonal inverses, indices, w (read + write), y, x_T, v_P
    bwd = dict(bytes=nl * (B + 4) + N * B + 3 * N * 4 + 3 * vec + 2 * N * 8,
               flops=2 * (nl * nb * nb + N * nb * nb))
    return {"spmv": spmv, "bilu_fwd": fwd, "bilu_bwd": bwd}


def load_traffic(kernel):
    """DRAM bytes per full-size launch of `kernel` from the committed ncu
    summary, or None if the kernel's source files changed since the capture."""
    import hashlib
    path = ROOT / "profiles" / "dram_traffic.json"
    if not path.exists():
        return None
    try:
        rec = json.loads(path.read_text()).get(kernel)
        if not rec:
            return None
        h = hashlib.sha256()
        for f in rec["source_files"]:
            h.update(f.encode())
            h.update((ROOT / f).read_bytes())
        if h.hexdigest() == rec["source_digest"]:
            return rec["bytes_per_launch_full_size"]
    except Exception:
        return None
    return None


# ---- rank aggregation (replicas: no data-path collective) ------------------------
def max_over_ranks(value, dist):
    """The slowest rank's time (all ranks get it); the identity with one rank."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_system_ms(ms, systems_per_rank, world):
    """Whole-job time per system: every rank solved systems_per_rank systems
    in (at most) ms, so the job did systems_per_rank * world systems."""
    return ms / (systems_per_rank * world)


# ---- our arm --------------------------------------------------------------------
def run_ours(a, rank, world, dist):
    import torch
    from __graft_entry__ import build
    from paper_1912_04385_gb300 import mss

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build()
    lib = mss.load()
    sysl = systems(a)
    dev = []
    for s in sysl:
        dev.append((torch.from_numpy(s.row_ptr).cuda(), torch.from_numpy(s.col_idx).cuda(),
                    torch.from_numpy(s.vals.reshape(-1)).cuda(), torch.from_numpy(s.b).cuda()))
    torch.cuda.synchronize()
    solver = mss.Solver()
    opts = mss.options(restart=a.restart, driver=a.driver, precision=a.precision)
    stream = torch.cuda.current_stream()

    def step(trace=False, info_out=None, o=None):
        for k, (rp, ci, v, b) in enumerate(dev):
            solver.setup(rp, ci, v, 6, 0, 1, opts=opts if o is None else o)
            x, info = solver.solve(b, tol=a.tol, maxit=a.maxit)
            if info["status"] != 0:
                raise RuntimeError(f"solve failed for Pe={PES[k]}: {info}")
            if info_out is not None:
                info_out.append(info)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(a.warmup):
        step()
    barrier()
    clocks = Clocks(not a.no_clocks, int(os.environ.get("LOCAL_RANK", "0")))
    solver.trace(True)
    solver.trace_read(reset=True)
    lib.mss_kernel_launches(1)
    infos = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(a.steps):
        step(info_out=infos)
    e1.record(stream)
    barrier()
    wall_ms = (time.perf_counter() - t0) * 1e3
    launches = int(lib.mss_kernel_launches(1))
    tr = solver.trace_read(reset=True)
    clk = clocks.stop()
    trace_from = "the timed steps"
    if a.driver == "graph":
        # a solve graph holds no events: kernel-class times come from one
        # host-driven step after the timed region (same kernels, same order)
        step(o=mss.options(restart=a.restart, driver="host", precision=a.precision))
        torch.cuda.synchronize()
        tr = solver.trace_read(reset=True)
        trace_from = "one host-driven step after the timed region"
    solver.trace(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    nsys = a.steps * len(PES)
    value = per_system_ms(ms, nsys, world)
    iters = [i["iters"] for i in infos[:len(PES)]]

    # roofline of the dominant single-kernel class (traced live above)
    s0 = sysl[0]
    N, nnzb = s0.n_cells, s0.nnzb
    alg = algorithmic(N, nnzb, 6)
    ncol = solver.bilu_ordering()[0]
    # the dominant single kernel of the solve: the FGMRES matrix-vector product
    # (the last-stage sweep classes span two kernels each; see trace_ms)
    top = "spmv"
    nl, tot = tr[top]
    calls = nl if top == "spmv" else nl / ncol        # sweeps: ncol launches per call
    per_call_ms = tot / max(calls, 1)
    per_launch_ms = tot / max(nl, 1)
    flops = alg[top]["flops"] / (per_call_ms * 1e-3) / 1e12
    gbs = alg[top]["bytes"] / (per_call_ms * 1e-3) / 1e9
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) \
        if (ROOT / "MEASURED_PEAKS.json").exists() else {"hbm_gbs": 6800.0}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    kname = {"spmv": "k_bsr_spmv", "bilu_fwd": "k_bilu_fwd", "bilu_bwd": "k_bilu_bwd"}[top]
    roofline = {"kernel": kname, "bound": "alu", "achieved": round(flops, 4),
                "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                "frac": round(flops / FP64_PEAK_TFLOPS, 4), "traffic": load_traffic(kname),
                "peak_source": "FP64 FMA: 2/clk/SM x 152 SMs x 2.07 GHz (probe measured 1.193 "
                               "TFLOP/s at 2.0 GHz)",
                "algorithmic_bytes_per_call": alg[top]["bytes"],
                "algorithmic_flops_per_call": alg[top]["flops"],
                "launches_per_call": 1 if top == "spmv" else ncol,
                "avg_launch_ms": round(per_launch_ms, 5), "avg_call_ms": round(per_call_ms, 5),
                "hbm_achieved_gbs": round(gbs, 1), "hbm_peak_gbs": hbm_peak,
                "hbm_frac": round(gbs / hbm_peak, 4)}
    # preconditioner apply: algorithmic bytes (apply_alg_bytes) over traced time
    n_apply, apply_ms = tr["apply"]
    out = {"metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms / a.steps, 3),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if a.precision == "fp64" else "bf16/f32 (FGMRES f64)",
           "data": DATA,
           "config": {**workload_config(a), "parallelism": f"replicas x{world}"},
           "iters": iters, "iters_mean": float(np.mean(iters)),
           "wall_ms_per_system": round(wall_ms / (nsys * world), 3),
           "setup_ms_mean": round(float(np.mean([i["setup_ms"] for i in infos])), 3),
           "solve_ms_mean": round(float(np.mean([i["solve_ms"] for i in infos])), 3),
           "apply_ms_mean": round(apply_ms / max(n_apply, 1), 4),
           "gpu_launches": launches,
           "roofline": roofline,
           "trace_ms": {k: [v[0], round(v[1], 3)] for k, v in tr.items()},
           "trace_from": trace_from,
           "clocks": clk}
    bytes_apply = apply_alg_bytes(N, nnzb, 6, solver, opts)
    out["precond_gbs"] = round(bytes_apply / (apply_ms / max(n_apply, 1) * 1e-3) / 1e9, 1)
    out["precond_alg_bytes"] = bytes_apply
    out["precond_roofline"] = precond_roofline(
        bytes_apply, apply_alg_flops(N, nnzb, 6, solver, opts), apply_ms / max(n_apply, 1),
        hbm_peak)

    # end to end through the C-ABI from pinned host buffers (right after the
    # timed region, before the other legs fill the allocators)
    if not a.no_e2e:
        out["e2e"] = e2e(a, sysl, solver, opts, torch)
    # the same workload with the mixed-precision preconditioner
    if not a.no_mixed:
        out["mixed"] = mixed_leg(a, dev, solver, torch, stream)
        if a.mixed_n > 0:
            out["mixed_config"] = mixed_config_leg(a, solver, torch, stream)
    if not a.no_condense:
        out["condense"] = condense_leg(a, torch)
    if not a.no_newton:
        out["newton"] = newton_leg(a, dev, solver, torch)
    if not a.no_smoothers:
        # the paper's smoother (symmetric Gauss-Seidel, multicolour form)
        out["mcsgs"] = variant_leg(a, dev, solver, torch, stream, smoother="mcsgs")
        out["mcsgs_v11"] = variant_leg(a, dev, solver, torch, stream, smoother="mcsgs",
                                       nu_pre=1, nu_post=1)
    if not a.no_schemes:
        # the other preconditioners of Sec. 4 on the same systems
        out["cptr"] = variant_leg(a, dev, solver, torch, stream, scheme="cptr")
        out["cpr"] = variant_leg(a, dev, solver, torch, stream, scheme="cpr")
    if a.batch > 0:
        out["batch"] = batch_leg(a, torch)
    if not a.no_learned:
        out["learned"] = learned_leg(a, dev, torch, stream)
    # CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(a, sysl)
    return out


def mixed_leg(a, dev, solver, torch, stream):
    """Mixed precision (BF16 storage, FP32 sweeps in M^-1; FP64 FGMRES) on the
    same three systems and tolerance: time per system, iterations, and the
    unscaled FP64 residual ||b - A x|| / ||b|| the solve reached."""
    from paper_1912_04385_gb300 import mss
    opts = mss.options(restart=a.restart, precision="mixed", driver=a.driver)
    host = mss.options(restart=a.restart, precision="mixed", driver="host")
    infos, rels = [], []

    def step(keep):
        for rp, ci, v, b in dev:
            solver.setup(rp, ci, v, 6, 0, 1, opts=opts)
            x, info = solver.solve(b, tol=a.tol, maxit=a.maxit)
            if info["status"] != 0:
                raise RuntimeError(f"mixed solve failed: {info}")
            if keep:
                infos.append(info)
                r, bn = solver.residual_norm(rp, ci, v, 6, b, x)
                rels.append(r / bn)

    steps = leg_steps(a, 5)
    for _ in range(max(1, min(a.warmup, 2))):
        step(False)
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for rp, ci, v, b in dev:
            solver.setup(rp, ci, v, 6, 0, 1, opts=opts)
            x, info = solver.solve(b, tol=a.tol, maxit=a.maxit)
            if info["status"] != 0:
                raise RuntimeError(f"mixed solve failed: {info}")
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    step(True)
    # kernel-class trace from one host-driven pass (a graph records no events)
    solver.trace(True)
    solver.trace_read(reset=True)
    for rp, ci, v, b in dev:
        solver.setup(rp, ci, v, 6, 0, 1, opts=host)
        solver.solve(b, tol=a.tol, maxit=a.maxit)
    torch.cuda.synchronize()
    tr = solver.trace_read(reset=True)
    solver.trace(False)
    n_apply, apply_ms = tr["apply"]
    return {"ms_per_system": round(ms / (steps * len(dev)), 3), "steps": steps,
            "iters": [i["iters"] for i in infos],
            "setup_ms_mean": round(float(np.mean([i["setup_ms"] for i in infos])), 3),
            "solve_ms_mean": round(float(np.mean([i["solve_ms"] for i in infos])), 3),
            "apply_ms_mean": round(apply_ms / max(n_apply, 1), 4),
            "rel_res_unscaled": [float(f"{v:.3e}") for v in rels],
            "trace_ms": {k: [v[0], round(v[1], 3)] for k, v in tr.items()},
            "storage": "bf16 blocks, fp32 vectors and sweeps, fp64 Krylov",
            "driver": a.driver}


def variant_leg(a, dev, solver, torch, stream, **kw):
    """The benchmark systems with other options (FP64): ms per system (CUDA
    events around set-up + solve), iterations, and the kernel-class times of
    one host-driven pass."""
    from paper_1912_04385_gb300 import mss
    opts = mss.options(restart=a.restart, driver=a.driver, **kw)
    host = mss.options(restart=a.restart, driver="host", **kw)

    def step(o, infos=None):
        # a variant that does not converge within maxit is reported, not fatal
        for rp, ci, v, b in dev:
            solver.setup(rp, ci, v, 6, 0, 1, opts=o)
            x, info = solver.solve(b, tol=a.tol, maxit=a.maxit)
            if infos is not None:
                infos.append(info)

    steps = leg_steps(a, 2)
    for _ in range(1):
        step(opts)
    torch.cuda.synchronize()
    infos = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step(opts, infos)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    solver.trace(True)
    solver.trace_read(reset=True)
    step(host)
    torch.cuda.synchronize()
    tr = solver.trace_read(reset=True)
    solver.trace(False)
    n_apply, apply_ms = tr["apply"]
    n_vc, vc_ms = tr["vcycle"]
    return {"options": kw, "ms_per_system": round(ms / (steps * len(dev)), 3), "steps": steps,
            "iters": [i["iters"] for i in infos[:len(dev)]],
            "status": [i["status"] for i in infos[:len(dev)]],
            "setup_ms_mean": round(float(np.mean([i["setup_ms"] for i in infos])), 3),
            "solve_ms_mean": round(float(np.mean([i["solve_ms"] for i in infos])), 3),
            "apply_ms_mean": round(apply_ms / max(n_apply, 1), 4),
            "vcycle_ms_mean": round(vc_ms / max(n_vc, 1), 4), "driver": a.driver}


def newton_leg(a, dev, solver, torch, pes=(12.0, 14.4, 17.28)):
    """Newton-loop reuse (Sec. 2.5): after the Pe = 10 benchmark system, later
    Jacobians on the same grid (same pattern) from the same generator with a
    drifting Peclet number, each handled by a new mss_setup, by
    mss_update_values keeping the pattern, and by mss_update_values keeping
    the coarsening too. Host wall ms of the set-up call (it returns with the
    set-up complete) and the iterations of the solve that follows."""
    from paper_1912_04385_gb300 import mss
    from paper_1912_04385_gb300 import synthetic as sy
    rp, ci, v, b = dev[1]
    opts = mss.options(restart=a.restart, driver=a.driver)
    jac = []
    for pe in pes:
        s = sy.plain_at_scale(a.n, pe=pe, seed=0)
        jac.append((torch.from_numpy(s.vals.reshape(-1)).cuda(), torch.from_numpy(s.b).cuda()))
    out = {}
    for mode in ("setup", "pattern", "coarsening"):
        solver.setup(rp, ci, v, 6, 0, 1, opts=opts)
        solver.solve(b, tol=a.tol, maxit=a.maxit)
        ms, its = [], []
        for vk, bk in jac:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode == "setup":
                solver.setup(rp, ci, vk, 6, 0, 1, opts=opts)
            else:
                solver.update_values(vk, reuse=mode)
            ms.append((time.perf_counter() - t0) * 1e3)
            x, info = solver.solve(bk, tol=a.tol, maxit=a.maxit)
            if info["status"] != 0:
                raise RuntimeError(f"Newton-sequence solve failed ({mode}): {info}")
            its.append(info["iters"])
        out[mode] = {"setup_ms": [round(t, 3) for t in ms], "iters": its}
    out["sequence"] = (f"the {a.n}x{a.n} Pe=10 system, then Pe " +
                       ", ".join(f"{p:g}" for p in pes) + " on the same grid; host ms of the "
                       "set-up call")
    return out


def condense_leg(a, torch, n1=6, n2=4, reps=10):
    """Static condensation (Sec. 3) of a global system on the benchmark grid
    with n1 primary and n2 secondary unknowns per cell: traced kernel times of
    mss_condense and mss_recover and their algorithmic bytes, against HBM."""
    from paper_1912_04385_gb300 import mss
    from paper_1912_04385_gb300 import synthetic as sy
    f = sy.make_full_system(a.n, a.n, n1, n2, seed=0, sigma=2.0, band=True, pe=10.0,
                            j21_neighbors=True)
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda().reshape(-1)
         for k in ("row_ptr", "col_idx", "j11", "j21", "j12", "j22", "r1", "r2")}
    fd = dict(tensors=t, n1=n1, n2=n2)
    N, nnzb = f.n_cells, f.nnzb
    del f
    g = mss.Solver()
    d1 = torch.ones(N * n1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        g.condense(fd, t["r1"], t["r2"])
        g.recover(fd, t["r2"], d1)
    g.trace(True)
    g.trace_read(reset=True)
    for _ in range(reps):
        g.condense(fd, t["r1"], t["r2"])
        g.recover(fd, t["r2"], d1)
    tr = g.trace_read(reset=True)
    g.trace(False)
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) \
        if (ROOT / "MEASURED_PEAKS.json").exists() else {"hbm_gbs": 6800.0}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # algorithmic bytes: every input and output once
    bc = (4 * (N + 1) + 8 * nnzb * (n1 * n1 + n2 * n1) + 8 * N * (n1 * n2 + n2 * n2)
          + 8 * N * (n1 + n2) + 8 * nnzb * n1 * n1 + 8 * N * n1)
    br = (4 * (N + 1) + 4 * nnzb + 8 * nnzb * n2 * n1 + 8 * N * n2 * n2 + 8 * N * n2
          + 8 * N * n1 + 8 * N * n2)
    # algorithmic FP64 flops (2 per multiply-add): Gauss-Jordan of J22 on
    # [J22 | I] (2 n2^3 FMA), T = J12 J22^-1, b, and T J21 per block
    fc = 2 * (N * (2 * n2 ** 3 + n1 * n2 * n2 + n1 * n2) + nnzb * n1 * n1 * n2)
    fr = 2 * (nnzb * n2 * n1 + N * n2 ** 3)
    out = {"workload": f"{a.n}x{a.n} cells, n1={n1} primary + n2={n2} secondary unknowns, "
                       f"J21 on the cell graph", "hbm_peak_gbs": hbm,
           "fp64_peak_tflops": round(FP64_PEAK_TFLOPS, 4)}
    for name, by, fl in (("condense", bc, fc), ("recover", br, fr)):
        nl, ms = tr[name]
        per = ms / max(nl, 1)
        gbs = by / (per * 1e-3) / 1e9
        t_hbm = by / (hbm * 1e9) * 1e3
        t_alu = fl / (FP64_PEAK_TFLOPS * 1e12) * 1e3
        out[name] = {"ms": round(per, 4), "alg_bytes": by, "alg_flops": fl, "gbs": round(gbs, 1),
                     "hbm_frac": round(gbs / hbm, 4),
                     "bound": "alu" if t_alu > t_hbm else "hbm",
                     "t_roofline_ms": round(max(t_hbm, t_alu), 4),
                     "frac": round(max(t_hbm, t_alu) / per, 4), "launches": nl}
    return out


def mixed_config_leg(a, solver, torch, stream):
    """The mixed-precision workload: one n x n, nb = 6 system (sigma = 3,
    Pe = 10), FGMRES to the bench tolerance with the FP64 and with the mixed
    preconditioner, each timed over the steps; both solutions are compared
    with an FP64 solve converged to 1e-10 (equal final accuracy check)."""
    from paper_1912_04385_gb300 import mss, synthetic as sy
    n = a.mixed_n
    s = sy.plain_at_scale(n, pe=10.0, seed=0, sigma=3.0)
    rp = torch.from_numpy(s.row_ptr).cuda()
    ci = torch.from_numpy(s.col_idx).cuda()
    v = torch.from_numpy(s.vals.reshape(-1)).cuda()
    b = torch.from_numpy(s.b).cuda()
    del s
    res = {"workload": f"cptr3-fgmres{a.restart}-{n}x{n}-nb6-sigma3-pe10", "cells": n * n,
           "driver": a.driver}
    xs = {}
    for prec in ("fp64", "mixed"):
        opts = mss.options(restart=a.restart, precision=prec, driver=a.driver)
        for _ in range(max(1, min(a.warmup, 2))):
            solver.setup(rp, ci, v, 6, 0, 1, opts=opts)
            solver.solve(b, tol=a.tol, maxit=a.maxit)
        torch.cuda.synchronize()
        ms, infos = 0.0, []
        for _ in range(leg_steps(a, 3)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.setup(rp, ci, v, 6, 0, 1, opts=opts)
            x, info = solver.solve(b, tol=a.tol, maxit=a.maxit)
            e1.record(stream)
            torch.cuda.synchronize()
            if info["status"] != 0:
                raise RuntimeError(f"{prec} solve failed at {n}x{n}: {info}")
            ms += e0.elapsed_time(e1)
            infos.append(info)
        r, bn = solver.residual_norm(rp, ci, v, 6, b, x)
        xs[prec] = x.clone()
        # kernel-class trace from one host-driven solve (a graph records no events)
        solver.trace(True)
        solver.trace_read(reset=True)
        solver.setup(rp, ci, v, 6, 0, 1,
                     opts=mss.options(restart=a.restart, precision=prec, driver="host"))
        solver.solve(b, tol=a.tol, maxit=a.maxit)
        torch.cuda.synchronize()
        tr = solver.trace_read(reset=True)
        solver.trace(False)
        n_apply, apply_ms = tr["apply"]
        res[prec] = {"ms": round(ms / leg_steps(a, 3), 3), "iters": infos[-1]["iters"],
                     "setup_ms": round(infos[-1]["setup_ms"], 3),
                     "solve_ms": round(infos[-1]["solve_ms"], 3),
                     "apply_ms_mean": round(apply_ms / max(n_apply, 1), 4),
                     "rel_res_unscaled": float(f"{r / bn:.3e}"),
                     "trace_ms": {k: [v[0], round(v[1], 3)] for k, v in tr.items()}}
    # reference solution: FP64 preconditioner, converged to 1e-10
    solver.setup(rp, ci, v, 6, 0, 1, opts=mss.options(restart=a.restart))
    xr, ir = solver.solve(b, tol=1e-10, maxit=4 * a.maxit)
    nr = float(torch.linalg.vector_norm(xr))
    for prec in ("fp64", "mixed"):
        res[prec]["rel_err_vs_fp64_1e-10"] = float(
            f"{float(torch.linalg.vector_norm(xs[prec] - xr)) / nr:.3e}")
    res["speedup_mixed_over_fp64"] = round(res["fp64"]["ms"] / res["mixed"]["ms"], 3)
    res["reference_iters"] = ir["iters"]
    return res


def learned_leg(a, dev, torch, stream):
    """Learned temperature interpolation against classical interpolation on the
    1024x1024 systems at Pe 0.1 and 1000 (set-up + solve to the bench
    tolerance, timed with CUDA events on the same stream)."""
    from paper_1912_04385_gb300 import mss
    path = ROOT / "paper_1912_04385_gb300" / "gnn_t_interp.npz"
    if not path.exists():
        return {"unavailable": "no trained parameters (paper_1912_04385_gb300/gnn_t_interp.npz)"}
    z = np.load(path)
    trained = torch.from_numpy(z["params_trained"] if "params_trained" in z else z["params"]).cuda()
    selected = torch.from_numpy(z["params"]).cuda()
    meta = json.loads(str(z["meta"]))
    solver = mss.Solver()
    out = {"params": "paper_1912_04385_gb300/gnn_t_interp.npz",
           "trained_on": f"{meta['systems']} systems of {meta['grid']}x{meta['grid']}, "
                         f"{meta['epochs']} epochs, loss norm {meta.get('norm', 'A')}",
           "loss_first_last": [meta["loss_history"][0], meta["loss_history"][-1]],
           "validation": meta["validation"],
           "fallback_to_classical": meta["fallback_to_classical"], "systems": []}
    for k, pe in enumerate(PES):
        if pe not in (0.1, 1000.0):
            continue
        rp, ci, v, b = dev[k]
        row = {"pe": pe}
        for name, kw in (("classical", {}), ("trained", {"learned_interp": trained}),
                         ("selected", {"learned_interp": selected})):
            opts = mss.options(restart=a.restart, **kw)
            solver.setup(rp, ci, v, 6, 0, 1, opts=opts)          # warm-up
            solver.solve(b, tol=a.tol, maxit=a.maxit)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.setup(rp, ci, v, 6, 0, 1, opts=opts)
            x, info = solver.solve(b, tol=a.tol, maxit=a.maxit)
            e1.record(stream)
            torch.cuda.synchronize()
            row[name] = {"iters": info["iters"], "ms": round(e0.elapsed_time(e1), 3),
                         "status": info["status"]}
        # fallback: classical whenever the trained network needs more iterations
        better = row["trained"]["iters"] < row["classical"]["iters"]
        row["with_fallback"] = dict(row["trained" if better else "classical"],
                                    uses="trained" if better else "classical")
        out["systems"].append(row)
    return out


def batch_systems(a):
    """The batched workload: grid sides uniform on [64, 512], nb in {4, 6},
    lognormal permeability (sigma 2, correlation 16), stiff band, Pe
    log-uniform on [0.1, 1000]; seeded."""
    from paper_1912_04385_gb300 import synthetic as sy
    rng = np.random.default_rng(1)
    out = []
    for k in range(a.batch):
        n = int(rng.integers(64, 513))
        nb = int(rng.choice([4, 6]))
        pe = float(10.0 ** rng.uniform(-1.0, 3.0))
        out.append(sy.make_system(n, n, nb, pe=pe, sigma=2.0, corr_len=16.0, band=True,
                                  seed=1000 + k))
    return out


def batch_leg(a, torch):
    """Aggregate solves/s and per-system latency of the batch API against the
    same systems solved one after another by one handle (host driver)."""
    from paper_1912_04385_gb300 import mss
    sysl = batch_systems(a)
    dev = [dict(row_ptr=torch.from_numpy(s.row_ptr).cuda(),
                col_idx=torch.from_numpy(s.col_idx).cuda(),
                vals=torch.from_numpy(np.ascontiguousarray(s.vals).reshape(-1)).cuda(),
                b=torch.from_numpy(s.b).cuda(), nb=s.nb, p_idx=0, t_idx=1) for s in sysl]
    cells = int(sum(s.n_cells for s in sysl))
    del sysl
    torch.cuda.synchronize()
    # one after another, one handle
    solver = mss.Solver()
    opts = mss.options(restart=a.restart)

    def sequential():
        lat, its = [], []
        for d in dev:
            t0 = time.perf_counter()
            solver.setup(d["row_ptr"], d["col_idx"], d["vals"], d["nb"], 0, 1, opts=opts)
            x, info = solver.solve(d["b"], tol=a.tol, maxit=a.maxit)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - t0) * 1e3)
            its.append(info["iters"])
            if info["status"] != 0:
                raise RuntimeError(f"sequential solve failed: {info}")
        return lat, its

    sequential()
    t0 = time.perf_counter()
    lat_s, its_s = sequential()
    wall_s = (time.perf_counter() - t0) * 1e3
    del solver
    # batched: lanes with their own streams; autotuned on the warm-up run
    B = mss.Batch(lanes=a.batch_lanes, autotune=True)
    B.solve(dev, tol=a.tol, maxit=a.maxit, restart=a.restart)
    walls, lat_b, its_b = [], [], []
    for _ in range(leg_steps(a, 3)):
        t0 = time.perf_counter()
        xs, res, inf = B.solve(dev, tol=a.tol, maxit=a.maxit, restart=a.restart)
        walls.append((time.perf_counter() - t0) * 1e3)
        if any(r["status"] != 0 for r in res):
            raise RuntimeError("batched solve failed")
        lat_b = [f["latency_ms"] for f in inf]
        its_b = [r["iters"] for r in res]
        setup_sum_b = sum(r["setup_ms"] for r in res)
        solve_sum_b = sum(r["solve_ms"] for r in res)
    wall_b = float(np.median(walls))
    assert its_b == its_s, "batched and sequential iteration counts differ"
    xs_lanes = [x.clone() for x in xs]
    # fused schedule: set-ups on the lanes, then one lock-step group solve per
    # block size through multi-system launches (tile shape tuned on the
    # warm-up run)
    F = mss.Batch(lanes=a.batch_lanes, autotune=True, schedule="fused")
    F.solve(dev, tol=a.tol, maxit=a.maxit, restart=a.restart)
    walls_f, lat_f, its_f, solve_f, setup_f = [], [], [], [], []
    for _ in range(leg_steps(a, 3)):
        t0 = time.perf_counter()
        xs, res, inf_f = F.solve(dev, tol=a.tol, maxit=a.maxit, restart=a.restart)
        walls_f.append((time.perf_counter() - t0) * 1e3)
        if any(r["status"] != 0 for r in res):
            raise RuntimeError("fused batched solve failed")
        lat_f = [f["latency_ms"] for f in inf_f]
        its_f = [r["iters"] for r in res]
        solve_f.append(max(r["solve_ms"] for r in res))
        setup_f.append(max(f["finish_ms"] - r["solve_ms"] for f, r in zip(inf_f, res)))
    wall_f = float(np.median(walls_f))
    assert its_f == its_s, "fused and sequential iteration counts differ"
    same_bits = all(bool(torch.equal(x, y)) for x, y in zip(xs, xs_lanes))
    groups = {}
    for f, d in zip(inf_f, dev):
        groups.setdefault(f["group"], {"nb": d["nb"], "systems": 0,
                                       "tile_blocks": f["tile_blocks"], "per_sm": f["per_sm"]})
        groups[f["group"]]["systems"] += 1
    n = len(dev)
    # the headline numbers are the fused schedule's (persistent multi-system
    # launches in one graph per group, tile shape from the autotuner); the
    # lanes and the one-by-one runs are the comparisons
    return {"workload": f"{n} systems, sides U[64,512], nb in {{4,6}}, Pe log-U[0.1,1000], "
                        f"sigma 2, fgmres{a.restart} to {a.tol:g}",
            "systems": n, "cells_total": cells, "schedule": "fused",
            "solves_per_s": round(n / (wall_f * 1e-3), 2),
            "wall_ms": round(wall_f, 2),
            "latency_p50_ms": round(float(np.percentile(lat_f, 50)), 3),
            "latency_p99_ms": round(float(np.percentile(lat_f, 99)), 3),
            "group_solve_ms": round(float(np.median(solve_f)), 2),
            "setup_phase_ms": round(float(np.median(setup_f)), 2),
            "groups": [groups[k] for k in sorted(groups)],
            "solutions_equal_lanes_bitwise": same_bits,
            "speedup_solves_per_s_over_sequential": round(wall_s / wall_f, 3),
            "speedup_solves_per_s_over_lanes": round(wall_b / wall_f, 3),
            "lanes": {"lanes": a.batch_lanes,
                      "solves_per_s": round(n / (wall_b * 1e-3), 2),
                      "wall_ms": round(wall_b, 2),
                      "latency_p50_ms": round(float(np.percentile(lat_b, 50)), 3),
                      "latency_p99_ms": round(float(np.percentile(lat_b, 99)), 3),
                      "setup_ms_sum": round(setup_sum_b, 1),
                      "solve_ms_sum": round(solve_sum_b, 1),
                      "tuned": [list(t) for t in B.tuned()]},
            "sequential": {"solves_per_s": round(n / (wall_s * 1e-3), 2),
                           "wall_ms": round(wall_s, 2),
                           "latency_p50_ms": round(float(np.percentile(lat_s, 50)), 3),
                           "latency_p99_ms": round(float(np.percentile(lat_s, 99)), 3)},
            "iters_total": int(sum(its_f)),
            "set_up_lanes": a.batch_lanes,
            "timing": "host clock around each call (every solution complete on return); "
                      "wall = median over the timed runs after one tuning run"}


def apply_alg_bytes(N, nnzb, nb, solver, opts):
    """Algorithmic bytes of one CPTR3 application: two V-cycles over the
    stored hierarchies (each level: A once per Jacobi sweep after the first
    pre-sweep from zero, once for the residual, P and R once, vectors), z_P,
    and both last-stage sweeps."""
    a_passes = opts.nu_pre + opts.nu_post
    tot = 0
    for which in (0, 1):
        levs = solver.amg_levels(which)
        for l, L in enumerate(levs):
            n = L["A"][0].numel() - 1
            nnz = L["A"][1].numel()
            if l == len(levs) - 1:
                tot += n * n * 8 + 2 * n * 8
                continue
            nnzp = L["P"][1].numel()
            tot += (a_passes * (nnz * 12 + (n + 1) * 4) + 2 * (nnzp * 12 + (n + 1) * 4)
                    + 8 * n * 8)
    tot += nnzb * 12 + (N + 1) * 4 + 3 * N * 8                  # z_P
    alg = algorithmic(N, nnzb, nb)
    tot += alg["bilu_fwd"]["bytes"] + alg["bilu_bwd"]["bytes"]
    tot += 2 * N * 8                                            # gather r_T
    return int(tot)


def apply_alg_flops(N, nnzb, nb, solver, opts):
    """Algorithmic FP64 flops of one CPTR3 application, counted like
    apply_alg_bytes: per V-cycle level 2 per stored entry of A for each A pass
    (the Jacobi sweeps after the first and the residual), 3 per row for each
    sweep's update, 2 per entry of P and of R; the coarsest level a dense GEMV
    (2 n^2); z_P 2 per block; both last-stage sweeps."""
    a_passes = opts.nu_pre + opts.nu_post
    tot = 0
    for which in (0, 1):
        levs = solver.amg_levels(which)
        for l, L in enumerate(levs):
            n = L["A"][0].numel() - 1
            nnz = L["A"][1].numel()
            if l == len(levs) - 1:
                tot += 2 * n * n
                continue
            nnzp = L["P"][1].numel()
            tot += a_passes * (2 * nnz + 3 * n) + 2 * (2 * nnzp)
    tot += 2 * nnzb                                             # z_P
    alg = algorithmic(N, nnzb, nb)
    tot += alg["bilu_fwd"]["flops"] + alg["bilu_bwd"]["flops"]
    return int(tot)


def precond_roofline(bytes_apply, flops_apply, apply_ms, hbm_gbs, fp64_tflops=FP64_PEAK_TFLOPS):
    """Roofline time of one application, max(bytes / HBM bandwidth, flops /
    FP64 peak), against its traced time; frac = roofline time / traced time."""
    t_hbm = bytes_apply / (hbm_gbs * 1e9) * 1e3
    t_fp64 = flops_apply / (fp64_tflops * 1e12) * 1e3
    t_roof = max(t_hbm, t_fp64)
    return {"bytes": int(bytes_apply), "flops": int(flops_apply),
            "t_hbm_ms": round(t_hbm, 4), "t_fp64_ms": round(t_fp64, 4),
            "bound": "alu" if t_fp64 >= t_hbm else "hbm", "t_roofline_ms": round(t_roof, 4),
            "achieved_ms": round(apply_ms, 4),
            "frac": round(t_roof / apply_ms, 4) if apply_ms > 0 else None}


def e2e(a, sysl, solver, opts, torch):
    pinned = []
    for s in sysl:
        pin = {}
        for name, arr in (("row_ptr", s.row_ptr), ("col_idx", s.col_idx), ("vals", s.vals),
                          ("b", s.b)):
            t = torch.empty(arr.shape, dtype={np.int32: torch.int32, np.float64: torch.float64}[
                arr.dtype.type], pin_memory=True)
            t.numpy()[...] = arr
            pin[name] = t
        x = torch.empty(s.b.shape, dtype=torch.float64, pin_memory=True)
        from paper_1912_04385_gb300 import synthetic as sy
        hs = sy.BlockSystem(pin["row_ptr"].numpy(), pin["col_idx"].numpy(), pin["vals"].numpy(),
                            pin["b"].numpy(), s.nx, s.ny, s.nb, s.p_idx, s.t_idx)
        pinned.append((hs, x, pin))
    h2d = sum(p[0].row_ptr.nbytes + p[0].col_idx.nbytes + p[0].vals.nbytes + p[0].b.nbytes
              for p in pinned)
    d2h = sum(p[1].numpy().nbytes for p in pinned)

    def step():
        for hs, x, _ in pinned:
            _, info = solver.solve_host(hs, tol=a.tol, maxit=a.maxit, opts=opts, x_out=x.numpy())
            if info["status"] != 0:
                raise RuntimeError(f"host solve failed: {info}")

    for _ in range(max(1, min(a.warmup, 2))):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    return {"value": round(ms / (a.steps * len(sysl)), 3), "unit": "ms",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "path": "mss_solve_host (pinned host buffers; copies, set-up, solve, copy-back)"}


def oracle_iterations(a):
    """The oracle's converged iteration counts of the benchmark systems by Pe
    (tests/golden/bench_oracle_iterations_<n>.json, written by a script that
    calls only the oracle), or {} when none is stored for this size."""
    it_path = ROOT / "tests" / "golden" / f"bench_oracle_iterations_{a.n}.json"
    if not it_path.exists():
        return {}
    rec = json.loads(it_path.read_text())
    return {float(r["pe"]): int(r["iters"]) for r in rec["systems"]}


def oracle_sample(a, s, iters, k=2):
    """One bounded sample of the oracle as it stands (single-threaded) on one
    benchmark system: its full set-up plus k FGMRES iterations, extrapolated
    to the system's own converged count. Returns (ms, set-up s, s/iteration,
    iterations)."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.OracleSolver.from_system(s, restart=a.restart)
    t_setup = time.perf_counter() - t0
    bb = o.scale_rhs(s.b)
    n_it = iters.get(float(s.meta["pe"]))
    if n_it is None and a.n <= 256:
        # no stored count for this size: small enough to run the oracle out
        _, info = o.fgmres(bb, tol=a.tol, maxit=a.maxit, restart=a.restart)
        n_it = info["iters"]
    t1 = time.perf_counter()
    o.fgmres(bb, tol=0.0, maxit=k, restart=a.restart)
    t_iter = (time.perf_counter() - t1) / k
    del o
    n_it = n_it or 0
    return (t_setup + n_it * t_iter) * 1e3, t_setup, t_iter, n_it


def cpu_baseline(a, sysl):
    """The oracle on a bounded sample of the same workload: for each of the
    three systems its set-up plus 2 FGMRES iterations, extrapolated with that
    system's own converged iteration count, averaged like the GPU value."""
    iters = oracle_iterations(a)
    res = [oracle_sample(a, s, iters) for s in sysl]
    value = float(np.mean([r[0] for r in res]))
    desc = "; ".join(f"Pe={s.meta['pe']:g}: set-up {r[1]:.2f} s + {r[3]} x {r[2]:.2f} s"
                     for s, r in zip(sysl, res))
    return {"value": round(value, 1), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": f"oracle set-up + 2 FGMRES iterations per {a.n}x{a.n} system, "
                      f"extrapolated to its converged count ({desc}); mean over the three "
                      f"systems",
            "iters": [r[3] for r in res]}


def run_reference(a, rank, world):
    """The oracle, single-threaded, timed on the same workload: step k samples
    system k mod 3 (set-up plus 2 iterations, extrapolated to its converged
    count); value = the mean over the systems of each system's median."""
    if rank != 0:
        return None
    sysl = systems(a)
    iters = oracle_iterations(a)
    per = {k: [] for k in range(len(sysl))}
    used = [None] * len(sysl)
    t0 = time.perf_counter()
    for step in range(a.steps):
        k = step % len(sysl)
        ms, _, _, used[k] = oracle_sample(a, sysl[k], iters)
        per[k].append(ms)
    total = time.perf_counter() - t0
    meds = [float(np.median(v)) for v in per.values() if v]
    value = float(np.mean(meds))
    sample = (f"per step one {a.n}x{a.n} system in turn (Pe {', '.join(f'{p:g}' for p in PES)}): "
              f"oracle set-up + 2 FGMRES iterations, extrapolated to that system's converged "
              f"count; value = mean over the systems of the per-system medians")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": round(total * 1e3 / max(a.steps, 1), 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA,
            "config": {**workload_config(a), "parallelism": f"replicas x{world}"},
            "cpu_baseline": {"value": round(value, 1), "unit": "ms", "cores": 1,
                             "kind": "oracle", "sample": sample,
                             "iters": used},
            "e2e": {"value": round(value, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    a = args_()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if a.impl == "ours" and world > 1:
        import torch
        import torch.distributed as dist_
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist_.init_process_group("nccl")
        dist = dist_
    if a.impl == "reference":
        out = run_reference(a, rank, world)
    else:
        out = run_ours(a, rank, world, dist)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
