"""Training of the learned temperature interpolation (the network behind
mss_gnn_* and mss_options.learned_interp) on temperature operators that the
method itself produces: every training system is set up with CPTR3, and the
network sees level 0 of its temperature hierarchy (the scaled C_TT), its C/F
split and classical interpolation.

    python -m paper_1912_04385_gb300.train_gnn [--systems 10000] [--grid 128]
           [--buffer 256] [--steps-per-system 4]
           [--out paper_1912_04385_gb300/gnn_t_interp.npz]

Streaming: the systems are generated in bounded chunks by a process pool
while the GPU trains; every arriving system becomes a training graph that
replaces a random one of a rolling buffer, and each arrival is followed by
--steps-per-system Adam steps on graphs drawn from the buffer (a training
graph keeps its activations on the device, so 10k of them do not fit at
once). With --systems <= --buffer every graph stays resident and --epochs
passes run over them instead.

Loss: the diagonal-weighted defect of smooth test vectors (norm "D", the
least-squares criterion of bootstrap AMG) by default. The residual norm
("A") is available; trained with it, the network lowered its loss but made
the temperature V-cycle much worse (up to 8x the FGMRES iterations).

Selection and fallback: after training, a few larger validation systems are
solved with classical and with learned interpolation (FGMRES(50) to 1e-6).
If the learned network needs more iterations in total, the selected
parameters ("params") are those of a zero read-out, i.e. classical
interpolation; the trained ones are kept as "params_trained".
"""
from __future__ import annotations

import argparse
import json
import time
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import get_context
from pathlib import Path

import numpy as np

WIDTH = 32
SHAPES = [("Wn", (2, 32)), ("bn", (32,)), ("We", (5, 32)), ("be", (32,)),
          ("W1", (64, 32)), ("b1", (32,)), ("W2", (64, 32)), ("b2", (32,)),
          ("W3", (64, 32)), ("b3", (32,)), ("Wo", (96, 32)), ("bo", (32,)),
          ("wr", (32,)), ("br", (1,))]
DEFAULT_OUT = Path(__file__).resolve().parent / "gnn_t_interp.npz"


def initial_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, zero read-out (classical to start)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("b") or name == "wr":
            parts.append(np.zeros(shp))
        else:
            parts.append(rng.standard_normal(shp) * np.sqrt(2.0 / shp[0]))
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def _make(args):
    grid, pe, seed = args
    from paper_1912_04385_gb300 import synthetic as sy
    s = sy.make_system(grid, grid, 6, pe=pe, sigma=2.0, corr_len=16.0, band=True, seed=seed)
    return (s.row_ptr, s.col_idx, np.ascontiguousarray(s.vals).reshape(-1), s.b)


def _jobs(count: int, grid: int, seed: int):
    rng = np.random.default_rng(seed)
    return [(grid, float(10.0 ** rng.uniform(-1.0, 3.0)), int(seed * 100003 + k))
            for k in range(count)]


def make_systems(count: int, grid: int, seed: int, workers: int = 8):
    """configs-style 6-unknown systems: lognormal sigma 2, stiff band, Pe
    log-uniform on [0.1, 1000]; generated in a spawn pool (no CUDA there)."""
    jobs = _jobs(count, grid, seed)
    with ProcessPoolExecutor(max_workers=workers, mp_context=get_context("spawn")) as ex:
        return list(ex.map(_make, jobs, chunksize=4)), [j[1] for j in jobs]


def stream_systems(count: int, grid: int, seed: int, workers: int = 8, chunk: int = 64):
    """The same systems as make_systems, yielded one by one; at most two
    chunks are generated ahead of the consumer (bounded host memory)."""
    jobs = _jobs(count, grid, seed)
    with ProcessPoolExecutor(max_workers=workers, mp_context=get_context("spawn")) as ex:
        pending = [ex.submit(_make, j) for j in jobs[:2 * chunk]]
        nxt = len(pending)
        while pending:
            fut = pending.pop(0)
            yield fut.result()
            if nxt < len(jobs):
                pending.append(ex.submit(_make, jobs[nxt]))
                nxt += 1


def _dev(torch, sysm):
    rp, ci, v, b = sysm
    return (torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(v).cuda(),
            torch.from_numpy(b).cuda())


def graph_of(torch, mss, sysm, K: int, nu: int, rng, norm: str = "D"):
    """A training graph: level 0 of the temperature hierarchy of a CPTR3
    set-up, with K smoothed test vectors."""
    rp, ci, v, b = _dev(torch, sysm)
    solver = mss.Solver().setup(rp, ci, v, 6, 0, 1)
    G = mss.Gnn(solver)
    G.set_vectors(torch.from_numpy(rng.standard_normal((G.n, K))).cuda(), nu=nu, norm=norm)
    return G


def build_graphs(torch, mss, systems, K: int, nu: int, seed: int, norm: str = "D"):
    rng = np.random.default_rng(seed)
    return [graph_of(torch, mss, sysm, K, nu, rng, norm) for sysm in systems]


def iterations(torch, mss, systems, params=None, tol=1e-6):
    its, ms = [], []
    for sysm in systems:
        rp, ci, v, b = _dev(torch, sysm)
        kw = {} if params is None else {"learned_interp": params}
        solver = mss.Solver()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.setup(rp, ci, v, 6, 0, 1, restart=50, **kw)
        x, info = solver.solve(b, tol=tol, maxit=1000)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
        its.append(info["iters"] if info["status"] == 0 else 10 ** 6)
    return its, ms


def select(torch, mss, val, params):
    """(selected parameters as numpy, classical iterations, learned iterations,
    classical ms, learned ms): the trained parameters unless they need more
    iterations than classical interpolation on the validation systems."""
    it_c, ms_c = iterations(torch, mss, val)
    it_l, ms_l = iterations(torch, mss, val, params=params)
    fallback = sum(it_l) > sum(it_c)
    zero = params.cpu().numpy().copy()
    zero[-(WIDTH + 1):] = 0.0          # read-out wr, br = 0: classical weights
    return (zero if fallback else params.cpu().numpy()), it_c, it_l, ms_c, ms_l, fallback


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=10000)
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--buffer", type=int, default=256,
                    help="training graphs resident on the device at once")
    ap.add_argument("--steps-per-system", type=int, default=4,
                    help="Adam steps after each arriving system (streaming)")
    ap.add_argument("--epochs", type=int, default=10,
                    help="passes over the graphs when they all fit in the buffer")
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--vectors", type=int, default=8)
    ap.add_argument("--sweeps", type=int, default=40)
    ap.add_argument("--norm", default="D", choices=["A", "D"],
                    help="loss: A = residual of the defect, D = diagonal-weighted defect")
    ap.add_argument("--val-grid", type=int, default=256)
    ap.add_argument("--val-systems", type=int, default=6)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default=str(DEFAULT_OUT))
    a = ap.parse_args()

    t0 = time.perf_counter()
    val, val_pes = make_systems(a.val_systems, a.val_grid, a.seed + 1)
    import torch
    from paper_1912_04385_gb300 import build, mss
    build.build()
    mss.load()
    p = torch.from_numpy(initial_params(a.seed)).cuda()
    m1, m2, grad = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    rng = np.random.default_rng(a.seed)
    vrng = np.random.default_rng(a.seed + 17)      # test-vector starts
    step = 0
    history = []
    t1 = time.perf_counter()
    if a.systems <= a.buffer:
        systems, _ = make_systems(a.systems, a.grid, a.seed)
        graphs = [graph_of(torch, mss, sysm, a.vectors, a.sweeps, vrng, a.norm) for sysm in systems]
        del systems
        history.append(float(np.mean([G.loss_grad(p)[0] for G in graphs])))
        for ep in range(a.epochs):
            losses = []
            for k in rng.permutation(len(graphs)):
                L, _ = graphs[k].loss_grad(p, grad)
                step += 1
                graphs[k].adam(p, m1, m2, grad, step, lr=a.lr)
                losses.append(L)
            history.append(float(np.mean(losses)))
            print(f"epoch {ep + 1}: mean loss {history[-1]:.5f}", flush=True)
        n_graphs = len(graphs)
    else:
        buf, losses = [], []
        report = max(1, a.systems // 10)
        for k, sysm in enumerate(stream_systems(a.systems, a.grid, a.seed)):
            G = graph_of(torch, mss, sysm, a.vectors, a.sweeps, vrng, a.norm)
            if k == 0:
                history.append(float(G.loss_grad(p)[0]))
            if len(buf) < a.buffer:
                buf.append(G)
            else:
                buf[int(rng.integers(len(buf)))] = G     # the replaced graph is freed
            for _ in range(a.steps_per_system):
                Gk = buf[int(rng.integers(len(buf)))]
                L, _ = Gk.loss_grad(p, grad)
                step += 1
                Gk.adam(p, m1, m2, grad, step, lr=a.lr)
                losses.append(L)
            if (k + 1) % report == 0:
                history.append(float(np.mean(losses[-report * a.steps_per_system:])))
                print(f"{k + 1} systems: mean loss {history[-1]:.5f}", flush=True)
        n_graphs = a.systems
        del buf
    t_train = time.perf_counter() - t1
    # selection against classical interpolation on the validation systems
    params, it_c, it_l, ms_c, ms_l, fallback = select(torch, mss, val, p)
    meta = {"systems": n_graphs, "grid": a.grid, "pe": "log-uniform [0.1, 1000]",
            "mode": "resident" if a.systems <= a.buffer else
                    f"streaming, buffer {a.buffer}, {a.steps_per_system} steps per system",
            "epochs": a.epochs if a.systems <= a.buffer else 1, "lr": a.lr,
            "vectors": a.vectors, "sweeps": a.sweeps, "norm": a.norm,
            "steps": step, "loss_history": history,
            "wall_s": round(time.perf_counter() - t0, 1), "train_s": round(t_train, 1),
            "validation": {"grid": a.val_grid, "pe": val_pes, "iters_classical": it_c,
                           "iters_learned": it_l, "ms_classical": ms_c, "ms_learned": ms_l},
            "fallback_to_classical": bool(fallback)}
    np.savez(a.out, params=params.astype(np.float32),
             params_trained=p.cpu().numpy().astype(np.float32), meta=json.dumps(meta))
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
