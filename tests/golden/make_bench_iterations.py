"""Write bench_oracle_iterations.json: the oracle's converged FGMRES(50)
iteration counts (CPTR3, tol 1e-6) for the 1024 x 1024, nb = 6 benchmark
systems (lognormal sigma 2, correlation length 16, stiff band, seed 0,
Pe in {0.1, 10, 1000}). Calls only the oracle. Takes several minutes.

    python tests/golden/make_bench_iterations.py [n]
"""
import json
import sys
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import get_context
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

PES = (0.1, 10.0, 1000.0)


def one(args):
    n, pe = args
    import oracle
    from paper_1912_04385_gb300 import synthetic as sy
    s = sy.plain_at_scale(n, pe=pe, seed=0)
    o = oracle.OracleSolver.from_system(s, restart=50)
    _, info = o.fgmres(o.scale_rhs(s.b), tol=1e-6, maxit=1000, restart=50)
    return pe, info


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 1024
    with ProcessPoolExecutor(max_workers=3, mp_context=get_context("spawn")) as ex:
        res = list(ex.map(one, [(n, pe) for pe in PES]))
    out = {"grid": n, "nb": 6, "restart": 50, "tol": 1e-6, "scheme": "cptr3",
           "systems": [{"pe": pe, **info} for pe, info in res]}
    path = Path(__file__).with_name(f"bench_oracle_iterations_{n}.json")
    path.write_text(json.dumps(out, indent=1) + "\n")
    print(path, out)


if __name__ == "__main__":
    main()
