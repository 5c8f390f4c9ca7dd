"""The learned temperature interpolation on the GPU (mss_gnn_*, BF16 tensor-core
dense layers, FP32 activations, FP64 loss) against the FP64 oracle
(oracle/gnn.py, pinned in test_gnn_oracle.py), both built from their own
set-ups of the same seeded system (the two hierarchies agree bit for bit).

* predicted weights, loss and gradient: relative error <= 1e-3 (the dense
  layers use split BF16 operands, hi*hi + lo*hi + hi*lo, which keeps them near
  FP32; the 1e-2 bar of a plain BF16 forward is met with a wide margin);
* a network with a zero read-out leaves the temperature hierarchy and the
  solve identical to classical interpolation, bit for bit;
* with a trained-looking (nonzero) network, level 0's interpolation carries
  exactly the predicted weights and level 1 is the Galerkin product R A P;
* Adam steps on the GPU lower the loss.
"""
import numpy as np
import pytest

import oracle
from oracle import gnn
from paper_1912_04385_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sps = pytest.importorskip("scipy.sparse")


@pytest.fixture(scope="module")
def mss():
    from paper_1912_04385_gb300 import build, mss as m
    build.build()
    m.load()
    return m


CASES = [dict(nx=24, ny=20, nb=4, pe=10.0, sigma=1.0, band=True, seed=2),
         dict(nx=33, ny=29, nb=6, pe=1000.0, sigma=2.0, band=True, seed=6)]


def _sys(c):
    c = dict(c)
    return sy.make_system(c.pop("nx"), c.pop("ny"), c.pop("nb"), **c)


def _oracle_graph(s):
    o = oracle.OracleSolver.from_system(s, max_coarse=40)
    L0 = o.amg_levels(0)[0]
    return gnn.Graph(*L0.A, L0.cf, *L0.P)


def _params(seed, scale):
    th32 = gnn.init_params(seed, readout_scale=scale).astype(np.float32)
    return th32, torch.from_numpy(th32).cuda()


@pytest.mark.parametrize("case,norm", [(0, "A"), (1, "A"), (0, "D"), (1, "D")])
def test_forward_loss_grad_match_oracle(mss, case, norm):
    s = _sys(CASES[case])
    g = mss.Solver().setup_system(s, amg_max_coarse=40)
    G = mss.Gnn(g)
    og = _oracle_graph(s)
    assert (G.n, G.m, G.t) == (og.n, og.m, og.ti.size)
    assert mss.Gnn.num_params() == gnn.NPARAMS
    th32, tht = _params(1, 1.0)
    th = th32.astype(np.float64)
    w = G.weights(tht).cpu().numpy()
    wo = gnn.weights(th, og)
    ew = np.max(np.abs(w - wo)) / np.max(np.abs(wo))
    starts = np.random.default_rng(case).standard_normal((og.n, 4))
    G.set_vectors(torch.from_numpy(starts).cuda(), nu=10, norm=norm)
    grad = torch.empty(gnn.NPARAMS, dtype=torch.float32, device="cuda")
    L, _ = G.loss_grad(tht, grad)
    ev = gnn.smooth_vectors(og, starts, nu=10)
    Lo, go = gnn.loss_and_grad(th, og, ev, norm)
    gg = grad.cpu().numpy().astype(np.float64)
    eg = np.linalg.norm(gg - go) / np.linalg.norm(go)
    print(f"case {case} norm {norm}: weights {ew:.2e}, loss {L:.6e} vs {Lo:.6e}, grad {eg:.2e}")
    assert ew <= 1e-3
    assert abs(L - Lo) <= 1e-4 * Lo
    assert eg <= 1e-3
    # per parameter group
    offs = np.cumsum([0] + [int(np.prod(sh)) for _, sh in gnn.SHAPES])
    for k, (name, _) in enumerate(gnn.SHAPES):
        a, b = gg[offs[k]:offs[k + 1]], go[offs[k]:offs[k + 1]]
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(go) + 1e-12, name


def test_zero_readout_is_classical_hierarchy(mss):
    s = _sys(CASES[1])
    th32, tht = _params(3, 0.0)
    gc = mss.Solver().setup_system(s, amg_max_coarse=40)
    gl = mss.Solver().setup_system(s, amg_max_coarse=40, learned_interp=tht)
    assert len(gc.amg_levels(0)) >= 3
    for a, b in zip(gc.amg_levels(0), gl.amg_levels(0)):
        for key in ("A", "P"):
            if a.get(key) is None:
                continue
            for u, v in zip(a[key], b[key]):
                assert torch.equal(u, v), key
    xc, ic = gc.solve(torch.from_numpy(s.b).cuda(), tol=1e-8, maxit=300)
    xl, il = gl.solve(torch.from_numpy(s.b).cuda(), tol=1e-8, maxit=300)
    assert ic["iters"] == il["iters"] and torch.equal(xc, xl)


def test_learned_weights_enter_the_hierarchy(mss):
    s = _sys(CASES[0])
    th32, tht = _params(4, 0.3)
    gc = mss.Solver().setup_system(s, amg_max_coarse=40)
    G = mss.Gnn(gc)
    w = G.weights(tht).cpu().numpy()
    gl = mss.Solver().setup_system(s, amg_max_coarse=40, learned_interp=tht)
    lc, ll = gc.amg_levels(0), gl.amg_levels(0)
    cf = lc[0]["cf"].cpu().numpy()
    prp, pci, pv = (t.cpu().numpy() for t in ll[0]["P"])
    pvc = lc[0]["P"][2].cpu().numpy()
    rows = np.repeat(np.arange(cf.size), np.diff(prp))
    fmask = cf[rows] == 0
    assert np.array_equal(pv[fmask], w)            # exactly the predicted weights
    assert np.array_equal(pv[~fmask], pvc[~fmask])  # C rows: injection
    assert not np.array_equal(pv, pvc)
    # level 1 = R A P with R = P^T (host FP64 product of the copied arrays)
    arp, aci, av = (t.cpu().numpy() for t in ll[0]["A"])
    n, nc = cf.size, int(cf.sum())
    A = sps.csr_matrix((av, aci, arp), shape=(n, n))
    P = sps.csr_matrix((pv, pci, prp), shape=(n, nc))
    Ac = (P.T @ A @ P).toarray()
    brp, bci, bv = (t.cpu().numpy() for t in ll[1]["A"])
    B = sps.csr_matrix((bv, bci, brp), shape=(nc, nc)).toarray()
    assert np.max(np.abs(B - Ac)) <= 1e-12 * np.max(np.abs(Ac))
    x, info = gl.solve(torch.from_numpy(s.b).cuda(), tol=1e-8, maxit=400)
    assert info["status"] == 0


def test_adam_lowers_the_loss(mss):
    s = _sys(CASES[0])
    g = mss.Solver().setup_system(s, amg_max_coarse=40)
    G = mss.Gnn(g)
    rng = np.random.default_rng(9)
    G.set_vectors(torch.from_numpy(rng.standard_normal((G.n, 8))).cuda(), nu=10, norm="D")
    th32, p = _params(5, 0.0)
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    grad = torch.empty_like(p)
    L0, _ = G.loss_grad(p, grad)
    for step in range(1, 61):
        G.loss_grad(p, grad)
        G.adam(p, m1, m2, grad, step, lr=2e-3)
    L1, _ = G.loss_grad(p, grad)
    print(f"loss {L0:.4e} -> {L1:.4e}")
    assert L1 < 0.97 * L0


def test_selection_never_worse_than_classical(mss):
    # the trained network is kept only if it needs no more iterations than
    # classical interpolation on the validation systems; otherwise the zero
    # read-out (classical) is selected -- so the selected form never loses
    from paper_1912_04385_gb300 import train_gnn as T

    def tup(s):
        return (s.row_ptr, s.col_idx, np.ascontiguousarray(s.vals).reshape(-1), s.b)

    train = [tup(_sys(dict(nx=40, ny=40, nb=6, pe=pe, sigma=2.0, band=True, seed=20 + k)))
             for k, pe in enumerate((0.3, 30.0, 300.0, 3.0))]
    val = [tup(_sys(dict(nx=48, ny=48, nb=6, pe=pe, sigma=2.0, band=True, seed=40 + k)))
           for k, pe in enumerate((1.0, 500.0))]
    graphs = T.build_graphs(torch, mss, train, 4, 20, 3, "D")
    p = torch.from_numpy(T.initial_params(3)).cuda()
    m1, m2, g = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    step = 0
    for _ in range(3):
        for G in graphs:
            G.loss_grad(p, g)
            step += 1
            G.adam(p, m1, m2, g, step, lr=3e-4)
    sel, it_c, it_l, _, _, fallback = T.select(torch, mss, val, p)
    its, _ = T.iterations(torch, mss, val, params=torch.from_numpy(sel).cuda())
    print(f"classical {it_c}, trained {it_l}, selected {its}, fallback {fallback}")
    assert sum(its) <= sum(it_c)
    if fallback:
        assert its == it_c
