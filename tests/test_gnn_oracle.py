"""Pins of the FP64 oracle of the learned temperature interpolation
(oracle/gnn.py) against what the mathematics fixes, not against itself:

* reverse-mode gradient = central finite differences of the loss (every
  parameter group, relative error <= 1e-6);
* a zero read-out reproduces classical interpolation exactly (w = p);
* the loss vanishes for test vectors that interpolation reproduces exactly
  (e = P c), and equals sum ||A e_F||^2 / sum ||A e||^2 for e zero at C points
  when P = 0 (s = -1), which pins the defect's sign and indices;
* the features of a 1D 3-point Laplacian are the hand-computed values;
* relabelling the nodes permutes the predicted weights with them.
"""
import numpy as np
import pytest

import oracle
from oracle import gnn
from paper_1912_04385_gb300 import synthetic as sy


def _graph(nx=9, ny=7, nb=4, pe=10.0, seed=2):
    s = sy.make_system(nx, ny, nb, pe=pe, sigma=1.0, band=True, seed=seed)
    o = oracle.OracleSolver.from_system(s, max_coarse=10)
    L0 = o.amg_levels(0)[0]
    return gnn.Graph(*L0.A, L0.cf, *L0.P)


@pytest.mark.parametrize("norm", ["A", "D"])
def test_gradient_matches_finite_differences(norm):
    g = _graph()
    th = gnn.init_params(1, readout_scale=1.0)
    rng = np.random.default_rng(0)
    ev = gnn.smooth_vectors(g, rng.standard_normal((g.n, 3)))
    L, gr = gnn.loss_and_grad(th, g, ev, norm)
    assert np.isclose(L, gnn.loss(th, g, ev, norm), rtol=1e-14)
    # a few parameters of every group
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in gnn.SHAPES])
    idx = np.concatenate([rng.choice(np.arange(offs[k], offs[k + 1]), min(6, offs[k + 1] - offs[k]),
                                     replace=False) for k in range(len(gnn.SHAPES))])
    h = 1e-6
    scale = np.abs(gr).max()
    for k in idx:
        tp = th.copy()
        tm = th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (gnn.loss(tp, g, ev, norm) - gnn.loss(tm, g, ev, norm)) / (2 * h)
        assert abs(fd - gr[k]) <= 1e-6 * max(abs(gr[k]), 1e-2 * scale), (k, fd, gr[k])


def test_zero_readout_is_classical():
    g = _graph()
    th = gnn.init_params(3)                  # read-out starts at zero
    assert np.array_equal(gnn.weights(th, g), g.tp)
    s, _ = gnn.forward(th, g)
    assert np.all(s == 0.0)


def test_loss_zero_in_range_of_p_and_full_defect():
    g = _graph(seed=5)
    th = gnn.init_params(0)                  # w = p
    cpts = np.nonzero(g.cf == 1)[0]
    rng = np.random.default_rng(1)
    c = rng.standard_normal((cpts.size, 2))
    e = np.zeros((g.n, 2))
    e[cpts] = c
    np.add.at(e, g.ti, g.tp[:, None] * e[g.tj])   # e_F = sum_j p_ij e_j: e = P c exactly
    assert gnn.loss(th, g, e) <= 1e-28 * max(1.0, np.sum(e ** 2))
    # s = -1 (br = -1, zero read-out weights): w = 0, defect = e at F points
    p = gnn.unpack(th)
    p["br"][:] = -1.0
    th2 = gnn.pack(p)
    e2 = rng.standard_normal((g.n, 2))
    dF = e2.copy()
    dF[g.cf == 1] = 0.0
    want = np.sum(g.matvec(dF) ** 2) / np.sum(g.matvec(e2) ** 2)
    assert np.isclose(gnn.loss(th2, g, e2), want, rtol=1e-13)
    dg = np.abs(g.diag)[:, None]
    want_d = np.sum(dg * dF ** 2) / np.sum(dg * e2 ** 2)
    assert np.isclose(gnn.loss(th2, g, e2, "D"), want_d, rtol=1e-13)


def test_features_of_1d_laplacian():
    n = 5
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                ci.append(j)
                v.append(2.0 if j == i else -1.0)
        rp.append(len(ci))
    cf = np.array([1, 0, 1, 0, 1])
    # classical P for this split: F points take 1/2 from each C neighbour
    prp = [0, 1, 3, 4, 6, 7]
    pci = [0, 0, 1, 1, 1, 2, 2]
    pv = [1.0, 0.5, 0.5, 1.0, 0.5, 0.5, 1.0]
    g = gnn.Graph(rp, ci, v, cf, prp, pci, pv)
    X, E = gnn.features(g)
    assert np.allclose(X[:, 0], 1.0)
    assert np.allclose(X[:, 1], [0.5, 0.0, 0.0, 0.0, 0.5])     # row sum / diagonal
    # edge (1, 0): a_10/a_11 = -1/2, a_01/a_00 = -1/2, |a_10|/max|a_1k| = 1, cf_1 = 0, cf_0 = 1
    e10 = [k for k in range(g.m) if g.esrc[k] == 1 and g.edst[k] == 0][0]
    assert np.allclose(E[e10], [-0.5, -0.5, 1.0, 0.0, 1.0])
    assert list(g.ti) == [1, 1, 3, 3] and list(g.tj) == [0, 2, 2, 4]


def test_relabelling_permutes_the_weights():
    g = _graph(nx=6, ny=5, seed=4)
    th = gnn.init_params(2, readout_scale=1.0)
    w = gnn.weights(th, g)
    perm = np.random.default_rng(3).permutation(g.n)      # new index of old node
    inv = np.argsort(perm)
    # permuted operator, split and interpolation (coarse order kept by C-point rank)
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    A = {(perm[i], perm[j]): a for i, j, a in zip(rows, g.ci, g.a)}
    rp2, ci2, v2 = [0], [], []
    for i in range(g.n):
        cols = sorted(j for (r, j) in A if r == i)
        ci2 += cols
        v2 += [A[(i, j)] for j in cols]
        rp2.append(len(ci2))
    cf2 = g.cf[inv]
    c_old = np.nonzero(g.cf == 1)[0]
    c_new = np.nonzero(cf2 == 1)[0]
    cidx_new = {int(f): k for k, f in enumerate(c_new)}
    entries = {}
    for t in range(g.ti.size):
        entries.setdefault(int(perm[g.ti[t]]), []).append((cidx_new[int(perm[g.tj[t]])], g.tp[t], t))
    prp2, pci2, pv2, order = [0], [], [], []
    for i in range(g.n):
        if cf2[i] == 1:
            pci2.append(cidx_new[i]); pv2.append(1.0); order.append(-1)
        else:
            for cj, pval, t in sorted(entries.get(i, [])):
                pci2.append(cj); pv2.append(pval); order.append(t)
        prp2.append(len(pci2))
    del c_old
    g2 = gnn.Graph(rp2, ci2, v2, cf2, prp2, pci2, pv2)
    w2 = gnn.weights(th, g2)
    order = np.array([t for t in order if t >= 0])
    assert np.allclose(w2, w[order], rtol=1e-12, atol=1e-14)
