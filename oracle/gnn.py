"""FP64 oracle of the learned temperature-AMG interpolation (not in the paper).

TEST INFRASTRUCTURE: imported only by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``. It shares no code with
the CUDA library.

What is learned. Classical direct interpolation (Sec. 5.1 names classical AMG;
our reading of it is in the AMG oracle) gives, for every F point i, weights
p_ij on its strong C neighbours j. A message-passing network on the graph of
the temperature operator A = C_TT (level 0) predicts a relative correction
s_ij, and the learned weight is w_ij = p_ij (1 + s_ij). A net whose read-out
is zero therefore reproduces classical interpolation exactly (the fallback).

Network (width 32, every matrix product written out below):
  node input  x_i  = [a_ii / mean_k a_kk,  (sum_j a_ij) / a_ii]
  edge input  e_ij = [a_ij / a_ii,  a_ji / a_jj,  |a_ij| / max_{k!=i} |a_ik|,  cf_i,  cf_j]
                     for every stored off-diagonal entry (i, j) of A (cf = 1 for C)
  H0 = relu(X Wn + bn),  G = relu(E We + be)
  for l = 1, 2, 3:  M_i = sum_{j in N(i)} G_ij * H_j^{l-1}   (elementwise)
                    H^l = relu([H^{l-1} | M] W_l + b_l)
  read-out for every interpolation entry (i, j):
                    z = relu([H3_i | H3_j | G_ij] Wo + bo),  s_ij = z . wr + br
Loss (least-squares interpolation of smooth vectors, as in bootstrap AMG):
  test vectors e_k: nu damped-Jacobi sweeps on A e = 0 from the given starts;
  d_k = e_k - P (e_k restricted to C) (zero at C points);
  norm "A": L = sum_k ||A d_k||^2 / sum_k ||A e_k||^2 (residual of the defect);
  norm "D": L = sum_k sum_i |a_ii| d_ki^2 / sum_k sum_i |a_ii| e_ki^2.
  The denominators do not depend on the parameters.

Parameter vector layout (float, this order): Wn 2x32, bn 32, We 5x32, be 32,
W1 64x32, b1 32, W2 64x32, b2 32, W3 64x32, b3 32, Wo 96x32, bo 32, wr 32, br 1.
Matrices are row-major [in x out].
"""
from __future__ import annotations

import numpy as np

WIDTH = 32
SHAPES = [("Wn", (2, 32)), ("bn", (32,)), ("We", (5, 32)), ("be", (32,)),
          ("W1", (64, 32)), ("b1", (32,)), ("W2", (64, 32)), ("b2", (32,)),
          ("W3", (64, 32)), ("b3", (32,)), ("Wo", (96, 32)), ("bo", (32,)),
          ("wr", (32,)), ("br", (1,))]
NPARAMS = int(sum(np.prod(s) for _, s in SHAPES))


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    assert theta.shape == (NPARAMS,)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed: int = 0, readout_scale: float = 0.0):
    """He-style normal weights, zero biases; the read-out starts at zero
    (classical interpolation) unless readout_scale > 0."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("b"):
            p[name] = np.zeros(shp)
        elif name == "wr":
            p[name] = readout_scale * rng.standard_normal(shp) / np.sqrt(32)
        else:
            p[name] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[0])
    return pack(p)


class Graph:
    """The temperature operator A (CSR, diagonal stored in every row), its
    C/F split and classical P (CSR with coarse column indices)."""

    def __init__(self, rp, ci, a, cf, prp, pci, pv):
        self.rp = np.asarray(rp, np.int64)
        self.ci = np.asarray(ci, np.int64)
        self.a = np.asarray(a, np.float64)
        self.n = self.rp.shape[0] - 1
        self.cf = np.asarray(cf, np.int64)
        n = self.n
        rows = np.repeat(np.arange(n), np.diff(self.rp))
        self.rows = rows
        diag = np.zeros(n)
        offd = rows != self.ci
        diag[rows[~offd]] = self.a[~offd]
        self.diag = diag
        # off-diagonal edges in CSR order
        self.esrc = rows[offd]
        self.edst = self.ci[offd]
        self.eval = self.a[offd]
        self.m = self.esrc.shape[0]
        # coarse index -> fine index of the C points
        cpts = np.nonzero(self.cf == 1)[0]
        prp = np.asarray(prp, np.int64)
        pci = np.asarray(pci, np.int64)
        pv = np.asarray(pv, np.float64)
        prow = np.repeat(np.arange(n), np.diff(prp))
        fine = cpts[pci]
        keep = self.cf[prow] == 0          # F rows carry the interpolation entries
        self.ti = prow[keep]
        self.tj = fine[keep]
        self.tp = pv[keep]
        # edge id of every interpolation entry (i, j)
        key = {(int(i), int(j)): e for e, (i, j) in enumerate(zip(self.esrc, self.edst))}
        self.te = np.array([key[(int(i), int(j))] for i, j in zip(self.ti, self.tj)],
                           dtype=np.int64)

    def matvec(self, x):
        """A x for x of shape (n,) or (n, K)."""
        y = np.zeros_like(x)
        np.add.at(y, self.rows, self.a[:, None] * x[self.ci] if x.ndim == 2 else self.a * x[self.ci])
        return y

    def rmatvec(self, x):
        """A^T x."""
        y = np.zeros_like(x)
        np.add.at(y, self.ci, self.a[:, None] * x[self.rows] if x.ndim == 2 else self.a * x[self.rows])
        return y


def features(g: Graph):
    n = g.n
    rowsum = np.zeros(n)
    np.add.at(rowsum, g.rows, g.a)
    X = np.stack([g.diag / g.diag.mean(), rowsum / g.diag], axis=1)
    absmax = np.zeros(n)
    np.maximum.at(absmax, g.esrc, np.abs(g.eval))
    # a_ji for every edge (i, j): 0 when (j, i) is not stored
    lookup = {(int(i), int(j)): v for i, j, v in zip(g.esrc, g.edst, g.eval)}
    aji = np.array([lookup.get((int(j), int(i)), 0.0) for i, j in zip(g.esrc, g.edst)])
    E = np.stack([g.eval / g.diag[g.esrc], aji / g.diag[g.edst],
                  np.abs(g.eval) / absmax[g.esrc],
                  g.cf[g.esrc].astype(np.float64), g.cf[g.edst].astype(np.float64)], axis=1)
    return X, E


def relu(x):
    return np.maximum(x, 0.0)


def forward(theta, g: Graph):
    """s_ij for every interpolation entry, and the intermediates."""
    p = unpack(theta)
    X, E = features(g)
    H = [relu(X @ p["Wn"] + p["bn"])]
    G = relu(E @ p["We"] + p["be"])
    INs = []
    for l in (1, 2, 3):
        Hp = H[-1]
        M = np.zeros_like(Hp)
        np.add.at(M, g.esrc, G * Hp[g.edst])
        IN = np.concatenate([Hp, M], axis=1)
        INs.append(IN)
        H.append(relu(IN @ p[f"W{l}"] + p[f"b{l}"]))
    R = np.concatenate([H[3][g.ti], H[3][g.tj], G[g.te]], axis=1)
    Z = relu(R @ p["Wo"] + p["bo"])
    s = Z @ p["wr"] + p["br"][0]
    cache = dict(X=X, E=E, H=H, G=G, INs=INs, R=R, Z=Z, p=p)
    return s, cache


def weights(theta, g: Graph):
    s, _ = forward(theta, g)
    return g.tp * (1.0 + s)


def smooth_vectors(g: Graph, starts, nu: int = 10, omega: float = 2.0 / 3.0):
    """nu damped-Jacobi sweeps e <- e - omega D^-1 A e on each column of starts (n x K)."""
    e = np.array(starts, np.float64, copy=True)
    for _ in range(nu):
        e = e - omega * g.matvec(e) / g.diag[:, None]
    return e


def _residuals(w, g: Graph, evecs):
    d = evecs.copy()
    d[g.cf == 1] = 0.0
    np.subtract.at(d, g.ti, w[:, None] * evecs[g.tj])
    return d, g.matvec(d)


def _op(g: Graph, x, norm):
    """A x for the residual norm, |D|^(1/2) x for the diagonal norm."""
    return g.matvec(x) if norm == "A" else np.sqrt(np.abs(g.diag))[:, None] * x


def _op_t(g: Graph, x, norm):
    return g.rmatvec(x) if norm == "A" else np.sqrt(np.abs(g.diag))[:, None] * x


def loss(theta, g: Graph, evecs, norm="A"):
    """norm "A": sum ||A d||^2 / sum ||A e||^2; "D": sum |a_ii| d^2 / sum |a_ii| e^2."""
    w = weights(theta, g)
    d, _ = _residuals(w, g, evecs)
    r = _op(g, d, norm)
    den = np.sum(_op(g, evecs, norm) ** 2)
    return float(np.sum(r ** 2) / den)


def loss_and_grad(theta, g: Graph, evecs, norm="A"):
    """L and dL/dtheta by reverse-mode differentiation of forward()."""
    s, c = forward(theta, g)
    p = c["p"]
    w = g.tp * (1.0 + s)
    d, _ = _residuals(w, g, evecs)
    r = _op(g, d, norm)
    den = np.sum(_op(g, evecs, norm) ** 2)
    L = float(np.sum(r ** 2) / den)
    dd = _op_t(g, 2.0 * r / den, norm)               # dL/dd
    dd[g.cf == 1] = 0.0
    dw = -np.sum(dd[g.ti] * evecs[g.tj], axis=1)      # d_i = e_i - sum_j w_ij e_j
    ds = dw * g.tp
    grads = {k: np.zeros_like(v) for k, v in p.items()}
    # read-out
    Z, R = c["Z"], c["R"]
    grads["wr"] = Z.T @ ds
    grads["br"] = np.array([ds.sum()])
    dZ = np.outer(ds, p["wr"]) * (Z > 0)
    grads["Wo"] = R.T @ dZ
    grads["bo"] = dZ.sum(axis=0)
    dR = dZ @ p["Wo"].T
    H, G, INs = c["H"], c["G"], c["INs"]
    dH = np.zeros_like(H[3])
    np.add.at(dH, g.ti, dR[:, 0:32])
    np.add.at(dH, g.tj, dR[:, 32:64])
    dG = np.zeros_like(G)
    np.add.at(dG, g.te, dR[:, 64:96])
    # message-passing layers, last to first
    for l in (3, 2, 1):
        dY = dH * (H[l] > 0)
        IN = INs[l - 1]
        grads[f"W{l}"] = IN.T @ dY
        grads[f"b{l}"] = dY.sum(axis=0)
        dIN = dY @ p[f"W{l}"].T
        dHp = dIN[:, 0:32].copy()
        dM = dIN[:, 32:64]
        Hp = H[l - 1]
        dG += dM[g.esrc] * Hp[g.edst]
        np.add.at(dHp, g.edst, dM[g.esrc] * G)
        dH = dHp
    # embeddings
    dYe = dG * (G > 0)
    grads["We"] = c["E"].T @ dYe
    grads["be"] = dYe.sum(axis=0)
    dY0 = dH * (H[0] > 0)
    grads["Wn"] = c["X"].T @ dY0
    grads["bn"] = dY0.sum(axis=0)
    return L, pack(grads)
