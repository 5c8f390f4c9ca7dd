"""Seeded synthetic cell-blocked Jacobians standing in for simulator output.

The paper's linear systems are Jacobians of a thermal-compositional simulator
(Sec. 2, Eqs. ADR/mass/energy) after static condensation (Sec. 3, Eq. reduced).
Those matrices are not available, so this module assembles systems with the
same structure on a 2D grid with a 5-point finite-volume stencil:

* one nb x nb block per cell pair (cell-interleaved BSR, Sec. 4 Remark on
  interleaving), unknown ``p_idx`` = pressure, ``t_idx`` = temperature, the
  remaining nb-2 unknowns are component/saturation variables;
* pressure rows: TPFA transmissibility Laplacian (harmonic-mean faces) plus a
  compressibility term on the diagonal (elliptic, Sec. 4.1);
* temperature rows: uniform conduction kappa plus first-order upwind
  advection in +x (the ADR structure of Eq. ADR / Eq. energy); the Peclet
  number of Eq. pe, Pe = v L / kappa with L = nx cells, is varied through
  kappa while the velocity is kept fixed, as the paper varies Pe (Sec. 5.1);
* component rows: the same upwind advection plus unit accumulation
  (hyperbolic);
* an optional band of stiff cells standing in for an Arrhenius reaction front
  (Eq. Arrhenius): exp(U(0, 8)) added to the temperature and component
  diagonals;
* random intra-cell coupling: every off-diagonal entry (r, c) of a diagonal
  block is U(-coupling, coupling) times the cell-local diagonal term of row r
  (its accumulation plus reaction stiffness, i.e. the part of the diagonal
  that does not come from face fluxes). Scaling by the whole diagonal, flux
  terms included, perturbs the decoupled pressure diagonal by a few percent
  of the transmissibility sum, far more than the compressibility, and makes
  the decoupled pressure matrix indefinite; the paper's decoupled pressure
  matrix is definite (Sec. 5.1, eigenvalue study).

This module only draws inputs. It contains none of the preconditioner's
arithmetic and serves both the oracle and the CUDA path.

Random draw order (numpy PCG64(seed)): permeability field, band position,
band stiffness, diagonal-block couplings, neighbour-block couplings, rhs.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["BlockSystem", "FullSystem", "make_system", "make_full_system", "lognormal_field",
           "tiny_plain", "plain_at_scale", "poisson_csr"]


@dataclass
class BlockSystem:
    """A BSR system A x = b with row-major nb x nb blocks (float64)."""
    row_ptr: np.ndarray      # int32 [N + 1]
    col_idx: np.ndarray      # int32 [nnzb], ascending within each row
    vals: np.ndarray         # float64 [nnzb, nb, nb]
    b: np.ndarray            # float64 [N * nb], cell-interleaved
    nx: int
    ny: int
    nb: int
    p_idx: int = 0
    t_idx: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return self.row_ptr.shape[0] - 1

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])


def lognormal_field(rng: np.random.Generator, nx: int, ny: int, sigma: float,
                    corr_len: float) -> np.ndarray:
    """k = exp(sigma * g), g = white noise convolved (periodic FFT) with a
    Gaussian kernel of standard deviation ``corr_len`` cells, normalised to
    zero mean and unit variance. Returns shape (ny, nx)."""
    white = rng.standard_normal((ny, nx))
    wx = 2.0 * np.pi * np.fft.fftfreq(nx)
    wy = 2.0 * np.pi * np.fft.fftfreq(ny)
    transfer = np.exp(-0.5 * corr_len ** 2 * (wy[:, None] ** 2 + wx[None, :] ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(white) * transfer))
    g -= g.mean()
    sd = g.std()
    if sd > 0:
        g /= sd
    return np.exp(sigma * g)


def make_system(nx: int, ny: int, nb: int = 4, *, pe: float = 1.0,
                sigma: float = 0.0, corr_len: float = 16.0, band: bool = False,
                seed: int = 0, p_idx: int = 0, t_idx: int = 1,
                compressibility: float = 1e-3, t_accumulation: float = 1e-3,
                coupling: float = 0.1, velocity: float = 1.0,
                couple_neighbors: bool = False,
                family: str = "standard") -> BlockSystem:
    """Assemble one synthetic thermal-compositional Jacobian.

    ``family="triangular"`` removes the couplings that would keep the scaled
    matrix from being exactly upper-block-triangular in [s, P, T] order:
    component rows keep only their diagonal block, and the (s, P) and (T, P)
    entries are zero everywhere.
    """
    if nb < 2:
        raise ValueError("nb must be >= 2")
    if not (0 <= p_idx < nb and 0 <= t_idx < nb and p_idx != t_idx):
        raise ValueError("p_idx and t_idx must be distinct indices in [0, nb)")
    if family not in ("standard", "triangular"):
        raise ValueError("family must be 'standard' or 'triangular'")
    if family == "triangular" and couple_neighbors:
        raise ValueError("the triangular family has no neighbour couplings")
    rng = np.random.Generator(np.random.PCG64(seed))
    N = nx * ny
    s_idx = [k for k in range(nb) if k not in (p_idx, t_idx)]

    # ---- permeability and face transmissibilities -------------------------
    if sigma > 0.0:
        perm = lognormal_field(rng, nx, ny, sigma, corr_len)
    else:
        perm = np.ones((ny, nx))
    kx = perm
    tx = 2.0 * kx[:, :-1] * kx[:, 1:] / (kx[:, :-1] + kx[:, 1:])   # (ny, nx-1)
    ty = 2.0 * kx[:-1, :] * kx[1:, :] / (kx[:-1, :] + kx[1:, :])   # (ny-1, nx)
    tx_mean = float(tx.mean()) if tx.size else 1.0
    flux_x = velocity * tx / tx_mean                  # upwind fluxes, +x
    flux_out = velocity * kx[:, -1] / tx_mean          # right-boundary outflow
    kappa = velocity * nx / pe

    # ---- block pattern (5-point, columns ascending) -----------------------
    cells = np.arange(N, dtype=np.int64)
    xs = cells % nx
    ys = cells // nx
    offs = [-nx, -1, 0, 1, nx]
    valid = np.stack([ys > 0, xs > 0, np.ones(N, bool), xs < nx - 1,
                      ys < ny - 1])                     # (5, N)
    counts = valid.sum(axis=0)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    slot = np.cumsum(valid, axis=0) - 1                  # position in row
    blk = np.where(valid, row_ptr[:-1][None, :] + slot, -1)   # (5, N)
    nnzb = int(row_ptr[-1])
    col_idx = np.empty(nnzb, dtype=np.int64)
    for d, off in enumerate(offs):
        m = valid[d]
        col_idx[blk[d, m]] = cells[m] + off
    vals = np.zeros((nnzb, nb, nb))
    diag = blk[2]

    # x faces: cell c (x < nx-1) -> c + 1 ; y faces: c (y < ny-1) -> c + nx
    cx = cells[xs < nx - 1]
    cy = cells[ys < ny - 1]
    Tx = tx.reshape(-1)            # ordered by (y, x) for x < nx-1: matches cx
    Ty = ty.reshape(-1)            # ordered by (y, x) for y < ny-1: matches cy
    bx_r = blk[3, cx]              # block (c, c+1)
    bx_l = blk[1, cx + 1]          # block (c+1, c)
    by_u = blk[4, cy]              # block (c, c+nx)
    by_d = blk[0, cy + nx]         # block (c+nx, c)

    # pressure: TPFA Laplacian + compressibility
    p = p_idx
    vals[bx_r, p, p] -= Tx
    vals[bx_l, p, p] -= Tx
    np.add.at(vals[:, p, p], diag[cx], Tx)
    np.add.at(vals[:, p, p], diag[cx + 1], Tx)
    vals[by_u, p, p] -= Ty
    vals[by_d, p, p] -= Ty
    np.add.at(vals[:, p, p], diag[cy], Ty)
    np.add.at(vals[:, p, p], diag[cy + nx], Ty)
    vals[diag, p, p] += compressibility
    local = np.zeros((N, nb))          # cell-local diagonal terms per row
    local[:, p] = compressibility

    # temperature: uniform conduction kappa
    t = t_idx
    vals[bx_r, t, t] -= kappa
    vals[bx_l, t, t] -= kappa
    np.add.at(vals[:, t, t], diag[cx], kappa)
    np.add.at(vals[:, t, t], diag[cx + 1], kappa)
    vals[by_u, t, t] -= kappa
    vals[by_d, t, t] -= kappa
    np.add.at(vals[:, t, t], diag[cy], kappa)
    np.add.at(vals[:, t, t], diag[cy + nx], kappa)
    vals[diag, t, t] += t_accumulation
    local[:, t] = t_accumulation

    # upwind advection in +x for temperature and components
    Fx = flux_x.reshape(-1)
    right = cells[xs == nx - 1]
    Fb = flux_out.reshape(-1)      # one per row y, ordered like `right`
    for var in [t] + s_idx:
        np.add.at(vals[:, var, var], diag[cx], Fx)          # outflow of c
        vals[bx_l, var, var] -= Fx                          # inflow of c+1
        np.add.at(vals[:, var, var], diag[right], Fb)       # boundary outflow
    for var in s_idx:
        vals[diag, var, var] += 1.0                         # accumulation
        local[:, var] = 1.0

    # stiff reaction band
    band_cells = np.zeros(0, dtype=np.int64)
    if band:
        w = int(math.ceil(0.05 * nx))
        x0 = int(rng.integers(0, nx - w + 1))
        band_cells = cells[(xs >= x0) & (xs < x0 + w)]
        rows_stiff = sorted([t] + s_idx)
        stiff = np.exp(rng.uniform(0.0, 8.0, size=(band_cells.size, len(rows_stiff))))
        for k, r in enumerate(rows_stiff):
            vals[diag[band_cells], r, r] += stiff[:, k]
            local[band_cells, r] += stiff[:, k]

    if family == "triangular":
        # component rows keep only their diagonal block
        off = np.ones(nnzb, bool)
        off[diag] = False
        for r in s_idx:
            vals[off, r, :] = 0.0

    # intra-cell couplings scaled by the cell-local diagonal term of the row
    cpl = rng.uniform(-coupling, coupling, size=(N, nb, nb))
    dblk = vals[diag]                                       # (N, nb, nb) copy
    offmask = ~np.eye(nb, dtype=bool)
    dblk = np.where(offmask[None], cpl * local[:, :, None], dblk)
    vals[diag] = dblk

    if couple_neighbors:
        off = np.ones(nnzb, bool)
        off[diag] = False
        nbl = vals[off]
        cpn = rng.uniform(-coupling, coupling, size=nbl.shape)
        nrd = np.abs(np.einsum("nii->ni", nbl))
        nbl = np.where(offmask[None], cpn * nrd[:, :, None], nbl)
        vals[off] = nbl

    if family == "triangular":
        for r in s_idx:
            vals[diag, r, p] = 0.0
        vals[:, t, p] = 0.0

    b = rng.standard_normal(N * nb)
    meta = dict(pe=pe, sigma=sigma, corr_len=corr_len, band=band, seed=seed,
                kappa=kappa, velocity=velocity, family=family,
                couple_neighbors=couple_neighbors, band_cells=int(band_cells.size),
                local_diag=local)
    return BlockSystem(row_ptr.astype(np.int32), col_idx.astype(np.int32),
                       np.ascontiguousarray(vals), b, nx, ny, nb, p_idx, t_idx,
                       meta)


@dataclass
class FullSystem:
    """The global system J delta = -r of Sec. 3 (Eq. global) before static
    condensation: per cell n1 primary and n2 secondary unknowns, the
    secondary ones coupled only inside their cell. J11 (primary equations,
    primary unknowns) and J21 (secondary equations, primary unknowns) have
    the cell graph's block pattern; J12 and J22 are one block per cell.
    Blocks row-major; vectors cell-interleaved."""
    row_ptr: np.ndarray      # int32 [N + 1]
    col_idx: np.ndarray      # int32 [nnzb]
    j11: np.ndarray          # float64 [nnzb, n1, n1]
    j21: np.ndarray          # float64 [nnzb, n2, n1]
    j12: np.ndarray          # float64 [N, n1, n2]
    j22: np.ndarray          # float64 [N, n2, n2]
    r1: np.ndarray           # float64 [N * n1]
    r2: np.ndarray           # float64 [N * n2]
    nx: int
    ny: int
    n1: int
    n2: int
    p_idx: int = 0
    t_idx: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return self.row_ptr.shape[0] - 1

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])


def make_full_system(nx: int, ny: int, n1: int = 6, n2: int = 4, *, seed: int = 0,
                     coupling: float = 0.1, j21_neighbors: bool = False,
                     **kw) -> FullSystem:
    """A global system with secondary unknowns around a ``make_system``
    primary block (J11 = its blocks, r1 = minus its right-hand side; ``kw``
    goes to make_system). The secondary rows stand in for the local
    constraints of Sec. 2.3 (fugacity, phase constraints), aligned with their
    unknowns so J22 needs no pivoting (Sec. 3):
    * J22: diagonal U(1, 2), off-diagonal U(-coupling, coupling) times the
      row's diagonal (diagonally dominant for n2 <= 10);
    * J12: U(-coupling, coupling) times the cell-local diagonal term of the
      primary row (as make_system's intra-cell couplings);
    * J21: diagonal block U(-0.5, 0.5) times the secondary row's diagonal;
      with ``j21_neighbors`` the neighbour blocks U(-coupling/5,
      coupling/5) times it, else zero;
    * r2: standard normal.
    Draws come from a second stream PCG64([seed, 1]) in this order, so the
    primary block is make_system's exactly."""
    if n1 < 2 or n2 < 0:
        raise ValueError("n1 >= 2 and n2 >= 0 required")
    base = make_system(nx, ny, n1, seed=seed, **kw)
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    N, nnzb = base.n_cells, base.nnzb
    d22 = rng.uniform(1.0, 2.0, size=(N, n2))
    j22 = rng.uniform(-coupling, coupling, size=(N, n2, n2)) * d22[:, :, None]
    j22[:, np.arange(n2), np.arange(n2)] = d22
    local = base.meta["local_diag"]
    j12 = rng.uniform(-coupling, coupling, size=(N, n1, n2)) * local[:, :, None]
    rows = np.repeat(np.arange(N), np.diff(base.row_ptr))
    diag = base.col_idx == rows
    j21 = np.zeros((nnzb, n2, n1))
    j21[diag] = rng.uniform(-0.5, 0.5, size=(N, n2, n1)) * d22[:, :, None]
    if j21_neighbors:
        off = ~diag
        j21[off] = (rng.uniform(-coupling / 5, coupling / 5, size=(int(off.sum()), n2, n1))
                    * d22[rows[off]][:, :, None])
    r2 = rng.standard_normal(N * n2)
    meta = dict(base.meta, n2=n2, j21_neighbors=j21_neighbors)
    return FullSystem(base.row_ptr, base.col_idx, base.vals, np.ascontiguousarray(j21),
                      np.ascontiguousarray(j12), np.ascontiguousarray(j22), -base.b, r2,
                      nx, ny, n1, n2, base.p_idx, base.t_idx, meta)


def tiny_plain(seed: int = 0, pe: float = 1.0, n: int = 32, nb: int = 4) -> BlockSystem:
    """32x32 grid, nb=4, homogeneous permeability, Pe=1 (the small case)."""
    return make_system(n, n, nb, pe=pe, sigma=0.0, band=False, seed=seed)


def plain_at_scale(n: int = 512, pe: float = 10.0, seed: int = 0, sigma: float = 2.0,
                   nb: int = 6) -> BlockSystem:
    """n x n grid, nb=6, lognormal permeability (sigma, correlation length 16),
    stiff reaction band; Pe from the sweep {0.1, 10, 1000}."""
    return make_system(n, n, nb, pe=pe, sigma=sigma, corr_len=16.0, band=True,
                       seed=seed)


def poisson_csr(nx: int, ny: int = 1):
    """Scalar 5-point (2D) or 3-point (1D) Dirichlet Poisson matrix in CSR:
    diagonal 2 per dimension, -1 per neighbour. Returns (row_ptr, col_idx, vals)."""
    N = nx * ny
    cells = np.arange(N)
    xs = cells % nx
    ys = cells // nx
    offs = [-nx, -1, 0, 1, nx]
    valid = np.stack([ys > 0, xs > 0, np.ones(N, bool), xs < nx - 1, ys < ny - 1])
    if ny == 1:
        valid[0] = False
        valid[4] = False
    dval = 2.0 * (2 if ny > 1 else 1)
    rows, cols, vs = [], [], []
    for d, off in enumerate(offs):
        m = valid[d]
        rows.append(cells[m])
        cols.append(cells[m] + off)
        vs.append(np.full(m.sum(), dval if off == 0 else -1.0))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vs = np.concatenate(vs)
    order = np.lexsort((cols, rows))
    rows, cols, vs = rows[order], cols[order], vs[order]
    rp = np.zeros(N + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    return rp.astype(np.int32), cols.astype(np.int32), vs.astype(np.float64)
