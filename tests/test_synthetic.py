"""The seeded input generator shared by the oracle and the CUDA path (CPU only).

The generator stands in for the simulator Jacobians of Sec. 2-3 (cell-blocked
BSR, 5-point stencil, pressure / temperature / component rows). These tests
check the structure the workload recipe states: the block pattern and its
size, determinism under the seed, the lognormal permeability (log-variance
and Gaussian correlation), the reaction band, and the row sums the pressure
and temperature operators must have.
"""
import math

import numpy as np
import pytest

from paper_1912_04385_gb300 import synthetic as sy


@pytest.mark.parametrize("nx,ny", [(1, 1), (7, 1), (5, 3), (32, 32), (33, 17)])
def test_five_point_block_pattern(nx, ny):
    s = sy.make_system(nx, ny, 4, seed=1)
    N = nx * ny
    assert s.n_cells == N and s.vals.shape == (s.nnzb, 4, 4) and s.b.shape == (4 * N,)
    assert s.nnzb == 5 * N - 2 * nx - 2 * ny          # interior faces counted twice
    for i in range(N):
        cols = s.col_idx[s.row_ptr[i]:s.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
        x, y = i % nx, i // nx
        want = {i} | {j for j, ok in ((i - 1, x > 0), (i + 1, x < nx - 1),
                                       (i - nx, y > 0), (i + nx, y < ny - 1)) if ok}
        assert set(cols.tolist()) == want


def test_seed_determinism():
    a = sy.plain_at_scale(24, pe=10.0, seed=3)
    b = sy.plain_at_scale(24, pe=10.0, seed=3)
    c = sy.plain_at_scale(24, pe=10.0, seed=4)
    assert np.array_equal(a.vals, b.vals) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.vals, c.vals) and not np.array_equal(a.b, c.b)


def test_lognormal_field_variance_and_correlation():
    # log k = sigma g with g normalised to zero mean, unit variance; white
    # noise filtered by a Gaussian of standard deviation l has the Gaussian
    # correlation exp(-h^2 / (4 l^2)) at lag h
    rng = np.random.Generator(np.random.PCG64(5))
    n, ell, sigma = 512, 8.0, 2.0
    k = sy.lognormal_field(rng, n, n, sigma, ell)
    g = np.log(k) / sigma
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    for h in (4, 8, 16):
        rho = 0.5 * (np.mean(g * np.roll(g, h, axis=1)) + np.mean(g * np.roll(g, h, axis=0)))
        assert abs(rho - math.exp(-h * h / (4 * ell * ell))) < 0.08, (h, rho)


def test_reaction_band_is_five_percent_of_columns():
    nx, ny = 60, 20
    s = sy.make_system(nx, ny, 6, band=True, seed=2)
    assert s.meta["band_cells"] == math.ceil(0.05 * nx) * ny
    plain = sy.make_system(nx, ny, 6, band=False, seed=2)
    assert plain.meta["band_cells"] == 0


def _diag_pos(s):
    return np.array([s.row_ptr[i] + int(np.nonzero(s.col_idx[s.row_ptr[i]:s.row_ptr[i + 1]] == i)[0][0])
                     for i in range(s.n_cells)])


def test_pressure_rows_sum_to_the_compressibility():
    # TPFA rows sum to zero (no-flow boundaries); only the compressibility
    # term remains, in any permeability field and with the reaction band
    s = sy.make_system(20, 12, 6, sigma=2.0, corr_len=4.0, band=True, seed=7,
                       compressibility=1e-3)
    p = s.p_idx
    rows = np.add.reduceat(s.vals[:, p, p], s.row_ptr[:-1])
    np.testing.assert_allclose(rows, 1e-3, rtol=0, atol=1e-12)
    d = _diag_pos(s)
    off = np.ones(s.nnzb, bool)
    off[d] = False
    assert np.all(s.vals[off, p, p] <= 0.0) and np.all(s.vals[d, p, p] > 0.0)


@pytest.mark.parametrize("pe", [0.1, 10.0, 1000.0])
def test_temperature_rows_conduction_and_upwind_advection(pe):
    # uniform permeability: conduction kappa = v nx / Pe on every face,
    # upwind advection with flux v in +x: the block (c+1, c) carries
    # -(kappa + v), the block (c, c+1) -kappa, and a row sums to the
    # accumulation plus v for the inflow column x = 0
    nx, ny, v = 16, 8, 1.0
    s = sy.make_system(nx, ny, 4, pe=pe, seed=1, t_accumulation=1e-3, velocity=v)
    t = s.t_idx
    kappa = v * nx / pe
    assert s.meta["kappa"] == pytest.approx(kappa)
    for i in range(s.n_cells):
        x = i % nx
        for e in range(s.row_ptr[i], s.row_ptr[i + 1]):
            j = s.col_idx[e]
            if j == i - 1:
                assert s.vals[e, t, t] == pytest.approx(-(kappa + v))
            elif j in (i + 1, i - nx, i + nx):
                assert s.vals[e, t, t] == pytest.approx(-kappa)
        rs = s.vals[s.row_ptr[i]:s.row_ptr[i + 1], t, t].sum()
        assert rs == pytest.approx(1e-3 + (v if x == 0 else 0.0), abs=1e-9 * (1 + kappa))


def test_intra_cell_couplings_scale_with_the_local_diagonal():
    # off-diagonal entries of a diagonal block are U(-c, c) times the
    # cell-local diagonal term of their row (accumulation plus reaction)
    s = sy.make_system(12, 10, 6, band=True, seed=9, coupling=0.1,
                       compressibility=1e-3, t_accumulation=1e-3)
    d = _diag_pos(s)
    blocks = s.vals[d]
    off = ~np.eye(6, dtype=bool)
    comp = [k for k in range(6) if k not in (s.p_idx, s.t_idx)]
    # pressure row: local term = compressibility
    assert np.all(np.abs(blocks[:, s.p_idx][:, off[s.p_idx]]) <= 0.1 * 1e-3 + 1e-18)
    # component rows: local term >= 1 (accumulation), bounded by the band stiffness
    for r in comp:
        mags = np.abs(blocks[:, r][:, off[r]])
        assert mags.max() <= 0.1 * (1.0 + math.exp(8.0)) and mags.max() > 0.0


def test_triangular_family_zero_structure():
    s = sy.make_system(10, 6, 5, family="triangular", seed=4)
    d = _diag_pos(s)
    off = np.ones(s.nnzb, bool)
    off[d] = False
    comp = [k for k in range(5) if k not in (s.p_idx, s.t_idx)]
    assert np.all(s.vals[off][:, comp, :] == 0.0)          # component rows: diagonal block only
    assert np.all(s.vals[:, s.t_idx, s.p_idx] == 0.0)      # (T, P) entries
    assert np.all(s.vals[d][:, comp][:, :, s.p_idx] == 0.0)  # (s, P) entries


def test_generator_rejects_bad_layouts():
    with pytest.raises(ValueError):
        sy.make_system(4, 4, 1)
    with pytest.raises(ValueError):
        sy.make_system(4, 4, 4, p_idx=1, t_idx=1)
    with pytest.raises(ValueError):
        sy.make_system(4, 4, 4, family="other")
