"""Pins of the oracle's finite element matrices against closed forms (Appendix)."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem


def _m1(n, h):
    """1D linear mass: tridiag(h/6, 4h/6, h/6), boundary diagonal 2h/6."""
    d = np.full(n, 4 * h / 6)
    d[0] = d[-1] = 2 * h / 6
    return sp.diags([np.full(n - 1, h / 6), d, np.full(n - 1, h / 6)], [-1, 0, 1]).toarray()


def _k1(n, h):
    """1D linear stiffness: tridiag(-1, 2, -1)/h, boundary diagonal 1/h."""
    d = np.full(n, 2 / h)
    d[0] = d[-1] = 1 / h
    return sp.diags([np.full(n - 1, -1 / h), d, np.full(n - 1, -1 / h)], [-1, 0, 1]).toarray()


def _g1(n):
    """1D int phi_i phi_j': off-diagonals -1/2 (j = i-1), +1/2 (j = i+1); ends -1/2, +1/2."""
    d = np.zeros(n)
    d[0], d[-1] = -0.5, 0.5
    return sp.diags([np.full(n - 1, -0.5), d, np.full(n - 1, 0.5)], [-1, 0, 1]).toarray()


@pytest.mark.parametrize("cells,lengths", [((3, 4, 2), (1.0, 0.7, 0.4)), ((2, 2, 5), (2.0, 1.0, 1.0))])
def test_constant_coefficients_match_kronecker_closed_forms(cells, lengths):
    a, v = 0.37, np.array([0.9, -0.4, 1.3])
    ncell = int(np.prod(cells))
    B, A, Es, K = fem.spatial_matrices(cells, lengths, np.full(ncell, a), np.tile(v, (ncell, 1)))
    (nx, ny, nz) = (c + 1 for c in cells)
    hx, hy, hz = (l / c for l, c in zip(lengths, cells))
    Mx, My, Mz = _m1(nx, hx), _m1(ny, hy), _m1(nz, hz)
    Kx, Ky, Kz = _k1(nx, hx), _k1(ny, hy), _k1(nz, hz)
    Gx, Gy, Gz = _g1(nx), _g1(ny), _g1(nz)
    kron3 = lambda z, y, x: np.kron(z, np.kron(y, x))   # node id = x + nx (y + ny z)
    B_ref = kron3(Mz, My, Mx)
    K_ref = kron3(Mz, My, Kx) + kron3(Mz, Ky, Mx) + kron3(Kz, My, Mx)
    E_ref = v[0] * kron3(Mz, My, Gx) + v[1] * kron3(Mz, Gy, Mx) + v[2] * kron3(Gz, My, Mx)
    for M_, R_ in ((B, B_ref), (K, K_ref), (A, a * K_ref), (Es, E_ref)):
        assert np.abs(M_.toarray() - R_).max() <= 1e-15 * max(1.0, np.abs(R_).max()) * 10


def test_row_sums_and_total_mass_with_variable_coefficients():
    rng = np.random.default_rng(0)
    cells, lengths = (4, 3, 5), (1.0, 2.0, 0.5)
    ncell = int(np.prod(cells))
    B, A, Es, K = fem.spatial_matrices(cells, lengths, rng.uniform(0.1, 2, ncell), rng.normal(size=(ncell, 3)))
    one = np.ones(B.shape[0])
    assert np.abs(K @ one).max() < 1e-13
    assert np.abs(A @ one).max() < 1e-13
    # sum_j phi_j = 1 so sum_j int (v . grad phi_j) phi_i = 0 for cellwise constant v
    assert np.abs(Es @ one).max() < 1e-13
    assert abs(one @ (B @ one) - np.prod(lengths)) < 1e-13
    # B symmetric positive definite, K and A symmetric
    for S in (B, K, A):
        assert abs(S - S.T).max() < 1e-15


def test_convection_integrates_by_parts_on_interior_nodes():
    """E_s + E_s^T = boundary term: for nodes i, j not both on the boundary the sum vanishes."""
    rng = np.random.default_rng(1)
    cells, lengths = (4, 4, 4), (1.0, 1.0, 1.0)
    ncell = 64
    v = np.tile(rng.normal(size=3), (ncell, 1))    # constant v: div v = 0 and no jumps
    _, _, Es, _ = fem.spatial_matrices(cells, lengths, np.ones(ncell), v)
    S = (Es + Es.T).toarray()
    nx = 5
    idx = np.arange(nx ** 3)
    ix, iy, iz = idx % nx, (idx // nx) % nx, idx // nx ** 2
    interior = (ix > 0) & (ix < 4) & (iy > 0) & (iy < 4) & (iz > 0) & (iz < 4)
    assert np.abs(S[interior]).max() < 1e-15


def test_time_matrices_closed_forms():
    M, tau = 7, 0.3
    Mt, Lt = fem.time_matrices(M, tau)
    assert np.abs(Mt.toarray() - _m1(M + 1, tau)).max() < 1e-15
    assert np.abs(Lt.toarray() - _k1(M + 1, tau)).max() < 1e-14
    one = np.ones(M + 1)
    assert abs(one @ Mt @ one - M * tau) < 1e-14
    assert np.abs(Lt @ one).max() < 1e-14


def test_dirichlet_mask_faces():
    m = fem.dirichlet_mask((2, 3, 4), 1)
    nx, ny, nz = 3, 4, 5
    idx = np.arange(nx * ny * nz)
    assert np.array_equal(m, idx % nx == 0)
    m = fem.dirichlet_mask((2, 3, 4), 63)
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    assert np.array_equal(m, (ix == 0) | (ix == 2) | (iy == 0) | (iy == 3) | (iz == 0) | (iz == 4))
