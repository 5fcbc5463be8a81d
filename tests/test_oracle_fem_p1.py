"""Pins of the P1 (linear tetrahedra, Kuhn split) spatial matrices (Sec. 3.1, Eq. 8).

Each check is a closed form that does not go through the oracle's quadrature:
the barycentric mass row sums, the exact Galerkin integrals of products of
linear functions, the edge graph of the split and the 7-point Laplacian that
the split's stiffness matrix reduces to on a uniform grid.
"""

import itertools
import math

import numpy as np
import pytest

from oracle import fem, forward, kkt
from paper_1508_06103_gb300 import workloads as W

H = (0.5, 0.3, 0.7)


def test_kuhn_tetrahedra_fill_the_cell_and_share_the_main_diagonal():
    tets = fem.kuhn_tetrahedra()
    assert len(tets) == 6 and len(set(tets)) == 6
    assert all(t[0] == 0 and t[3] == 7 for t in tets)
    # every point of the unit cube lies in exactly one tetrahedron (up to faces):
    # s_i >= s_j >= s_k for exactly one ordering of distinct coordinates
    rng = np.random.default_rng(3)
    for s in rng.random((200, 3)):
        inside = 0
        for t in tets:
            i, j = int(math.log2(t[1])), int(math.log2(t[2] - t[1]))
            k = 3 - i - j
            inside += s[i] >= s[j] >= s[k]
        assert inside == 1


def test_p1_mass_row_sums_count_the_tetrahedra_of_each_node():
    # int phi_a over a tetrahedron is |T| / 4; a node in k of the six tetrahedra
    # of a cell of volume V has row sum k V / 24 (nodes 0 and 7: all six).
    Me, Ke, G = fem.element_matrices_p1(*H)
    V = np.prod(H)
    k = np.array([6, 2, 2, 2, 2, 2, 2, 6])
    assert np.allclose(Me.sum(axis=1), k * V / 24.0, rtol=1e-14, atol=0)
    assert np.allclose(Me, Me.T, atol=1e-16)
    assert np.abs(Ke.sum(axis=1)).max() < 1e-13
    for d in range(3):   # derivative of the constant: sum_b G[d][a, b] = 0
        assert np.abs(G[d].sum(axis=1)).max() < 1e-15
    # nodes that share no tetrahedron edge (e.g. e_x and e_y) do not couple
    for a, b in [(1, 2), (1, 4), (2, 4), (3, 5), (3, 6), (5, 6)]:
        assert Me[a, b] == 0 and Ke[a, b] == 0 and all(G[d][a, b] == 0 for d in range(3))


def _box_moments(L):
    """int over [0,L] of 1, x_i and x_i x_j."""
    V = float(np.prod(L))
    m1 = np.array([V * l / 2.0 for l in L])
    m2 = np.array([[V * L[i] * L[j] / (3.0 if i == j else 4.0) for j in range(3)] for i in range(3)])
    return V, m1, m2


@pytest.mark.parametrize("element", ["q1", "p1"])
def test_products_of_linear_functions_are_integrated_exactly(element):
    # Both elements reproduce linear functions, so the Galerkin matrices give
    # the exact integrals: u^T B w = int u w, u^T K w = V grad u . grad w,
    # u^T A w = sum_e a_e V_e grad u . grad w, u^T E w = sum_e (v_e . grad w) int_e u.
    cells, L = (3, 4, 2), (1.5, 1.2, 0.8)
    ncell = int(np.prod(cells))
    rng = np.random.default_rng(7)
    a_cell = 0.5 + rng.random(ncell)
    v_cell = rng.standard_normal((ncell, 3))
    B, A, Es, K = fem.spatial_matrices(cells, L, a_cell, v_cell, element)
    h = np.array(L) / np.array(cells)
    nx, ny, nz = (c + 1 for c in cells)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xyz = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1) * h
    al0, al, be0, be = 0.3, np.array([1.0, -2.0, 0.5]), -0.7, np.array([0.25, 1.5, -1.0])
    u, w = al0 + xyz @ al, be0 + xyz @ be
    V, m1, m2 = _box_moments(L)
    exact_uw = al0 * be0 * V + al0 * be @ m1 + be0 * al @ m1 + al @ m2 @ be
    assert u @ (B @ w) == pytest.approx(exact_uw, rel=1e-13)
    assert u @ (K @ w) == pytest.approx(V * al @ be, rel=1e-13)
    Ve = np.prod(h)
    assert u @ (A @ w) == pytest.approx(Ve * a_cell.sum() * al @ be, rel=1e-13)
    ez, ey, ex = np.meshgrid(np.arange(cells[2]), np.arange(cells[1]), np.arange(cells[0]), indexing="ij")
    cen = (np.stack([ex.ravel(), ey.ravel(), ez.ravel()], axis=1) + 0.5) * h
    exact_e = np.sum((v_cell @ be) * Ve * (al0 + cen @ al))
    assert u @ (Es @ w) == pytest.approx(exact_e, rel=1e-12)


def test_p1_couples_the_fifteen_kuhn_neighbours_and_its_stiffness_is_the_7_point_laplacian():
    cells = (4, 4, 4)
    L = tuple(c * h for c, h in zip(cells, H))
    ncell = 64
    B, A, Es, K = fem.spatial_matrices(cells, L, np.ones(ncell), np.tile([0.3, -0.2, 0.4], (ncell, 1)), "p1")
    n = 5
    j = 2 + n * (2 + n * 2)   # an interior node
    kuhn = {(0, 0, 0)}
    for d in range(3):
        e = [0, 0, 0]
        e[d] = 1
        kuhn |= {tuple(e), tuple(-x for x in e)}
    for d1, d2 in itertools.combinations(range(3), 2):
        e = [0, 0, 0]
        e[d1] = e[d2] = 1
        kuhn |= {tuple(e), tuple(-x for x in e)}
    kuhn |= {(1, 1, 1), (-1, -1, -1)}
    assert len(kuhn) == 15

    def offsets(M):
        row = M.getrow(j).toarray().ravel()
        return {(i % n - 2, (i // n) % n - 2, i // (n * n) - 2): row[i] for i in np.nonzero(row)[0]}

    assert set(offsets(B)) == kuhn
    assert set(offsets(Es)) <= kuhn and set(offsets(A)) <= kuhn
    V = np.prod(H)
    lap = {(0, 0, 0): 2 * V * sum(1 / h ** 2 for h in H)}
    for d in range(3):
        for s in (1, -1):
            e = [0, 0, 0]
            e[d] = s
            lap[tuple(e)] = -V / H[d] ** 2
    got = {o: v for o, v in offsets(K).items() if abs(v) > 1e-13}
    assert set(got) == set(lap)
    for o, v in lap.items():
        assert got[o] == pytest.approx(v, rel=1e-13)
    # interior mass entries: a_ii = sum over the 24 tetrahedra at a node of
    # 2 |T| / 20; an off-diagonal entry is |T| / 20 per tetrahedron holding the
    # edge: 6 for an axis edge (2 + 1 + 1 + 2 over its four cells) and for the
    # main diagonal (one cell), 4 for a face diagonal (2 in each of its two cells)
    Bo = offsets(B)
    T = V / 6.0
    assert Bo[(0, 0, 0)] == pytest.approx(24 * T / 10.0, rel=1e-13)
    assert Bo[(1, 0, 0)] == pytest.approx(6 * T / 20.0, rel=1e-13)
    assert Bo[(1, 1, 1)] == pytest.approx(6 * T / 20.0, rel=1e-13)
    assert Bo[(1, 1, 0)] == pytest.approx(4 * T / 20.0, rel=1e-13)


def _p1_mms_error(c):
    """Forward march of C = S(x) e^{-t} with P1 elements (second order in h and tau)."""
    a, v = 0.2, np.array([0.3, -0.2, 0.1])
    ncell = c ** 3
    p = kkt.Problem((c, c, c), (1.0, 1.0, 1.0), 1.0, c, 0.5, W.ALL_FACES, np.full(ncell, a),
                    np.tile(v, (ncell, 1)), np.zeros(0, dtype=np.int64), 1e-3, 1e-2, "h1h1", "p1")
    nx = c + 1
    iz, iy, ix = np.meshgrid(np.arange(nx), np.arange(nx), np.arange(nx), indexing="ij")
    xyz = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1) / c
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    pi = math.pi
    S0 = np.sin(pi * x) * np.sin(pi * y) * np.sin(pi * z)
    gS = pi * np.stack([np.cos(pi * x) * np.sin(pi * y) * np.sin(pi * z),
                        np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z),
                        np.sin(pi * x) * np.sin(pi * y) * np.cos(pi * z)], axis=1)
    t = np.arange(c + 1) * p.tau
    f = np.outer(np.exp(-t), -S0 + 3 * pi ** 2 * a * S0 + gS @ v)
    C = forward.forward_march(p, f, c0=S0)
    return np.sqrt(np.mean((C - np.outer(np.exp(-t), S0)) ** 2))


def test_p1_forward_march_converges_second_order():
    grids = (8, 16, 24)
    e = [_p1_mms_error(c) for c in grids]
    rates = [math.log(e[i] / e[i + 1]) / math.log(grids[i + 1] / grids[i]) for i in range(2)]
    assert all(1.8 < r < 2.3 for r in rates), (e, rates)


def test_p1_kkt_assembly_and_levelwise_matvec_agree():
    w = W.random_small(11, cells=(3, 4, 2), M=4)
    import dataclasses
    p = kkt.Problem.from_workload(dataclasses.replace(w, element="p1"))
    q = kkt.Problem.from_workload(w)
    F, Fq = kkt.assemble(p), kkt.assemble(q)
    x = W.random_vector(p.n, 5)
    assert np.abs(F @ x - kkt.apply(p, x)).max() < 1e-11 * np.abs(F).max() * np.abs(x).max()
    assert np.abs(F - Fq).max() > 1e-3 * np.abs(Fq).max()   # a different discretisation
