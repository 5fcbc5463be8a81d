"""Spatial finite elements on a uniform box, and the 1D time elements.

Test infrastructure (see the package header).

The paper discretises the state and adjoint equations with continuous
piecewise-linear elements in space on a regular triangulation (Sec. 3.1,
Eq. 8) and the source with piecewise-linear elements in space and time
(Eq. 9).  Two spatial elements are built on the structured grid of cells:
  "q1": trilinear elements on the hexahedral cells;
  "p1": piecewise-linear elements on the Kuhn split of every cell into six
        tetrahedra around its main diagonal (0,0,0)-(1,1,1) (the same split
        in every cell, so the triangulation is conforming).
The Appendix names the matrices:

    A = (a grad phi_i, grad phi_j)          stiffness with diffusivity a
    B = (phi_i, phi_j)                      mass
    E : convection, (div(v phi), phi)       state and adjoint use E and E^T
    L^{mn}, K^{mn}, D^{mn}                  space-time blocks of the f equation

Every Q1 element matrix is obtained by integrating the basis functions with
2-point Gauss quadrature per axis, which is exact for these integrands
(degree <= 2 per axis).  A P1 cell matrix is the sum over its six
tetrahedra; on each, the barycentric coordinates come from inverting the
4x4 vertex matrix and the integrals from the symmetric 4-point rule, exact
for degree 2.  Coefficients a and v are constant per cell.

Convention for E (the reading of the weak form Eq. 8): the state row i
(test function phi_i) and column j (trial phi_j) hold
    E_s[i, j] = sum_e  integral_e (v_e . grad phi_j) phi_i,
and the adjoint operator uses its exact transpose.

Pins: tests/test_oracle_fem.py (Kronecker closed forms, row sums, total
mass, transpose identity; for P1: the mass row sums k V / 24 of a node in k
tetrahedra, exact integrals of products of linear functions for B, K and E,
the 15-point coupling of the split, the 7-point Laplacian stencil).
"""

from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

_GP = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])   # on [0, 1]
_GW = np.array([0.5, 0.5])


def _hat(local: int, s: np.ndarray) -> np.ndarray:
    """1D linear Lagrange basis on [0, 1]: local 0 -> 1 - s, local 1 -> s."""
    return 1.0 - s if local == 0 else s


def _dhat(local: int) -> float:
    return -1.0 if local == 0 else 1.0


def element_matrices(hx: float, hy: float, hz: float):
    """8x8 element matrices of one cell [0,hx]x[0,hy]x[0,hz].

    Local node l = lx + 2*ly + 4*lz.  Returns (Me, Ke, G) with
      Me[a, b]   = int phi_a phi_b
      Ke[a, b]   = int grad phi_a . grad phi_b
      G[d][a, b] = int (d phi_b / d x_d) phi_a
    """
    h = (hx, hy, hz)
    vol = hx * hy * hz
    Me = np.zeros((8, 8))
    Ke = np.zeros((8, 8))
    G = np.zeros((3, 8, 8))
    for qz, wz in zip(_GP, _GW):
        for qy, wy in zip(_GP, _GW):
            for qx, wx in zip(_GP, _GW):
                q = (qx, qy, qz)
                w = wx * wy * wz * vol
                val = np.zeros(8)
                grad = np.zeros((8, 3))
                for l in range(8):
                    loc = (l & 1, (l >> 1) & 1, (l >> 2) & 1)
                    f = [_hat(loc[d], q[d]) for d in range(3)]
                    val[l] = f[0] * f[1] * f[2]
                    for d in range(3):
                        g = _dhat(loc[d]) / h[d]
                        others = [f[e] for e in range(3) if e != d]
                        grad[l, d] = g * others[0] * others[1]
                Me += w * np.outer(val, val)
                Ke += w * grad @ grad.T
                for d in range(3):
                    G[d] += w * np.outer(val, grad[:, d])
    return Me, Ke, G


def kuhn_tetrahedra():
    """Local node ids (l = lx + 2 ly + 4 lz) of the six tetrahedra of the Kuhn split.

    For each ordering (i, j, k) of the axes the tetrahedron runs from node 0
    along e_i, then e_j, then e_k to node 7: the points with
    1 >= s_i >= s_j >= s_k >= 0 in cell coordinates s = x / h.
    """
    out = []
    for i, j, _ in itertools.permutations(range(3)):
        a = 1 << i
        out.append((0, a, a | (1 << j), 7))
    return out


# symmetric 4-point rule on a tetrahedron, exact for degree 2 (barycentric
# point (A, B, B, B) and its permutations, weight |T| / 4 each)
_TQ_A = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
_TQ_B = (5.0 - math.sqrt(5.0)) / 20.0


def element_matrices_p1(hx: float, hy: float, hz: float):
    """8x8 cell matrices (Me, Ke, G) of P1 elements on the Kuhn split of one cell.

    Same layout and meaning as element_matrices; each is the sum of the
    4x4 tetrahedron matrices scattered to the cell's local nodes.
    """
    h = np.array([hx, hy, hz])
    Me = np.zeros((8, 8))
    Ke = np.zeros((8, 8))
    G = np.zeros((3, 8, 8))
    for tet in kuhn_tetrahedra():
        X = np.array([[(l & 1) * h[0], ((l >> 1) & 1) * h[1], ((l >> 2) & 1) * h[2]] for l in tet])
        Tm = np.vstack([np.ones(4), X.T])   # columns (1, x, y, z) of the vertices
        vol = abs(np.linalg.det(Tm)) / 6.0
        inv = np.linalg.inv(Tm)             # lambda_k(x) = inv[k] . (1, x, y, z)
        grad = inv[:, 1:]                   # (4, 3): grad lambda_k
        idx = list(tet)
        for q in range(4):
            lam = np.full(4, _TQ_B)
            lam[q] = _TQ_A
            w = vol / 4.0
            Me[np.ix_(idx, idx)] += w * np.outer(lam, lam)
            Ke[np.ix_(idx, idx)] += w * grad @ grad.T
            for d in range(3):
                G[d][np.ix_(idx, idx)] += w * np.outer(lam, grad[:, d])
    return Me, Ke, G


ELEMENTS = ("q1", "p1")


def cell_nodes(cells) -> np.ndarray:
    """(ncell, 8) global node ids of each cell's local nodes."""
    cx, cy, cz = cells
    nx, ny = cx + 1, cy + 1
    ez, ey, ex = np.meshgrid(np.arange(cz), np.arange(cy), np.arange(cx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    out = np.zeros((ex.size, 8), dtype=np.int64)
    for l in range(8):
        ix = ex + (l & 1)
        iy = ey + ((l >> 1) & 1)
        iz = ez + ((l >> 2) & 1)
        out[:, l] = ix + nx * (iy + ny * iz)
    return out


def _assemble(cells, coef_elem) -> sp.csr_matrix:
    """sum_e coef_elem[e] (8x8) scattered to the global node numbering."""
    nodes = cell_nodes(cells)
    N = int(np.prod([c + 1 for c in cells]))
    rows = np.repeat(nodes, 8, axis=1).ravel()
    cols = np.tile(nodes, (1, 8)).ravel()
    vals = coef_elem.reshape(len(nodes), 64).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()


def spatial_matrices(cells, lengths, a_cell, v_cell, element: str = "q1"):
    """Global B (mass), A (stiffness with a), E_s (state convection), K (Laplacian).

    Appendix element matrices; E_s follows the weak form of Eq. 8 (row = test).
    element: "q1" (trilinear hexahedra) or "p1" (linear tetrahedra, Kuhn split).
    """
    if element not in ELEMENTS:
        raise ValueError(f"element must be one of {ELEMENTS}")
    hx, hy, hz = (l / c for l, c in zip(lengths, cells))
    Me, Ke, G = (element_matrices if element == "q1" else element_matrices_p1)(hx, hy, hz)
    ncell = int(np.prod(cells))
    a_cell = np.asarray(a_cell, dtype=np.float64).reshape(ncell)
    v_cell = np.asarray(v_cell, dtype=np.float64).reshape(ncell, 3)
    B = _assemble(cells, np.broadcast_to(Me, (ncell, 8, 8)))
    K = _assemble(cells, np.broadcast_to(Ke, (ncell, 8, 8)))
    A = _assemble(cells, a_cell[:, None, None] * Ke[None])
    conv = np.einsum("ed,dab->eab", v_cell, G)
    Es = _assemble(cells, conv)
    return B, A, Es, K


def time_matrices(M: int, tau: float):
    """1D linear-hat mass Mt and stiffness Lt on the levels t^0..t^M (step tau).

    Mt[m, n] = int g^m g^n dt,  Lt[m, n] = int (g^m)' (g^n)' dt  (Appendix
    L^{mn}, D^{mn} time factors), by 2-point Gauss on each interval.
    """
    Mt = np.zeros((M + 1, M + 1))
    Lt = np.zeros((M + 1, M + 1))
    for k in range(M):   # interval [t^k, t^{k+1}]
        for q, w in zip(_GP, _GW):
            val = np.array([1.0 - q, q])
            der = np.array([-1.0, 1.0]) / tau
            idx = [k, k + 1]
            for a in range(2):
                for b in range(2):
                    Mt[idx[a], idx[b]] += w * tau * val[a] * val[b]
                    Lt[idx[a], idx[b]] += w * tau * der[a] * der[b]
    return sp.csr_matrix(Mt), sp.csr_matrix(Lt)


def dirichlet_mask(cells, faces: int) -> np.ndarray:
    """Boolean (N,) mask of the nodes on the Dirichlet faces Gamma_1."""
    cx, cy, cz = cells
    nx, ny, nz = cx + 1, cy + 1, cz + 1
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = np.zeros(ix.shape, dtype=bool)
    if faces & 1:
        m |= ix == 0
    if faces & 2:
        m |= ix == cx
    if faces & 4:
        m |= iy == 0
    if faces & 8:
        m |= iy == cy
    if faces & 16:
        m |= iz == 0
    if faces & 32:
        m |= iz == cz
    return m.ravel()
