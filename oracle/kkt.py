"""The all-at-once space-time KKT system F_h U = b (Sec. 3.1-3.2, Appendix).

Test infrastructure (see the package header).

Unknowns are ordered point-block by point-block, time slowest (Sec. 3.2):
    U[((n * N + j) * 3 + c)],  c = 0 (C), 1 (G), 2 (f).

The matrix is written first in the field-major order of the Appendix,
U~ = (C^0..C^M, G^0..G^M, f^0..f^M), block row by block row, and then
permuted to the point-block order.  With a time-stepping weight theta
(theta = 1/2 is the paper's Crank-Nicolson scheme, Eq. 8) and S = A + E_s:

  A1 = B + theta tau S,      A2 = -B + (1 - theta) tau S
  B1 = B + theta tau S^T,    B2 = -B + (1 - theta) tau S^T   (= A1^T, A2^T)

  C rows, n = 0        : C^0                                          = C_0
  C rows, n = 1..M     : A2 C^{n-1} + A1 C^n
                         - tau B ((1-theta) f^{n-1} + theta f^n)      = 0
  G rows, n = 0..M-1   : B1 G^n + B2 G^{n+1}
                         + tau B3 ((1-theta) C^n + theta C^{n+1})
                                 = tau B3 ((1-theta) Ceps^n + theta Ceps^{n+1})
  G rows, n = M        : G^M                                          = 0
  f rows, n = 0..M     : sum_m (-D^{nm} G^m + W^{nm} f^m)             = 0
      D^{nm} = Mt[n,m] B,  W^{nm} = beta1 Lt[n,m] B + beta2 Mt[n,m] K

K is the stiffness matrix of the H1-H1 regularisation N_beta (Eq. 3, the
(grad f, grad g) term of Eq. 9); the H1-L2 regularisation of Sec. 4
(Example 2) replaces |grad f|^2 by f^2, so K becomes the mass matrix B
there (reg = "h1l2").

The spatial matrices B, A, E_s and K come from oracle.fem with either Q1
elements on the hexahedral cells (element = "q1") or P1 elements on the
Kuhn split of every cell (element = "p1"); the block rows are the same.

B3 = diag(s), s_j = number of sensors snapped to node j.  On Dirichlet nodes
(Gamma_1) the C and G rows are identity rows (the columns are kept), with
right-hand side p = 0 (all workloads use homogeneous Dirichlet data); the
Neumann data q is zero in all workloads, so its boundary term vanishes.

Pins: tests/test_oracle_kkt.py (two independent constructions agree, block
transposition B1 = A1^T, forward-march consistency of the state rows,
convergence orders, exact solves; both regularisers on a constant source against
the hat-function integrals and on a multilinear source against its exact energy;
the adjoint identity <A u, w> = <u, A^T w> between the state and adjoint rows;
recovery of a known source from noise-free data as beta -> 0).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem


class Problem:
    """Discrete data of one inverse problem (everything the KKT needs)."""

    def __init__(self, cells, lengths, T, M, theta, dirichlet_faces, a_cell, v_cell,
                 sensor_node, beta1, beta2, reg="h1h1", element="q1"):
        self.cells = tuple(int(c) for c in cells)
        self.lengths = tuple(float(l) for l in lengths)
        self.nodes = tuple(c + 1 for c in self.cells)
        self.N = int(np.prod(self.nodes))
        self.T = float(T)
        self.M = int(M)
        self.L = self.M + 1
        self.tau = self.T / self.M
        self.theta = float(theta)
        self.faces = int(dirichlet_faces)
        self.a_cell = np.asarray(a_cell, dtype=np.float64)
        self.v_cell = np.asarray(v_cell, dtype=np.float64).reshape(-1, 3)
        self.sensor_node = np.asarray(sensor_node, dtype=np.int64)
        self.beta1 = float(beta1)
        self.beta2 = float(beta2)
        if reg not in ("h1h1", "h1l2"):
            raise ValueError("reg must be 'h1h1' or 'h1l2'")
        self.reg = reg
        self.element = element
        self.B, self.A, self.Es, self.K = fem.spatial_matrices(self.cells, self.lengths, self.a_cell, self.v_cell,
                                                               element)
        # spatial matrix of the beta2 term: stiffness (H1-H1) or mass (H1-L2)
        self.W2 = self.K if reg == "h1h1" else self.B
        self.S = (self.A + self.Es).tocsr()
        self.Mt, self.Lt = fem.time_matrices(self.M, self.tau)
        self.dirichlet = fem.dirichlet_mask(self.cells, self.faces)
        s = np.zeros(self.N)
        np.add.at(s, self.sensor_node, 1.0)
        self.s = s
        self.P = self.N * self.L
        self.n = 3 * self.P

    @classmethod
    def from_workload(cls, w):
        return cls(w.cells, w.lengths, w.T, w.M, w.theta, w.dirichlet_faces, w.a_cell,
                   w.v_cell, w.sensor_nodes(), w.beta1, w.beta2, getattr(w, "reg", "h1h1"),
                   getattr(w, "element", "q1"))

    # index helpers ------------------------------------------------------
    def pb_index(self, n, j, c):
        """Point-block index of unknown (level n, node j, component c)."""
        return (np.asarray(n) * self.N + np.asarray(j)) * 3 + np.asarray(c)

    def field_to_pointblock(self) -> np.ndarray:
        """perm[k] = point-block index of field-major unknown k."""
        k = np.arange(self.n)
        c, rem = np.divmod(k, self.P)
        n, j = np.divmod(rem, self.N)
        return (n * self.N + j) * 3 + c


def _state_blocks(p: Problem):
    th, tau = p.theta, p.tau
    A1 = (p.B + th * tau * p.S).tocsr()
    A2 = (-p.B + (1.0 - th) * tau * p.S).tocsr()
    St = p.S.T.tocsr()
    B1 = (p.B + th * tau * St).tocsr()
    B2 = (-p.B + (1.0 - th) * tau * St).tocsr()
    return A1, A2, B1, B2


def _identity_rows(Mblk: sp.csr_matrix, rows_mask: np.ndarray, diag: bool) -> sp.csr_matrix:
    """Replace the masked rows by zero rows (diag=False) or identity rows (diag=True)."""
    keep = sp.diags((~rows_mask).astype(np.float64))
    out = keep @ Mblk
    if diag:
        out = out + sp.diags(rows_mask.astype(np.float64))
    return out.tocsr()


def assemble_field_major(p: Problem, nodes=None, levels=None) -> sp.csr_matrix:
    """F_h in the Appendix's field-major ordering (C^0..C^M, G^0..G^M, f^0..f^M).

    With `nodes` (sorted node ids) and `levels` (a contiguous range of levels)
    only the principal submatrix on those nodes and levels is built, in the
    same field-major order restricted to them (used for subdomain matrices).
    """
    M = p.M
    th, tau = p.theta, p.tau
    nodes = np.arange(p.N) if nodes is None else np.asarray(nodes)
    levels = list(range(p.L)) if levels is None else list(levels)
    N, L = len(nodes), len(levels)
    sub = lambda A: A[nodes][:, nodes].tocsr()
    A1, A2, B1, B2 = (sub(X) for X in _state_blocks(p))
    Bs, Ws = sub(p.B), sub(p.W2)
    I = sp.identity(N, format="csr")
    Z = None
    D = p.dirichlet[nodes]
    B3 = sp.diags(np.where(p.dirichlet, 0.0, p.s)[nodes])
    Mt = p.Mt.toarray()
    Lt = p.Lt.toarray()
    col = {n: k for k, n in enumerate(levels)}      # level -> block column within a field
    blocks = [[Z] * (3 * L) for _ in range(3 * L)]

    def put(r, field, m, blk):
        if m in col:
            blocks[r][field * L + col[m]] = blk

    # C rows
    for k, n in enumerate(levels):
        r = k
        if n == 0:
            put(r, 0, 0, I)
            continue
        put(r, 0, n - 1, _identity_rows(A2, D, False))
        put(r, 0, n, _identity_rows(A1, D, True))
        put(r, 2, n - 1, _identity_rows(-(1.0 - th) * tau * Bs, D, False))
        put(r, 2, n, _identity_rows(-th * tau * Bs, D, False))
    # G rows
    for k, n in enumerate(levels):
        r = L + k
        if n == M:
            put(r, 1, M, I)
            continue
        put(r, 1, n, _identity_rows(B1, D, True))
        put(r, 1, n + 1, _identity_rows(B2, D, False))
        put(r, 0, n, (1.0 - th) * tau * B3)
        put(r, 0, n + 1, th * tau * B3)
    # f rows
    for k, n in enumerate(levels):
        r = 2 * L + k
        for m in range(max(0, n - 1), min(M, n + 1) + 1):
            put(r, 1, m, -Mt[n, m] * Bs)
            put(r, 2, m, p.beta1 * Lt[n, m] * Bs + p.beta2 * Mt[n, m] * Ws)
    # every block row and column needs a defined shape for bmat
    for r in range(3 * L):
        if blocks[r][r] is None:
            blocks[r][r] = sp.csr_matrix((N, N))
    return sp.bmat(blocks, format="csr")


def assemble(p: Problem) -> sp.csr_matrix:
    """F_h in point-block order (Sec. 3.2): F = Pi F~ Pi^T with Pi the reordering."""
    Ff = assemble_field_major(p)
    perm = p.field_to_pointblock()
    Pi = sp.csr_matrix((np.ones(p.n), (perm, np.arange(p.n))), shape=(p.n, p.n))
    return (Pi @ Ff @ Pi.T).tocsr()


def assemble_box(p: Problem, nodes, levels) -> sp.csr_matrix:
    """Principal submatrix of F_h on the unknowns of `nodes` x `levels`, in the local
    point-block order (level slowest, then the given node order, then component)."""
    Ff = assemble_field_major(p, nodes, levels)
    N, L = len(nodes), len(levels)
    n = 3 * N * L
    k = np.arange(n)
    c, rem = np.divmod(k, N * L)
    t, j = np.divmod(rem, N)
    perm = (t * N + j) * 3 + c
    Pi = sp.csr_matrix((np.ones(n), (perm, k)), shape=(n, n))
    return (Pi @ Ff @ Pi.T).tocsr()


def rhs(p: Problem, c_obs: np.ndarray, c0: np.ndarray | None = None) -> np.ndarray:
    """Right-hand side b in point-block order (Appendix).

    c_obs: (M+1, s) noisy observations Ceps at the sensors, per time level.
    c0:    (N,) nodal initial state (zero if None).
    """
    N, M, th, tau = p.N, p.M, p.theta, p.tau
    b = np.zeros((p.L, N, 3))
    if c0 is not None:
        b[0, :, 0] = c0
    b[0, p.dirichlet, 0] = 0.0          # p = 0 on Gamma_1
    for n in range(M):
        g = np.zeros(N)
        np.add.at(g, p.sensor_node, (1.0 - th) * c_obs[n] + th * c_obs[n + 1])
        g *= tau
        g[p.dirichlet] = 0.0
        b[n, :, 1] = g
    return b.reshape(-1)


def apply(p: Problem, U: np.ndarray) -> np.ndarray:
    """y = F_h U level by level, from the same block rows (second construction)."""
    N, M, th, tau = p.N, p.M, p.theta, p.tau
    X = np.asarray(U, dtype=np.float64).reshape(p.L, N, 3)
    C, G, f = X[:, :, 0], X[:, :, 1], X[:, :, 2]
    A1, A2, B1, B2 = _state_blocks(p)
    D = p.dirichlet
    s = np.where(D, 0.0, p.s)
    Mt = p.Mt.toarray()
    Lt = p.Lt.toarray()
    Y = np.zeros_like(X)
    Y[0, :, 0] = C[0]
    for n in range(1, M + 1):
        yc = A2 @ C[n - 1] + A1 @ C[n] - tau * (p.B @ ((1.0 - th) * f[n - 1] + th * f[n]))
        Y[n, :, 0] = np.where(D, C[n], yc)
    for n in range(M):
        yg = B1 @ G[n] + B2 @ G[n + 1] + tau * s * ((1.0 - th) * C[n] + th * C[n + 1])
        Y[n, :, 1] = np.where(D, G[n], yg)
    Y[M, :, 1] = G[M]
    for n in range(M + 1):
        acc = np.zeros(N)
        for m in range(max(0, n - 1), min(M, n + 1) + 1):
            acc += -Mt[n, m] * (p.B @ G[m]) + p.beta1 * Lt[n, m] * (p.B @ f[m]) + p.beta2 * Mt[n, m] * (p.W2 @ f[m])
        Y[n, :, 2] = acc
    return Y.reshape(-1)


def source(p: Problem, U: np.ndarray) -> np.ndarray:
    """f component of U as an (M+1, N) array (Sec. 3.2 ordering)."""
    return np.asarray(U).reshape(p.L, p.N, 3)[:, :, 2].copy()


def structural_pattern_row(p: Problem, n: int, j: int, c: int):
    """Structural column set of row (n, j, c) as a list of (m, k, c') triples.

    The stencil of each block row above: spatial neighbours of node j are the
    nodes sharing a cell with it (27-point); identity rows hold only their
    diagonal; the sensor coupling of a G row exists only where s_j > 0.
    """
    nx, ny, nz = p.nodes
    ix, rem = j % nx, j // nx
    iy, iz = rem % ny, rem // ny
    nbrs = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                x, y, z = ix + dx, iy + dy, iz + dz
                if 0 <= x < nx and 0 <= y < ny and 0 <= z < nz:
                    nbrs.append(x + nx * (y + ny * z))
    out = []
    if c == 0:
        if n == 0 or p.dirichlet[j]:
            return [(n, j, 0)]
        for m in (n - 1, n):
            for k in nbrs:
                out += [(m, k, 0), (m, k, 2)]
    elif c == 1:
        if n == p.M or p.dirichlet[j]:
            return [(n, j, 1)]
        for m in (n, n + 1):
            for k in nbrs:
                out.append((m, k, 1))
        if p.s[j] > 0:
            out += [(n, j, 0), (n + 1, j, 0)]
    else:
        for m in (n - 1, n, n + 1):
            if 0 <= m <= p.M:
                for k in nbrs:
                    out += [(m, k, 1), (m, k, 2)]
    return out
