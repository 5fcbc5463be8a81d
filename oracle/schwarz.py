"""Space-time Schwarz preconditioners (Sec. 3.2).

Test infrastructure (see the package header).

* partition / subdomain boxes: the space-time domain is split into
  N_s x N_t non-overlapping boxes of nodes x time levels (part k of n items
  over p parts holds floor(n/p) + (k < n mod p) items), each extended by
  `overlap` nodes / levels on every side and trimmed to the domain (Sec. 3.2,
  Fig. 1).
* M_ij: the principal submatrix of F_h on the extended box (all three
  unknowns of every point), which equals the discretisation of Eq. 10 with
  the homogeneous Dirichlet conditions Eqs. 11-12 on the cut faces.
* Local solvers: ILU(0) on the structural pattern of F_h (the stencil of
  each block row, textbook IKJ order), ILU(k) (the same elimination on the
  pattern grown by levels of fill up to k, Table 1), the 3x3 point-block
  ILU(0) (the same elimination on the pattern of whole point blocks, Sec. 3.2's
  point-block ordering), or exact sparse LU (scipy, as one step).
* One-level restricted additive Schwarz, the cited Cai-Sarkis form
      z = sum_ij (R^0_ij)^T  M_ij^{-1}  R^delta_ij r
  (restricted prolongation); variant="harmonic" gives the literal operand
  order of the paper's formula, (R^delta)^T M^{-1} R^0.
* Nested coarse space-time mesh, multilinear interpolation I^h_c in
  (x, y, z, t) for each of C, G, f, restriction I^c_h = (I^h_c)^T, and the
  multiplicative two-level hybrid
      y = I^h_c F_c^{-1} I^c_h x,   z = y + M_one^{-1} (x - F_h y)
  with F_c^{-1} = GMRES right-preconditioned by the coarse one-level RAS.
* The coarse operator is rediscretised on the coarse mesh: a and v of a
  coarse cell are the means over its fine cells, and each fine sensor node
  is snapped to the nearest coarse node (ties toward the lower index).

Pins: tests/test_oracle_schwarz.py (ILU(0) defining property (LU)_ij = a_ij
on the pattern, ILU(0) = LU without fill, one box with exact LU = exact
inverse, interpolation reproduces multilinear functions, <Pu, w> = <u, P^T w>,
coarse mesh equal to fine mesh with an exact coarse solve is exact; ILU(k):
the textbook fill diagonals of the 5-point Laplacian for k = 1, 2, the ILU
property on the level-1 pattern of a KKT box, exact LU at a high level;
point-block ILU(0): whole 3x3 blocks of the 81-point neighbourhood, exact LU
on a box of one spatial node, where the block matrix is block tridiagonal).
"""

from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import kkt, krylov


def partition(n: int, p: int) -> List[Tuple[int, int]]:
    """Split range(n) into p contiguous parts, the first n mod p one longer."""
    base, extra = divmod(n, p)
    out, s = [], 0
    for k in range(p):
        e = s + base + (1 if k < extra else 0)
        out.append((s, e))
        s = e
    return out


@dataclasses.dataclass
class Box:
    own: Tuple[Tuple[int, int], ...]   # (x, y, z, t) half-open owned ranges
    ext: Tuple[Tuple[int, int], ...]   # extended (overlapping) ranges, trimmed

    def shape(self):
        return tuple(e - s for s, e in self.ext)


def boxes(p: kkt.Problem, nsub: Sequence[int], overlap: int) -> List[Box]:
    dims = list(p.nodes) + [p.L]
    parts = [partition(n, k) for n, k in zip(dims, nsub)]
    out = []
    for it in range(nsub[3]):
        for iz in range(nsub[2]):
            for iy in range(nsub[1]):
                for ix in range(nsub[0]):
                    own = (parts[0][ix], parts[1][iy], parts[2][iz], parts[3][it])
                    ext = tuple((max(0, s - overlap), min(n, e + overlap)) for (s, e), n in zip(own, dims))
                    out.append(Box(own, ext))
    return out


def box_nodes_levels(p: kkt.Problem, b: Box):
    """Node ids (x fastest) and level range of a box's extended set."""
    nx, ny, nz = p.nodes
    (x0, x1), (y0, y1), (z0, z1), (t0, t1) = b.ext
    z, y, x = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    return (x + nx * (y + ny * z)).ravel(), range(t0, t1)


def box_unknowns(p: kkt.Problem, b: Box):
    """Global point-block indices of the box's unknowns in local lexicographic
    order (t slowest, then z, y, x, then component), and a mask of the owned ones."""
    nx, ny, nz = p.nodes
    (x0, x1), (y0, y1), (z0, z1), (t0, t1) = b.ext
    t, z, y, x, c = np.meshgrid(np.arange(t0, t1), np.arange(z0, z1), np.arange(y0, y1),
                                np.arange(x0, x1), np.arange(3), indexing="ij")
    j = x + nx * (y + ny * z)
    idx = ((t * p.N + j) * 3 + c).ravel()
    (ox0, ox1), (oy0, oy1), (oz0, oz1), (ot0, ot1) = b.own
    owned = ((x >= ox0) & (x < ox1) & (y >= oy0) & (y < oy1) & (z >= oz0) & (z < oz1)
             & (t >= ot0) & (t < ot1)).ravel()
    return idx, owned


class ILU0:
    """ILU(0) of a local matrix on a given structural pattern (IKJ variant).

    For each row i in order, for each k < i in the pattern of row i (ascending):
        a_ik <- a_ik / u_kk
        a_ij <- a_ij - a_ik u_kj   for every j > k in both patterns.
    The strictly lower part is L (unit diagonal), the rest is U.
    """

    def __init__(self, Aloc: sp.csr_matrix, pattern: List[np.ndarray], rows: int | None = None):
        """rows: factor only the leading rows x rows block (its ILU(0) is the
        leading part of the full one, as row i only uses rows k < i)."""
        n = Aloc.shape[0] if rows is None else int(rows)
        Aloc = Aloc.tocsr()
        self.n = n
        self.L: List[dict] = []
        self.U: List[dict] = []
        self.diag = np.zeros(n)
        for i in range(n):
            vals = dict(zip(Aloc.indices[Aloc.indptr[i]:Aloc.indptr[i + 1]].tolist(),
                            Aloc.data[Aloc.indptr[i]:Aloc.indptr[i + 1]].tolist()))
            cols = sorted(int(c) for c in pattern[i] if c < n)
            row = {c: vals.get(c, 0.0) for c in cols}
            for k in cols:
                if k >= i:
                    break
                lik = row[k] / self.diag[k]
                row[k] = lik
                for j, ukj in self.U[k].items():
                    if j in row:
                        row[j] -= lik * ukj
            self.diag[i] = row[i]
            self.L.append({k: v for k, v in row.items() if k < i})
            self.U.append({k: v for k, v in row.items() if k > i})

    def solve(self, r: np.ndarray) -> np.ndarray:
        y = np.array(r, dtype=np.float64)
        for i in range(self.n):
            y[i] -= sum(v * y[k] for k, v in self.L[i].items())
        z = y
        for i in range(self.n - 1, -1, -1):
            z[i] = (z[i] - sum(v * z[j] for j, v in self.U[i].items())) / self.diag[i]
        return z

    def value(self, i: int, j: int) -> float:
        """Entry (i, j) of the combined factor storage (L below, U on/above)."""
        if j < i:
            return self.L[i].get(j, 0.0)
        if j == i:
            return self.diag[i]
        return self.U[i].get(j, 0.0)


def iluk_pattern(Aloc: sp.csr_matrix, pattern: List[np.ndarray], k: int) -> List[np.ndarray]:
    """Structural pattern of ILU(k) by levels of fill (Sec. 4, Table 1: ILU(k) subdomain solves).

    An entry of the given pattern has level 0.  Eliminating row i in IKJ order, each
    kept lower entry (i, m) meets each upper entry (m, j) of row m and proposes
    (i, j) with level lev(i, m) + lev(m, j) + 1; an entry is kept when its smallest
    proposed level is <= k.  Rows are processed in order, the lower entries of a
    row in ascending column order (a fill entry left of the diagonal joins the
    queue), so every lev(i, m) is final when it is used.
    """
    import heapq

    n = Aloc.shape[0]
    ulev: List[dict] = []
    out = []
    for i in range(n):
        lev = {int(c): 0 for c in pattern[i] if c < n}
        heap = [c for c in lev if c < i]
        heapq.heapify(heap)
        done = set()
        while heap:
            m = heapq.heappop(heap)
            if m in done:
                continue
            done.add(m)
            lm = lev[m]
            for j, lmj in ulev[m].items():
                nl = lm + lmj + 1
                if nl > k:
                    continue
                if j in lev:
                    if nl < lev[j]:
                        lev[j] = nl
                else:
                    lev[j] = nl
                    if j < i:
                        heapq.heappush(heap, j)
        ulev.append({j: l for j, l in lev.items() if j > i})
        out.append(np.array(sorted(lev), dtype=np.int64))
    return out


class ExactLU:
    """Exact local solve by sparse LU (scipy's SuperLU as one step)."""

    def __init__(self, Aloc: sp.csr_matrix):
        self.lu = spla.splu(Aloc.tocsc())

    def solve(self, r):
        return self.lu.solve(np.asarray(r, dtype=np.float64))


def local_pattern(p: kkt.Problem, idx: np.ndarray, rows: int | None = None) -> List[np.ndarray]:
    """Structural pattern of F_h restricted to the unknowns idx (local numbering);
    with `rows`, only the first rows rows."""
    pos = {int(g): k for k, g in enumerate(idx)}
    out = []
    for g in (idx if rows is None else idx[:rows]):
        c = int(g % 3)
        pt = int(g // 3)
        n, j = divmod(pt, p.N)
        cols = []
        for (m, k, cc) in kkt.structural_pattern_row(p, n, j, c):
            gi = (m * p.N + k) * 3 + cc
            if gi in pos:
                cols.append(pos[gi])
        out.append(np.array(sorted(cols), dtype=np.int64))
    return out


def block_pattern(p: kkt.Problem, idx: np.ndarray) -> List[np.ndarray]:
    """Pattern of the 3x3 point-block ILU(0) on the unknowns idx (local numbering).

    The point-block order (Sec. 3.2) groups the unknowns C, G, f of a space-time
    point into a 3x3 block; block (p, q) belongs to the pattern when some entry
    of F_h couples the two points, i.e. q is one of the 27 spatial neighbours of
    p at levels n-1, n, n+1.  Every entry of such a block is kept, so the
    incomplete factorisation on this pattern is the block ILU(0) whose diagonal
    blocks are factored exactly (no fill is dropped inside a block).
    """
    pos = {int(g): k for k, g in enumerate(idx)}
    out = []
    for g in idx:
        n, j = divmod(int(g // 3), p.N)
        # the f row of a point is never an identity row and reaches every point
        # its C and G rows reach (levels n-1..n+1, the 27 neighbours)
        pts = {(m, k) for (m, k, _) in kkt.structural_pattern_row(p, n, j, 2)}
        cols = []
        for (m, k) in pts:
            for cc in range(3):
                gi = (m * p.N + k) * 3 + cc
                if gi in pos:
                    cols.append(pos[gi])
        out.append(np.array(sorted(cols), dtype=np.int64))
    return out


class RAS:
    """One-level space-time restricted additive Schwarz preconditioner."""

    def __init__(self, p: kkt.Problem, F: sp.csr_matrix, nsub, overlap: int,
                 local: str = "ilu0", variant: str = "restricted"):
        self.p = p
        self.variant = variant
        self.boxes = boxes(p, nsub, overlap)
        self.idx, self.owned, self.solvers = [], [], []
        for b in self.boxes:
            idx, owned = box_unknowns(p, b)
            Aloc = F[idx][:, idx].tocsr()
            if local == "ilu0":
                solver = ILU0(Aloc, local_pattern(p, idx))
            elif local == "bilu0":   # 3x3 point-block ILU(0)
                solver = ILU0(Aloc, block_pattern(p, idx))
            elif local.startswith("ilu"):   # "ilu1", "ilu2", ...: ILU(k) on the level-k pattern
                solver = ILU0(Aloc, iluk_pattern(Aloc, local_pattern(p, idx), int(local[3:])))
            elif local == "lu":
                solver = ExactLU(Aloc)
            else:
                raise ValueError(local)
            self.idx.append(idx)
            self.owned.append(owned)
            self.solvers.append(solver)

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros(len(r))
        for idx, owned, solver in zip(self.idx, self.owned, self.solvers):
            if self.variant == "restricted":
                zl = solver.solve(r[idx])
                z[idx[owned]] = zl[owned]
            else:   # literal operand order: (R^delta)^T M^{-1} R^0
                zl = solver.solve(np.where(owned, r[idx], 0.0))
                np.add.at(z, idx, zl)
        return z


# ---------------------------------------------------------------------------
# coarse level
# ---------------------------------------------------------------------------

def _interp_1d(nf: int, nc: int) -> sp.csr_matrix:
    """Linear interpolation from nc nested coarse points to nf fine points."""
    r = (nf - 1) // (nc - 1)
    assert (nc - 1) * r == nf - 1, "meshes are not nested"
    rows, cols, vals = [], [], []
    for i in range(nf):
        I, rem = divmod(i, r)
        if rem == 0:
            rows.append(i); cols.append(I); vals.append(1.0)
        else:
            w = rem / r
            rows += [i, i]; cols += [I, I + 1]; vals += [1.0 - w, w]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def interpolation(pf: kkt.Problem, pc: kkt.Problem) -> sp.csr_matrix:
    """I^h_c: multilinear in (x, y, z, t), applied to C, G and f alike (point-block order)."""
    Px = _interp_1d(pf.nodes[0], pc.nodes[0])
    Py = _interp_1d(pf.nodes[1], pc.nodes[1])
    Pz = _interp_1d(pf.nodes[2], pc.nodes[2])
    Pt = _interp_1d(pf.L, pc.L)
    # point index = x + nx (y + ny (z + nz t)): kron order t, z, y, x, component
    P = sp.kron(Pt, sp.kron(Pz, sp.kron(Py, sp.kron(Px, sp.identity(3)))))
    return P.tocsr()


def injection(pf: kkt.Problem, pc: kkt.Problem) -> sp.csr_matrix:
    """I^c_h as injection: coarse value = fine value at the same point (Sec. 3.2)."""
    rx = (pf.nodes[0] - 1) // (pc.nodes[0] - 1)
    ry = (pf.nodes[1] - 1) // (pc.nodes[1] - 1)
    rz = (pf.nodes[2] - 1) // (pc.nodes[2] - 1)
    rt = (pf.L - 1) // (pc.L - 1)
    rows, cols = [], []
    nxc, nyc, nzc = pc.nodes
    for t in range(pc.L):
        for z in range(nzc):
            for y in range(nyc):
                for x in range(nxc):
                    jc = x + nxc * (y + nyc * z)
                    jf = rx * x + pf.nodes[0] * (ry * y + pf.nodes[1] * rz * z)
                    for c in range(3):
                        rows.append((t * pc.N + jc) * 3 + c)
                        cols.append((rt * t * pf.N + jf) * 3 + c)
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(pc.n, pf.n))


def coarse_problem(pf: kkt.Problem, ccells: Sequence[int], cM: int) -> kkt.Problem:
    """Rediscretisation on the nested coarse mesh (cell means of a and v, re-snapped sensors)."""
    rx, ry, rz = (f // c for f, c in zip(pf.cells, ccells))
    assert all(f == c * r for f, c, r in zip(pf.cells, ccells, (rx, ry, rz)))
    assert pf.M % cM == 0
    cx, cy, cz = pf.cells
    a = pf.a_cell.reshape(cz, cy, cx)
    v = pf.v_cell.reshape(cz, cy, cx, 3)
    ac = a.reshape(ccells[2], rz, ccells[1], ry, ccells[0], rx).mean(axis=(1, 3, 5)).ravel()
    vc = v.reshape(ccells[2], rz, ccells[1], ry, ccells[0], rx, 3).mean(axis=(1, 3, 5)).reshape(-1, 3)
    nxf, nyf = pf.nodes[0], pf.nodes[1]
    j = pf.sensor_node
    ix, iy, iz = j % nxf, (j // nxf) % nyf, j // (nxf * nyf)

    def snap(i, r):   # nearest coarse index, ties toward the lower one
        return (i + (r - 1) // 2) // r if r > 1 else i

    cxn = ccells[0] + 1
    cyn = ccells[1] + 1
    sc = snap(ix, rx) + cxn * (snap(iy, ry) + cyn * snap(iz, rz))
    return kkt.Problem(ccells, pf.lengths, pf.T, cM, pf.theta, pf.faces, ac, vc, sc, pf.beta1, pf.beta2, pf.reg,
                       pf.element)


class TwoLevel:
    """Multiplicative two-level hybrid space-time Schwarz preconditioner (Sec. 3.2)."""

    def __init__(self, pf: kkt.Problem, Ff: sp.csr_matrix, nsub, overlap: int,
                 ccells, cM: int, c_overlap: int = 1, c_rtol: float = 1e-1, c_maxit: int = 4,
                 local: str = "ilu0", restriction: str = "transpose"):
        self.pf, self.Ff = pf, Ff
        self.fine = RAS(pf, Ff, nsub, overlap, local)
        self.pc = coarse_problem(pf, ccells, cM)
        self.Fc = kkt.assemble(self.pc)
        self.coarse = RAS(self.pc, self.Fc, nsub, c_overlap, local)
        self.P = interpolation(pf, self.pc)
        self.R = self.P.T.tocsr() if restriction == "transpose" else injection(pf, self.pc)
        self.c_rtol, self.c_maxit = c_rtol, c_maxit

    def coarse_solve(self, rc: np.ndarray) -> np.ndarray:
        res = krylov.gmres(lambda u: self.Fc @ u, rc, self.coarse.apply, restart=max(self.c_maxit, 1),
                           rtol=self.c_rtol, maxit=self.c_maxit, flexible=False, true_residual_check=False)
        return res.x

    def apply(self, x: np.ndarray) -> np.ndarray:
        y = self.P @ self.coarse_solve(self.R @ x)
        return y + self.fine.apply(x - self.Ff @ y)
