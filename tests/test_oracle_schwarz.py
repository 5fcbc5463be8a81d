"""Pins of the oracle's Schwarz preconditioners and Krylov solvers (Sec. 3.2, 4)."""

import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import kkt, krylov, schwarz
from paper_1508_06103_gb300 import workloads as W


def _small(seed=21, cells=(3, 3, 2), M=3, faces=W.FACE_X0, element="q1"):
    w = W.random_small(seed, cells=cells, M=M, dirichlet_faces=faces, nsens=4)
    p = kkt.Problem.from_workload(dataclasses.replace(w, element=element))
    return p, kkt.assemble(p)


def test_partition_rule():
    assert schwarz.partition(33, 4) == [(0, 9), (9, 17), (17, 25), (25, 33)]
    assert schwarz.partition(65, 4) == [(0, 17), (17, 33), (33, 49), (49, 65)]
    assert schwarz.partition(5, 5) == [(k, k + 1) for k in range(5)]


def test_owned_sets_partition_the_unknowns():
    p, F = _small()
    owner = np.zeros(p.n, dtype=int)
    for b in schwarz.boxes(p, (2, 2, 1, 2), 1):
        idx, owned = schwarz.box_unknowns(p, b)
        owner[idx[owned]] += 1
        assert len(np.unique(idx)) == len(idx)
    assert np.all(owner == 1)


@pytest.mark.parametrize("element", ["q1", "p1"])
def test_ilu0_defining_property_on_pattern(element):
    """(L U)_ij = a_ij for every (i, j) in the pattern (the definition of ILU(0)).

    For P1 the structural pattern is still the 27-point cell-sharing stencil:
    the entries the Kuhn split does not couple are structural zeros."""
    p, F = _small(element=element)
    b = schwarz.boxes(p, (2, 1, 1, 2), 1)[1]
    idx, _ = schwarz.box_unknowns(p, b)
    Aloc = F[idx][:, idx].toarray()
    pat = schwarz.local_pattern(p, idx)
    ilu = schwarz.ILU0(sp.csr_matrix(Aloc), pat)
    n = len(idx)
    Lm = np.eye(n)
    Um = np.zeros((n, n))
    for i in range(n):
        for k, v in ilu.L[i].items():
            Lm[i, k] = v
        Um[i, i] = ilu.diag[i]
        for j, v in ilu.U[i].items():
            Um[i, j] = v
    LU = Lm @ Um
    mask = np.zeros((n, n), dtype=bool)
    for i, cols in enumerate(pat):
        mask[i, cols] = True
    assert np.abs((LU - Aloc)[mask]).max() < 1e-13 * np.abs(Aloc).max()
    # the factors live on the pattern only
    assert not np.any(Lm[~mask & ~np.eye(n, dtype=bool)]) and not np.any(Um[~mask])
    # every stored entry of F is inside the structural pattern
    assert not np.any(Aloc[~mask])
    # and it is not exact (the KKT pattern has fill)
    assert np.abs(LU - Aloc).max() > 1e-8 * np.abs(Aloc).max()


def test_ilu0_without_fill_is_exact_lu():
    rng = np.random.default_rng(4)
    n = 40
    A = sp.diags([rng.normal(size=n - 1), 4 + rng.random(n), rng.normal(size=n - 1)], [-1, 0, 1]).tocsr()
    pat = [np.array([j for j in (i - 1, i, i + 1) if 0 <= j < n]) for i in range(n)]
    ilu = schwarz.ILU0(A, pat)
    r = rng.normal(size=n)
    assert np.allclose(ilu.solve(r), np.linalg.solve(A.toarray(), r), rtol=1e-13, atol=1e-13)


def test_one_box_exact_lu_is_the_inverse_and_gmres_takes_one_step():
    p, F = _small(cells=(2, 2, 2), M=2)
    ras = schwarz.RAS(p, F, (1, 1, 1, 1), 0, "lu")
    r = W.random_vector(p.n, 3)
    assert np.allclose(F @ ras.apply(r), r, rtol=1e-11, atol=1e-11)
    res = krylov.gmres(lambda u: F @ u, r, ras.apply, restart=10, rtol=1e-10)
    assert res.iterations == 1 and res.converged


def test_ras_variants_agree_without_overlap():
    """With zero overlap R^delta = R^0, so both operand orders give block Jacobi."""
    p, F = _small()
    r = W.random_vector(p.n, 8)
    a = schwarz.RAS(p, F, (2, 2, 1, 2), 0, "lu").apply(r)
    b = schwarz.RAS(p, F, (2, 2, 1, 2), 0, "lu", variant="harmonic").apply(r)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-13)


def test_restricted_form_takes_owned_values_from_its_own_box_alone():
    """Pins the RAS operand order at overlap >= 1 (Sec. 3.2; the restricted form of Cai and
    Sarkis, z = sum (R^0)^T M^{-1} R^delta r).  Owned sets are disjoint, so z on box k's owned
    points is the owned part of M_k^{-1} (r on k's extended set): it must equal a dense solve of
    the principal submatrix and must not move when r changes outside the extended set.  The
    literal order (R^delta)^T M^{-1} R^0 sums, at an owned point, the solves of every box that
    overlaps it, each fed only its own owned residual, and fails both."""
    p, F = _small(cells=(4, 3, 3), M=5)
    nsub = (2, 2, 1, 2)
    ras = schwarz.RAS(p, F, nsub, 1, "lu")
    har = schwarz.RAS(p, F, nsub, 1, "lu", variant="harmonic")
    r = W.random_vector(p.n, 4)
    for k in (0, len(ras.boxes) - 1):
        idx, owned = schwarz.box_unknowns(p, ras.boxes[k])
        outside = np.ones(p.n, dtype=bool)
        outside[idx] = False
        r2 = r.copy()
        r2[outside] += W.random_vector(int(outside.sum()), 5 + k)
        zo = ras.apply(r)[idx[owned]]
        zd = np.linalg.solve(F[idx][:, idx].toarray(), r[idx])[owned]
        assert np.allclose(zo, zd, rtol=1e-9, atol=1e-12 * np.abs(zd).max())
        assert np.array_equal(zo, ras.apply(r2)[idx[owned]])
        assert not np.allclose(har.apply(r)[idx[owned]], zd, rtol=1e-3, atol=1e-3 * np.abs(zd).max())
        assert not np.allclose(har.apply(r)[idx[owned]], har.apply(r2)[idx[owned]])


def test_ras_with_overlap_is_a_better_preconditioner():
    p, F = _small(cells=(4, 3, 3), M=5)
    b = W.random_vector(p.n, 2)
    its = []
    for ov in (0, 1, 2):
        ras = schwarz.RAS(p, F, (2, 2, 2, 2), ov, "lu")
        its.append(krylov.gmres(lambda u: F @ u, b, ras.apply, restart=60, rtol=1e-8).iterations)
    assert its[0] > its[1] >= its[2], its


def test_interpolation_reproduces_multilinear_functions():
    wf = W.random_small(1, cells=(4, 2, 6), M=4)
    pf = kkt.Problem.from_workload(wf)
    pc = schwarz.coarse_problem(pf, (2, 1, 3), 2)
    P = schwarz.interpolation(pf, pc)

    def field(p):
        nx, ny, nz = p.nodes
        h = [l / c for l, c in zip(p.lengths, p.cells)]
        t, z, y, x = np.meshgrid(np.arange(p.L) * p.tau, np.arange(nz) * h[2], np.arange(ny) * h[1],
                                 np.arange(nx) * h[0], indexing="ij")
        base = (1 + 2 * x) * (3 - y) * (0.5 + z) * (2 + 5 * t)
        return np.stack([base, -base, 2 * base], axis=-1).ravel()

    assert np.allclose(P @ field(pc), field(pf), rtol=1e-13, atol=1e-13)
    # injection after interpolation is the identity on the coarse points
    Rinj = schwarz.injection(pf, pc)
    assert np.allclose((Rinj @ P).toarray(), np.eye(pc.n))
    # the transpose restriction preserves the weighted sum of each component
    u = W.random_vector(pf.n, 4)
    w = W.random_vector(pc.n, 5)
    assert abs((P @ w) @ u - w @ (P.T @ u)) < 1e-12 * np.abs(u).sum()


def test_coarse_problem_averages_and_resnaps():
    wf = W.random_small(2, cells=(4, 4, 2), M=4, nsens=5)
    pf = kkt.Problem.from_workload(wf)
    pc = schwarz.coarse_problem(pf, (2, 2, 1), 2)
    assert pc.element == "q1"
    assert schwarz.coarse_problem(kkt.Problem.from_workload(dataclasses.replace(wf, element="p1")),
                                  (2, 2, 1), 2).element == "p1"
    a = pf.a_cell.reshape(2, 4, 4)
    assert np.isclose(pc.a_cell[0], a[0:2, 0:2, 0:2].mean())
    assert np.isclose(pc.a_cell.mean(), pf.a_cell.mean())
    assert np.allclose(pc.v_cell.mean(0), pf.v_cell.mean(0))
    assert pc.s.sum() == pf.s.sum()


@pytest.mark.parametrize("element", ["q1", "p1"])
def test_two_level_with_identical_coarse_mesh_and_exact_coarse_solve_is_exact(element):
    p, F = _small(cells=(2, 2, 2), M=2, faces=W.FACE_X0, element=element)
    tl = schwarz.TwoLevel(p, F, (2, 1, 1, 1), 1, p.cells, p.M, c_overlap=0, c_rtol=1e-14,
                          c_maxit=200, local="ilu0")
    tl.coarse = schwarz.RAS(tl.pc, tl.Fc, (1, 1, 1, 1), 0, "lu")
    x = W.random_vector(p.n, 6)
    z = tl.apply(x)
    assert np.allclose(F @ z, x, rtol=1e-10, atol=1e-10 * np.abs(x).max())


# ---------------------------------------------------------------------------
# Krylov
# ---------------------------------------------------------------------------

def test_gmres_matches_dense_solve_with_restarts():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 3 + rng.normal(size=(n, n)) / np.sqrt(n)
    b = rng.normal(size=n)
    res = krylov.gmres(lambda u: A @ u, b, restart=10, rtol=1e-12, maxit=500)
    assert res.converged
    assert np.allclose(res.x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-10)


def test_gmres_terminates_in_n_steps_without_restart():
    rng = np.random.default_rng(1)
    n = 12
    A = rng.normal(size=(n, n)) + 0.1 * np.eye(n)
    b = rng.normal(size=n)
    res = krylov.gmres(lambda u: A @ u, b, restart=n, rtol=1e-10, maxit=n)
    assert res.iterations <= n and res.relres < 1e-8


def test_flexible_and_standard_gmres_agree_for_a_fixed_preconditioner():
    rng = np.random.default_rng(2)
    n = 50
    A = np.eye(n) * 2 + rng.normal(size=(n, n)) / np.sqrt(n)
    Minv = np.linalg.inv(np.diag(np.diag(A)) + np.triu(A, 1) * 0.5)
    b = rng.normal(size=n)
    r1 = krylov.gmres(lambda u: A @ u, b, lambda v: Minv @ v, restart=8, rtol=1e-10, maxit=300)
    r2 = krylov.gmres(lambda u: A @ u, b, lambda v: Minv @ v, restart=8, rtol=1e-10, maxit=300, flexible=True)
    assert r1.iterations == r2.iterations
    assert np.allclose(r1.x, r2.x, rtol=1e-8, atol=1e-9)
    # an exact preconditioner gives one step
    r3 = krylov.gmres(lambda u: A @ u, b, lambda v: np.linalg.solve(A, v), restart=8, rtol=1e-10)
    assert r3.iterations == 1


def test_box_assembly_is_the_principal_submatrix():
    p, F = _small(cells=(4, 3, 3), M=5)
    for b in schwarz.boxes(p, (2, 2, 1, 2), 1)[::3]:
        idx, _ = schwarz.box_unknowns(p, b)
        nodes, levels = schwarz.box_nodes_levels(p, b)
        Fb = kkt.assemble_box(p, nodes, levels)
        assert abs(Fb - F[idx][:, idx]).max() == 0.0


def test_partial_ilu0_is_the_leading_block_of_the_full_one():
    p, F = _small()
    b = schwarz.boxes(p, (2, 1, 1, 2), 1)[1]
    idx, _ = schwarz.box_unknowns(p, b)
    Aloc = F[idx][:, idx].tocsr()
    full = schwarz.ILU0(Aloc, schwarz.local_pattern(p, idx))
    part = schwarz.ILU0(Aloc, schwarz.local_pattern(p, idx, rows=40), rows=40)
    for i in range(40):
        assert part.L[i] == full.L[i] and part.diag[i] == full.diag[i]
        assert part.U[i] == {j: v for j, v in full.U[i].items() if j < 40}


def _laplace5(n):
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n, n))
    A = (sp.kron(sp.eye(n), T) + sp.kron(T, sp.eye(n))).tocsr()
    A.eliminate_zeros()
    return A, [A.indices[A.indptr[i]:A.indptr[i + 1]] for i in range(n * n)]


def test_iluk_levels_of_fill_on_the_five_point_laplacian():
    """Textbook levels of fill (Saad, Iterative Methods, Sec. 10.3): on an n x n grid with the
    5-point stencil, ILU(1) adds the diagonals at offsets +-(n - 1) and ILU(2) also +-(n - 2);
    each new diagonal has (n - 1)^2 entries."""
    n = 6
    A, pat = _laplace5(n)
    offsets = lambda P: sorted({int(j) - i for i, row in enumerate(P) for j in row})
    p0, p1, p2 = (schwarz.iluk_pattern(A, pat, k) for k in (0, 1, 2))
    assert offsets(p0) == [-n, -1, 0, 1, n]
    assert offsets(p1) == [-n, -(n - 1), -1, 0, 1, n - 1, n]
    assert offsets(p2) == [-n, -(n - 1), -(n - 2), -1, 0, 1, n - 2, n - 1, n]
    nnz = lambda P: sum(len(r) for r in P)
    assert nnz(p1) - nnz(p0) == 2 * (n - 1) ** 2
    assert all(set(a.tolist()) <= set(b.tolist()) for a, b in zip(p1, p2))


def test_iluk_on_a_kkt_box_has_the_ilu_property_and_reaches_exact_lu():
    p, F = _small()
    b = schwarz.boxes(p, (2, 1, 1, 2), 1)[1]
    idx, _ = schwarz.box_unknowns(p, b)
    A = F[idx][:, idx].tocsr()
    pat = schwarz.local_pattern(p, idx)
    n = len(idx)
    assert [r.tolist() for r in schwarz.iluk_pattern(A, pat, 0)] == [sorted(r.tolist()) for r in pat]
    p1 = schwarz.iluk_pattern(A, pat, 1)
    ilu = schwarz.ILU0(A, p1)
    Lm, Um = np.eye(n), np.zeros((n, n))
    for i in range(n):
        for k, v in ilu.L[i].items():
            Lm[i, k] = v
        Um[i, i] = ilu.diag[i]
        for j, v in ilu.U[i].items():
            Um[i, j] = v
    mask = np.zeros((n, n), dtype=bool)
    for i, cols in enumerate(p1):
        mask[i, cols] = True
    Ad = A.toarray()
    assert np.abs((Lm @ Um - Ad)[mask]).max() < 1e-13 * np.abs(Ad).max()
    assert sum(len(r) for r in p1) > sum(len(r) for r in pat)
    # with a level above any path length the pattern is the full fill: exact LU
    full = schwarz.ILU0(A, schwarz.iluk_pattern(A, pat, n))
    r = W.random_vector(n, 5)
    np.testing.assert_allclose(full.solve(r), np.linalg.solve(Ad, r), rtol=1e-9, atol=1e-12)


def test_higher_fill_level_needs_no_more_iterations():
    """Table 1's trend: more fill, fewer (or equal) preconditioned iterations."""
    p, F = _small(cells=(4, 3, 3), M=5)
    bvec = W.random_vector(p.n, 2)
    its = [krylov.gmres(lambda u: F @ u, bvec, schwarz.RAS(p, F, (2, 2, 2, 2), 1, loc).apply, restart=60,
                        rtol=1e-8).iterations for loc in ("ilu0", "ilu1", "lu")]
    assert its[0] >= its[1] >= its[2], its


# ---------------------------------------------------------------------------
# point-block ILU(0)
# ---------------------------------------------------------------------------

def test_block_pattern_holds_whole_blocks_of_the_81_point_neighbourhood():
    p, F = _small(cells=(3, 3, 2), M=3)
    b = schwarz.boxes(p, (1, 1, 1, 1), 0)[0]
    idx, _ = schwarz.box_unknowns(p, b)
    pat = schwarz.block_pattern(p, idx)
    scal = schwarz.local_pattern(p, idx)
    nx, ny, nz = p.nodes
    for i, g in enumerate(idx):
        n, j = divmod(int(g // 3), p.N)
        ix, iy, iz = j % nx, (j // nx) % ny, j // (nx * ny)
        cnt = 1
        for lo, hi, v in ((0, p.M, n), (0, nx - 1, ix), (0, ny - 1, iy), (0, nz - 1, iz)):
            cnt *= min(hi, v + 1) - max(lo, v - 1) + 1
        assert len(pat[i]) == 3 * cnt                            # all three components of every neighbour
        assert set(scal[i].tolist()) <= set(pat[i].tolist())     # contains the scalar pattern
        assert set((pat[i] // 3).tolist()) == set((pat[i - i % 3] // 3).tolist())   # same points for C, G, f


def test_block_ilu0_is_exact_on_boxes_of_one_spatial_node():
    """A box of one node over all levels couples point n only to n-1 and n+1: its
    block matrix is block tridiagonal, block LU makes no fill outside it, so the
    point-block ILU(0) is the exact inverse (scalar ILU(0) is not: it drops fill
    inside the blocks)."""
    p, F = _small(cells=(2, 2, 1), M=4)
    nx, ny, nz = p.nodes
    r = W.random_vector(p.n, 6)
    zb = schwarz.RAS(p, F, (nx, ny, nz, 1), 0, "bilu0").apply(r)
    zl = schwarz.RAS(p, F, (nx, ny, nz, 1), 0, "lu").apply(r)
    zs = schwarz.RAS(p, F, (nx, ny, nz, 1), 0, "ilu0").apply(r)
    np.testing.assert_allclose(zb, zl, rtol=1e-10, atol=1e-12 * np.abs(zl).max())
    assert np.abs(zs - zl).max() > 1e-6 * np.abs(zl).max()


def test_block_ilu0_has_the_ilu_property_on_its_pattern():
    p, F = _small()
    b = schwarz.boxes(p, (2, 1, 1, 2), 1)[1]
    idx, _ = schwarz.box_unknowns(p, b)
    A = F[idx][:, idx].tocsr()
    pat = schwarz.block_pattern(p, idx)
    ilu = schwarz.ILU0(A, pat)
    n = len(idx)
    Lm, Um = np.eye(n), np.zeros((n, n))
    for i in range(n):
        for k, v in ilu.L[i].items():
            Lm[i, k] = v
        Um[i, i] = ilu.diag[i]
        for j, v in ilu.U[i].items():
            Um[i, j] = v
    mask = np.zeros((n, n), dtype=bool)
    for i, cols in enumerate(pat):
        mask[i, cols] = True
    Ad = A.toarray()
    assert np.abs((Lm @ Um - Ad)[mask]).max() < 1e-13 * np.abs(Ad).max()
