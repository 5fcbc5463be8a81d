"""Pins of the oracle's KKT system (Sec. 3.1, Eq. 8-9, Appendix) and time marching."""

import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, forward, kkt
from paper_1508_06103_gb300 import workloads as W

PI = math.pi


def _cube_problem(c, M, theta=0.5, a=0.2, v=(0.3, -0.2, 0.1), faces=W.ALL_FACES, sensors=(), beta=(1e-3, 1e-2),
                  reg="h1h1"):
    ncell = c ** 3
    return kkt.Problem((c, c, c), (1.0, 1.0, 1.0), 1.0, M, theta, faces, np.full(ncell, a),
                       np.tile(v, (ncell, 1)), np.asarray(sensors, dtype=np.int64), beta[0], beta[1], reg)


def _sxyz(xyz):
    return np.sin(PI * xyz[:, 0]) * np.sin(PI * xyz[:, 1]) * np.sin(PI * xyz[:, 2])


def _grad_sxyz(xyz):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    return PI * np.stack([np.cos(PI * x) * np.sin(PI * y) * np.sin(PI * z),
                          np.sin(PI * x) * np.cos(PI * y) * np.sin(PI * z),
                          np.sin(PI * x) * np.sin(PI * y) * np.cos(PI * z)], axis=1)


def _coords(p):
    nx, ny, nz = p.nodes
    h = [l / c for l, c in zip(p.lengths, p.cells)]
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([ix.ravel() * h[0], iy.ravel() * h[1], iz.ravel() * h[2]], axis=1)


def _forward_mms_error(c, M, theta):
    a, v = 0.2, np.array([0.3, -0.2, 0.1])
    p = _cube_problem(c, M, theta, a, v)
    xyz = _coords(p)
    S0, gS = _sxyz(xyz), _grad_sxyz(xyz)
    t = np.arange(M + 1) * p.tau
    # C = S(x) e^{-t}: f = C_t - a Lap C + v . grad C
    f = np.outer(np.exp(-t), -S0 + 3 * PI ** 2 * a * S0 + gS @ v)
    C = forward.forward_march(p, f, c0=S0)
    exact = np.outer(np.exp(-t), S0)
    return np.sqrt(np.mean((C - exact) ** 2))


GRIDS = (8, 16, 24)


def _rates(errs, grids=GRIDS):
    return [math.log(errs[i] / errs[i + 1]) / math.log(grids[i + 1] / grids[i]) for i in range(len(errs) - 1)]


def test_forward_march_converges_second_order_crank_nicolson():
    e = [_forward_mms_error(c, c, 0.5) for c in GRIDS]
    rates = _rates(e)
    assert all(1.8 < r < 2.3 for r in rates), (e, rates)


def test_forward_march_first_order_in_time_implicit_euler():
    # fixed fine space grid; error against the CN solution with a tiny step
    c = 8
    p_ref = _cube_problem(c, 256, 0.5)
    xyz = _coords(p_ref)
    S0 = _sxyz(xyz)

    def run(M, theta):
        p = _cube_problem(c, M, theta)
        f = np.zeros((M + 1, p.N))
        return forward.forward_march(p, f, c0=S0)[-1]

    ref = run(256, 0.5)
    e = [np.sqrt(np.mean((run(M, 1.0) - ref) ** 2)) for M in (16, 32, 64)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert all(0.9 < r < 1.25 for r in rates), (e, rates)


def test_adjoint_march_converges_second_order():
    a, v = 0.2, np.array([0.3, -0.2, 0.1])
    errs = []
    for c in GRIDS:
        p = _cube_problem(c, c, 0.5, a, v)
        xyz = _coords(p)
        S0, gS = _sxyz(xyz), _grad_sxyz(xyz)
        t = np.arange(c + 1) * p.tau
        # G = S(x) (1 - t): g = -G_t - a Lap G - v . grad G
        g = np.outer(np.ones_like(t), S0) + np.outer(1 - t, 3 * PI ** 2 * a * S0 - gS @ v)
        extra = np.array([p.tau * (p.B @ (0.5 * g[n] + 0.5 * g[n + 1])) for n in range(c)])
        G = forward.adjoint_march(p, np.zeros((c + 1, p.N)), np.zeros((c + 1, 0)), rhs_extra=extra)
        errs.append(np.sqrt(np.mean((G - np.outer(1 - t, S0)) ** 2)))
    rates = _rates(errs)
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)


def test_source_equation_converges_second_order():
    """f rows: W f = D G for G = -beta1 f_tt - beta2 Lap f (natural BCs, Eq. 7)."""
    b1, b2 = 0.3, 0.7
    errs = []
    for c in GRIDS:
        p = _cube_problem(c, c, 0.5, faces=0, beta=(b1, b2))
        xyz = _coords(p)
        cx = np.cos(PI * xyz[:, 0]) * np.cos(PI * xyz[:, 1]) * np.cos(PI * xyz[:, 2])
        t = np.arange(c + 1) * p.tau
        fex = np.outer(np.cos(PI * t), cx)
        G = b1 * PI ** 2 * fex + b2 * 3 * PI ** 2 * fex
        Wm = b1 * sp.kron(p.Lt, p.B) + b2 * sp.kron(p.Mt, p.K)
        Dm = sp.kron(p.Mt, p.B)
        rhs = Dm @ G.ravel()
        # W is singular with the constants as null space and rhs is consistent
        # (mean-free G): solve by CG and compare mean-free parts
        sol, info = spla.cg(Wm.tocsr(), rhs, rtol=1e-12, maxiter=20000)
        assert info == 0
        sol = sol - sol.mean()
        fex = fex - fex.mean()
        errs.append(np.sqrt(np.mean((sol - fex.ravel()) ** 2)))
    rates = _rates(errs)
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)


def test_assembly_and_levelwise_matvec_agree_and_blocks_are_tridiagonal_in_time():
    w = W.random_small(11, cells=(3, 4, 2), M=4)
    p = kkt.Problem.from_workload(w)
    F = kkt.assemble(p)
    x = W.random_vector(p.n, 5)
    assert np.abs(F @ x - kkt.apply(p, x)).max() < 1e-13 * np.abs(F).max() * np.abs(x).max() * 100
    # block (n, m) is nonzero only for |n - m| <= 1 (Sec. 3.2)
    Fc = F.tocoo()
    n_row = Fc.row // (3 * p.N)
    n_col = Fc.col // (3 * p.N)
    assert np.abs(n_row - n_col).max() == 1


def test_kkt_blocks_against_appendix_closed_forms():
    """Rows of F_h for an interior node equal the Appendix block products."""
    w = W.random_small(12, cells=(3, 3, 3), M=3, dirichlet_faces=W.FACE_X0)
    p = kkt.Problem.from_workload(w)
    F = kkt.assemble(p).toarray()
    N, tau, th = p.N, p.tau, p.theta
    B, S, K = p.B.toarray(), p.S.toarray(), p.K.toarray()
    Mt, Lt = p.Mt.toarray(), p.Lt.toarray()
    ids = lambda n, c: (n * N + np.arange(N)) * 3 + c
    D = p.dirichlet
    free = ~D
    # C row, level 2: A2 C^1 + A1 C^2 - tau/2 B f^1 - tau/2 B f^2
    r = ids(2, 0)[free]
    np.testing.assert_allclose(F[np.ix_(r, ids(1, 0))], (-B + (1 - th) * tau * S)[free], atol=1e-15)
    np.testing.assert_allclose(F[np.ix_(r, ids(2, 0))], (B + th * tau * S)[free], atol=1e-15)
    np.testing.assert_allclose(F[np.ix_(r, ids(1, 2))], (-(1 - th) * tau * B)[free], atol=1e-15)
    np.testing.assert_allclose(F[np.ix_(r, ids(2, 2))], (-th * tau * B)[free], atol=1e-15)
    # G row, level 1: B1 G^1 + B2 G^2 + tau/2 B3 (C^1 + C^2)
    r = ids(1, 1)[free]
    np.testing.assert_allclose(F[np.ix_(r, ids(1, 1))], (B + th * tau * S.T)[free], atol=1e-15)
    np.testing.assert_allclose(F[np.ix_(r, ids(2, 1))], (-B + (1 - th) * tau * S.T)[free], atol=1e-15)
    B3 = np.diag(np.where(D, 0, p.s))
    np.testing.assert_allclose(F[np.ix_(r, ids(1, 0))], ((1 - th) * tau * B3)[free], atol=1e-15)
    np.testing.assert_allclose(F[np.ix_(r, ids(2, 0))], (th * tau * B3)[free], atol=1e-15)
    # f row, level 1: -D^{1m} G^m + W^{1m} f^m
    for m in (0, 1, 2):
        np.testing.assert_allclose(F[np.ix_(ids(1, 2), ids(m, 1))], -Mt[1, m] * B, atol=1e-15)
        np.testing.assert_allclose(F[np.ix_(ids(1, 2), ids(m, 2))],
                                   p.beta1 * Lt[1, m] * B + p.beta2 * Mt[1, m] * K, atol=1e-15)
    # identity rows: C^0, G^M, Dirichlet C and G
    for rr in list(ids(0, 0)) + list(ids(p.M, 1)) + list(ids(2, 0)[D]) + list(ids(1, 1)[D]):
        row = F[rr]
        assert row[rr] == 1.0 and np.count_nonzero(row) == 1


def test_state_and_adjoint_rows_vanish_on_marched_solutions():
    """The C rows of F_h U = b hold for the forward march and the G rows for the adjoint march."""
    w = W.random_small(13, cells=(4, 3, 3), M=6, theta=0.5)
    p = kkt.Problem.from_workload(w)
    F = kkt.assemble(p)
    rng = np.random.default_rng(3)
    f = rng.normal(size=(p.L, p.N))
    c0 = rng.normal(size=p.N)
    C = forward.forward_march(p, f, c0=c0)
    cobs = rng.normal(size=(p.L, len(p.sensor_node)))
    G = forward.adjoint_march(p, C, cobs)
    U = np.stack([C, G, f], axis=2).ravel()
    r = (F @ U - kkt.rhs(p, cobs, c0)).reshape(p.L, p.N, 3)
    scale = np.abs(F).max() * np.abs(U).max()
    assert np.abs(r[:, :, 0]).max() < 1e-13 * scale
    assert np.abs(r[:, :, 1]).max() < 1e-13 * scale
    # the f rows carry W f - D G, the (approximate) reduced gradient
    assert np.abs(r[:, :, 2]).max() > 1e-6 * scale


def _objective(p, f, cobs):
    """Discrete J_h(f): trapezoid-in-time sensor misfit + 1/2 f^T W f (Eq. 2-3)."""
    C = forward.forward_march(p, f)
    keep = ~p.dirichlet[p.sensor_node]
    w = np.full(p.L, p.tau)
    w[0] = w[-1] = p.tau / 2
    mis = 0.0
    for n in range(p.L):
        d = (C[n, p.sensor_node] - cobs[n])[keep]
        mis += 0.5 * w[n] * np.sum(d * d)
    Wm = p.beta1 * sp.kron(p.Lt, p.B) + p.beta2 * sp.kron(p.Mt, p.K)
    return mis + 0.5 * f.ravel() @ (Wm @ f.ravel())


def test_kkt_gradient_matches_finite_differences_up_to_discretisation_error():
    """Optimize-then-discretize (Sec. 2): W f - D G approximates dJ_h/df; the gap shrinks with tau."""
    rng = np.random.default_rng(7)
    gaps = []
    for M in (4, 8, 16):
        ncell = 27
        sens = np.array([1 + 4 + 16, 2 + 8 + 16])      # nodes (1,1,1) and (2,2,1) of the 4^3 node grid
        p = kkt.Problem((3, 3, 3), (1.0, 1.0, 1.0), 1.0, M, 0.5, W.FACE_X0, np.full(ncell, 0.1),
                        np.tile([0.5, 0.2, 0.0], (ncell, 1)), sens, 1e-3, 1e-2)
        t = np.arange(M + 1) / M
        xyz = _coords(p)
        f = np.outer(1 + t, np.exp(-((xyz - 0.5) ** 2).sum(1)))
        cobs = np.outer(np.sin(PI * t), [0.3, 0.1])
        C = forward.forward_march(p, f)
        G = forward.adjoint_march(p, C, cobs)
        Wm = p.beta1 * sp.kron(p.Lt, p.B) + p.beta2 * sp.kron(p.Mt, p.K)
        grad_kkt = Wm @ f.ravel() - sp.kron(p.Mt, p.B) @ G.ravel()
        dirn = np.outer(np.cos(PI * t), np.exp(-((xyz - 0.3) ** 2).sum(1))).ravel()
        eps = 1e-3
        fd = (_objective(p, f + eps * dirn.reshape(f.shape), cobs)
              - _objective(p, f - eps * dirn.reshape(f.shape), cobs)) / (2 * eps)
        gaps.append(abs(fd - grad_kkt @ dirn) / abs(fd))
    # sign and scale right: the gap falls at least like tau as tau halves and ends small
    assert gaps[1] < 0.5 * gaps[0] and gaps[2] < 0.5 * gaps[1], gaps
    assert gaps[2] < 0.05, gaps


def test_finite_difference_machinery_is_exact_on_the_regulariser():
    """J_h with no sensors is the quadratic 1/2 f^T W f: central differences equal W f exactly."""
    p = _cube_problem(3, 4, 0.5, faces=W.FACE_X0, sensors=())
    rng = np.random.default_rng(9)
    f = rng.normal(size=(p.L, p.N))
    d = rng.normal(size=f.shape)
    Wm = p.beta1 * sp.kron(p.Lt, p.B) + p.beta2 * sp.kron(p.Mt, p.K)
    fd = (_objective(p, f + 1e-3 * d, np.zeros((p.L, 0))) - _objective(p, f - 1e-3 * d, np.zeros((p.L, 0)))) / 2e-3
    assert abs(fd - (Wm @ f.ravel()) @ d.ravel()) < 1e-7 * abs(fd)


def test_micro_kkt_solution_is_consistent_with_marching():
    """Sparse direct solve of F_h U = b; its C is the forward march of its f, its G the
    adjoint march of its C, and W f = D G (the reduced-space optimality condition)."""
    cells, M = (3, 3, 3), 4
    ncell = 27
    p0 = kkt.Problem(cells, (1, 1, 1), 1.0, M, 0.5, W.FACE_X0, np.full(ncell, 0.1),
                     np.tile([0.2, 0.1, 0.0], (ncell, 1)), np.array([21, 26, 42, 21]), 1e-3, 1e-1)
    xyz = _coords(p0)
    t = np.arange(M + 1) / M
    ftrue = np.outer(1 + t, np.exp(-((xyz - 0.5) ** 2).sum(1) / 0.1))
    C = forward.forward_march(p0, ftrue)
    cobs = C[:, p0.sensor_node] * (1 + 0.01 * np.cos(np.arange(4))[None, :])
    F = kkt.assemble(p0)
    b = kkt.rhs(p0, cobs)
    U = spla.spsolve(F.tocsc(), b)
    assert np.linalg.norm(F @ U - b) < 1e-12 * np.linalg.norm(b)
    X = U.reshape(p0.L, p0.N, 3)
    Cm = forward.forward_march(p0, X[:, :, 2])
    Gm = forward.adjoint_march(p0, Cm, cobs)
    assert np.abs(Cm - X[:, :, 0]).max() < 1e-10 * np.abs(Cm).max()
    assert np.abs(Gm - X[:, :, 1]).max() < 1e-10 * np.abs(Gm).max()
    Wm = p0.beta1 * sp.kron(p0.Lt, p0.B) + p0.beta2 * sp.kron(p0.Mt, p0.K)
    grad = Wm @ X[:, :, 2].ravel() - sp.kron(p0.Mt, p0.B) @ Gm.ravel()
    assert np.abs(grad).max() < 1e-10 * np.abs(Wm @ X[:, :, 2].ravel()).max()


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
def test_regulariser_rows_on_constant_source_closed_form(reg):
    """F_h applied to (C, G, f) = (0, 0, 1): the time stiffness and the spatial stiffness
    annihilate constants, so the f rows are 0 for H1-H1 (Eq. 3) and beta2 (int psi_n dt)
    (int phi_j dx) for H1-L2 (Example 2); the C rows are -tau (int phi_j dx) off the
    Dirichlet nodes for both.  The integrals of the hat functions are written out from the
    grid (h/2 at an end node, h inside), not taken from the oracle's matrices."""
    c, M = 3, 4
    p = _cube_problem(c, M, faces=W.FACE_X0, beta=(2e-3, 5e-2), reg=reg)
    h, tau = 1.0 / c, p.tau
    w1 = np.full(c + 1, h)
    w1[[0, -1]] = h / 2
    phi = np.einsum("k,j,i->kji", w1, w1, w1).ravel()      # node order x fastest
    psi = np.full(M + 1, tau)
    psi[[0, -1]] = tau / 2
    U = np.zeros(p.n)
    U[2::3] = 1.0
    y = kkt.apply(p, U).reshape(M + 1, p.N, 3)
    want_f = np.zeros((M + 1, p.N)) if reg == "h1h1" else p.beta2 * np.outer(psi, phi)
    np.testing.assert_allclose(y[:, :, 2], want_f, rtol=1e-13, atol=1e-16)
    free = ~p.dirichlet
    np.testing.assert_allclose(y[1:, free, 0], -tau * np.tile(phi[free], (M, 1)), rtol=1e-13, atol=1e-17)
    np.testing.assert_array_equal(y[:, :, 1], 0.0)


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
def test_regulariser_energy_of_a_multilinear_source_is_exact(reg):
    """f = (1+x)(1+2y)(2-z)(1+t) is its own Q1 x P1 interpolant, and the element mass and
    stiffness integrals are exact for it, so f . (F_h (0, 0, f))_f equals the regulariser
    2 N_beta(f) in closed form: beta1 int int f_t^2 + beta2 int int |grad f|^2 (H1-H1) or
    beta2 int int f^2 (H1-L2), on the unit cube over T = 1."""
    c, M = 3, 4
    p = _cube_problem(c, M, beta=(2e-3, 5e-2), reg=reg)
    xyz = _coords(p)
    x, y_, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    t = np.arange(M + 1) * p.tau
    f = np.outer(1 + t, (1 + x) * (1 + 2 * y_) * (2 - z))
    U = np.zeros(p.n)
    U[2::3] = f.ravel()
    Y = kkt.apply(p, U)[2::3]
    X2, Y2, Z2, T2 = 7 / 3, 13 / 3, 7 / 3, 7 / 3            # integrals of (1+x)^2, (1+2y)^2, (2-z)^2, (1+t)^2
    time_term = X2 * Y2 * Z2 * 1.0                           # f_t = (1+x)(1+2y)(2-z)
    if reg == "h1h1":
        space_term = (Y2 * Z2 + 4 * X2 * Z2 + X2 * Y2) * T2  # |grad f|^2 over the cube and [0, 1]
    else:
        space_term = X2 * Y2 * Z2 * T2
    want = p.beta1 * time_term + p.beta2 * space_term
    assert abs(f.ravel() @ Y - want) <= 1e-12 * want


def test_known_source_is_recovered_from_noise_free_data_at_small_beta():
    """Sensors at every node, no noise: as beta -> 0 the KKT solution's source tends to the
    true one, with an error proportional to beta (the regulariser's bias).  Implicit Euler
    (theta = 1), levels 1..M: the state sees f^n only through B f^n at n >= 1, so f^0 is
    fixed by the regulariser alone (with theta = 1/2 the time average of f over each interval
    is all the state sees, and a time checkerboard is invisible)."""
    c, M = 4, 6
    ncell = c ** 3
    xyz = None
    errs = []
    for beta in (1e-7, 1e-9):
        p = kkt.Problem((c, c, c), (1.0, 1.0, 1.0), 1.0, M, 1.0, 0, np.full(ncell, 0.1),
                        np.tile([0.3, 0.2, 0.1], (ncell, 1)), np.arange((c + 1) ** 3), beta * 1e-2, beta)
        xyz = _coords(p)
        t = np.arange(M + 1) / M
        ftrue = np.outer(1 + t, np.exp(-((xyz - 0.5) ** 2).sum(axis=1) / 0.1))
        cobs = forward.forward_march(p, ftrue)[:, p.sensor_node]
        U = spla.spsolve(kkt.assemble(p).tocsc(), kkt.rhs(p, cobs)).reshape(p.L, p.N, 3)
        errs.append(np.linalg.norm(U[1:, :, 2] - ftrue[1:]) / np.linalg.norm(ftrue[1:]))
    assert errs[1] < 1e-2, errs
    assert errs[0] / errs[1] > 30, errs


def test_adjoint_identity_between_state_and_adjoint_rows():
    """<A u, w> = <u, A^T w> to 1e-12, where A u is taken from the state rows of F_h (C rows,
    C columns) and A^T w from the adjoint rows (G rows, G columns), which the oracle assembles
    separately: G^n is the multiplier of the state equation of interval n+1 (slot (G, n)), so
    the G rows at level n give (A^T w) at level n+1.  u^0 = 0 (C^0 is fixed by the initial
    condition and has no adjoint equation); no Dirichlet nodes, so no identity rows."""
    w_ = W.random_small(5, cells=(3, 4, 2), M=5, theta=0.7, dirichlet_faces=0, nsens=5)
    p = kkt.Problem.from_workload(w_)
    F = kkt.assemble(p).tocsr()
    N, M = p.N, p.M
    ids = lambda n, c: (n * N + np.arange(N)) * 3 + c
    rng = np.random.default_rng(3)
    u = rng.standard_normal((M + 1, N))
    u[0] = 0.0
    wv = rng.standard_normal((M + 1, N))          # wv[n]: multiplier of interval n (n >= 1)
    wv[0] = 0.0
    ucol = np.zeros(p.n)
    ucol[ids(np.arange(M + 1)[:, None], 0).ravel()] = u.ravel()
    Au = F @ ucol
    lhs = sum(wv[n] @ Au[ids(n, 0)] for n in range(1, M + 1))
    gcol = np.zeros(p.n)
    for n in range(M):
        gcol[ids(n, 1)] = wv[n + 1]
    ATw = F @ gcol
    rhs = sum(u[n + 1] @ ATw[ids(n, 1)] for n in range(M))
    scale = sum(abs(wv[n]) @ abs(Au[ids(n, 0)]) for n in range(1, M + 1))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)
