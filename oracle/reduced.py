"""The reduced-space ("traditional") method of Sec. 1 as the oracle's independent KKT solve.

Test infrastructure (see the package header).

The paper contrasts its all-at-once method with the usual approach that keeps
only the source f as unknown (Sec. 1): for a given f the state C comes from a
forward march in time, the adjoint G from a backward march driven by the data
misfit, and the first-order condition of the f rows (Eq. 9, Appendix),

    W f - D G(C(f)) = b_f,    W = beta1 Lt (x) B + beta2 Mt (x) K  (or Mt (x) B, H1-L2),
                              D = Mt (x) B,

is solved for f by a Krylov method.  Each evaluation needs one sequential
forward and one backward sweep over all M time levels.  The C and G rows of
F_h are then met to the accuracy of the time-step solves, and (C, G, f) is
the KKT solution U in point-block order, the same solution as the all-at-once
solve, reached without any of its machinery (no Schwarz, no coarse level, no
space-time operator).

Steps, in the order of the method:
  1. C0 = forward march with f = 0 (the initial state c0), G0 = adjoint march
     of C0 against the observations: the affine part.
  2. H f = W f - D G_lin(C_lin(f)) with C_lin, G_lin the marches with zero
     data: the linear part; the system is H f = b_f - (W 0 - D G0) = b_f + D G0.
  3. GMRES (oracle.krylov) on H f = g, right-preconditioned by P^{-1},
     P = W + sigma Mt (x) B: the regulariser with a small mass shift (W alone
     has the constant source in its null space).  On the uniform grid B and K
     are Kronecker products of the 1D linear-element mass and stiffness
     matrices (pinned in tests/test_oracle_fem.py), so P is diagonalised by
     the 1D generalised eigenvectors (Kx u = lambda Mx u per axis, Lt v =
     lambda Mt v in time) and P^{-1} costs four dense 1D transforms each way.
     The preconditioner only changes the iteration count, not the solution.
  4. C = C0 + C_lin(f), G = adjoint march of C against the data; U = (C, G, f).

Step solves: scipy's sparse LU, or Jacobi-BiCGSTAB to a relative residual of
1e-14 per step on meshes where the LU is slow (both library routines used as
one step).

Pins: tests/test_oracle_reduced.py (agrees with a sparse direct solve of the
assembled F_h to 1e-10 on small cases with both regularisers and both time
schemes; the U it returns has a true KKT residual at the GMRES tolerance; P is
the regulariser's matrix: P applied to P^{-1} x returns x).
"""

from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import forward, krylov
from .kkt import Problem


def _mass_stiff_1d(n_cells: int, h: float):
    """Linear-element mass and stiffness matrices on n_cells uniform cells (dense)."""
    n = n_cells + 1
    Mx = np.zeros((n, n))
    Kx = np.zeros((n, n))
    for e in range(n_cells):
        i = [e, e + 1]
        Mx[np.ix_(i, i)] += h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
        Kx[np.ix_(i, i)] += 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    return Mx, Kx


class RegularisationPreconditioner:
    """x = P^{-1} y for P = beta1 Lt (x) B + beta2 Mt (x) W2 + sigma Mt (x) B, by fast diagonalisation.

    f is an (M+1, N) array with the node index j = ix + nx (iy + ny iz).
    """

    def __init__(self, p: Problem, sigma: float | None = None):
        """sigma None: 1e-3 times the regulariser's smallest non-zero eigenvalue (relative to Mt (x) B)."""
        self.shape = (p.L, p.nodes[2], p.nodes[1], p.nodes[0])
        lam_t, self.V = sla.eigh(p.Lt.toarray(), p.Mt.toarray())
        self.U, lam = [], []
        for ax in (2, 1, 0):   # z, y, x: the array axes after time
            Mx, Kx = _mass_stiff_1d(p.cells[ax], p.lengths[ax] / p.cells[ax])
            d, U = sla.eigh(Kx, Mx)
            self.U.append(U)
            lam.append(d)
        dz, dy, dx = np.meshgrid(lam[0], lam[1], lam[2], indexing="ij")
        space = (dz + dy + dx) if p.reg == "h1h1" else np.ones_like(dz)
        base = p.beta1 * lam_t[:, None, None, None] + p.beta2 * space[None]
        if sigma is None:
            sigma = 1e-3 * base[base > 1e-12 * base.max()].min()
        self.sigma = sigma
        self.diag = base + sigma

    def _transform(self, X, mats, transpose):
        for ax, A in enumerate(mats):
            X = np.moveaxis(np.tensordot(A.T if transpose else A, X, axes=([1], [ax])), 0, ax)
        return X

    def apply(self, y: np.ndarray) -> np.ndarray:
        mats = [self.V] + self.U
        X = self._transform(np.asarray(y).reshape(self.shape), mats, True)
        X = X / self.diag
        return self._transform(X, mats, False).reshape(-1)


@dataclasses.dataclass
class ReducedResult:
    U: np.ndarray            # KKT solution in point-block order
    f: np.ndarray            # (M+1, N)
    iterations: int
    converged: bool
    relres: float            # GMRES relative residual of the reduced system H f = g


class ReducedSpace:
    """The reduced system of one problem with its data (steps 1-2)."""

    def __init__(self, p: Problem, c_obs: np.ndarray, c0: np.ndarray | None = None,
                 solver: str = "lu", step_rtol: float = 1e-14):
        self.p = p
        self.c_obs = np.asarray(c_obs, dtype=np.float64)
        self.zero_obs = np.zeros_like(self.c_obs)
        self.c0 = c0
        self.state = forward.state_step(p, solver, step_rtol)
        self.adjoint = forward.adjoint_step(p, solver, step_rtol)
        self.Mt = p.Mt.toarray()
        self.Lt = p.Lt.toarray()
        zero = np.zeros((p.L, p.N))
        self.C0 = forward.forward_march(p, zero, c0, step=self.state)
        self.G0 = forward.adjoint_march(p, self.C0, self.c_obs, step=self.adjoint)
        self.evaluations = 0

    def f_rows(self, G: np.ndarray, f: np.ndarray) -> np.ndarray:
        """sum_m -Mt[n,m] B G^m + beta1 Lt[n,m] B f^m + beta2 Mt[n,m] W2 f^m, shape (M+1, N)."""
        p = self.p
        BG = (p.B @ G.T).T
        Bf = (p.B @ f.T).T
        Wf = (p.W2 @ f.T).T
        return -self.Mt @ BG + p.beta1 * (self.Lt @ Bf) + p.beta2 * (self.Mt @ Wf)

    def hess(self, fv: np.ndarray) -> np.ndarray:
        """H f: the f rows at the marched (C_lin(f), G_lin(C_lin(f)), f)."""
        p = self.p
        f = fv.reshape(p.L, p.N)
        C = forward.forward_march(p, f, None, step=self.state)
        G = forward.adjoint_march(p, C, self.zero_obs, step=self.adjoint)
        self.evaluations += 1
        return self.f_rows(G, f).reshape(-1)

    def rhs(self) -> np.ndarray:
        """g = D G0 (b_f = 0: the f rows of the right-hand side are zero, Appendix)."""
        return -self.f_rows(self.G0, np.zeros_like(self.G0)).reshape(-1)

    def assemble(self, f: np.ndarray) -> np.ndarray:
        """U = (C, G, f) in point-block order (step 4)."""
        p = self.p
        C = forward.forward_march(p, f, self.c0, step=self.state)
        G = forward.adjoint_march(p, C, self.c_obs, step=self.adjoint)
        return np.stack([C, G, f], axis=-1).reshape(-1)


def solve(p: Problem, c_obs: np.ndarray, c0: np.ndarray | None = None, rtol: float = 1e-13,
          restart: int = 400, maxit: int = 4000, sigma: float | None = None, solver: str = "lu",
          step_rtol: float = 1e-14, log=None) -> ReducedResult:
    """The KKT solution by the reduced-space method (steps 1-4)."""
    rs = ReducedSpace(p, c_obs, c0, solver, step_rtol)
    P = RegularisationPreconditioner(p, sigma)
    g = rs.rhs()

    def hess(f):
        y = rs.hess(f)
        if log is not None and rs.evaluations % 10 == 0:
            log(f"reduced-space GMRES: {rs.evaluations} march pairs")
        return y

    res = krylov.gmres(hess, g, P.apply, restart=restart, rtol=rtol, maxit=maxit)
    if log is not None:
        log(f"reduced-space GMRES: {res.iterations} iterations, relres {res.relres:.2e}, "
            f"{rs.evaluations} march pairs")
    f = res.x.reshape(p.L, p.N)
    return ReducedResult(rs.assemble(f), f, res.iterations, res.converged, res.relres)
