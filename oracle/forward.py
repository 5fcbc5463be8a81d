"""Time marching of the state and adjoint equations (Eq. 8; Sec. 1 reduced-space steps).

Test infrastructure (see the package header).

forward_march : C^0 = C_0, then for n = 1..M solve
                (B + theta tau S) C^n = (B - (1-theta) tau S) C^{n-1}
                                        + tau B ((1-theta) f^{n-1} + theta f^n)
                with C = 0 on the Dirichlet nodes (p = 0).
adjoint_march : G^M = 0, then for n = M-1..0 solve
                (B + theta tau S^T) G^n = (B - (1-theta) tau S^T) G^{n+1}
                                          - tau B3 ((1-theta) (C^n - Ceps^n)
                                                    + theta (C^{n+1} - Ceps^{n+1}))
                with G = 0 on the Dirichlet nodes.
observations  : C at the sensor nodes with multiplicative noise
                C^eps = C + eps r C (Sec. 4), r passed in.
observations_refined : the same from a forward solve on a mesh `refine`
                times finer in space and time (Sec. 4 generates the data "on a
                very fine mesh with a small time step"), sampled at the coarse
                levels 0, refine, 2 refine, ...

The linear solves use scipy's sparse LU (a library routine as one step); on
meshes whose LU fill is too large, Jacobi-preconditioned BiCGSTAB to a relative
residual of 1e-13 per step instead.

Pins: tests/test_oracle_kkt.py (manufactured-solution convergence orders in
h and tau; the marched (C, f) pair zeroes the C rows of F_h; the marched
adjoint zeroes the G rows) and tests/test_oracle_data.py (refining by 1 gives the
same-mesh data; refined data converge at second order).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .kkt import Problem


def _dirichlet_rows(Mat: sp.csr_matrix, D: np.ndarray) -> sp.csr_matrix:
    keep = sp.diags((~D).astype(np.float64))
    return (keep @ Mat + sp.diags(D.astype(np.float64))).tocsc()


def _step_solver(A: sp.csc_matrix, solver: str, rtol: float):
    """x = A^{-1} r: sparse LU, or (for meshes whose LU fill is too large) Jacobi-preconditioned
    BiCGSTAB to relative residual rtol, started from the previous step; where BiCGSTAB breaks
    down (it can on the layered, 100x-contrast diffusivity), Jacobi-preconditioned GMRES(30)
    from the same start instead.  All are library routines used as one step."""
    if solver == "lu":
        lu = spla.splu(A)
        return lambda r, x0: lu.solve(r)
    if solver != "bicgstab":
        raise ValueError(solver)
    A = A.tocsr()
    dinv = 1.0 / A.diagonal()
    M = spla.LinearOperator(A.shape, matvec=lambda v: dinv * v)

    def solve(r, x0):
        if not np.any(r):
            return np.zeros_like(r)
        x, info = spla.bicgstab(A, r, x0=x0, rtol=rtol, atol=0.0, M=M, maxiter=5000)
        if info != 0:
            x, info = spla.gmres(A, r, x0=x0, rtol=rtol, atol=0.0, M=M, restart=30, maxiter=500)
        if info != 0:
            raise RuntimeError(f"the step solve did not reach rtol {rtol} (info {info})")
        return x
    return solve


def state_step(p: Problem, solver: str = "lu", rtol: float = 1e-13):
    """x = (B + theta tau S)^{-1} r with identity rows at the Dirichlet nodes (one state step)."""
    return _step_solver(_dirichlet_rows(p.B + p.theta * p.tau * p.S, p.dirichlet), solver, rtol)


def adjoint_step(p: Problem, solver: str = "lu", rtol: float = 1e-13):
    """x = (B + theta tau S^T)^{-1} r with identity rows at the Dirichlet nodes (one adjoint step)."""
    return _step_solver(_dirichlet_rows(p.B + p.theta * p.tau * p.S.T.tocsr(), p.dirichlet), solver, rtol)


def forward_march(p: Problem, f: np.ndarray, c0: np.ndarray | None = None,
                  rhs_extra: np.ndarray | None = None, solver: str = "lu", rtol: float = 1e-13,
                  step=None) -> np.ndarray:
    """State C^0..C^M (shape (M+1, N)) for nodal source values f (shape (M+1, N)).

    rhs_extra[n] (n >= 1), if given, is added to the right-hand side of step n
    (used by the manufactured-solution tests).  solver "lu" (default) or
    "bicgstab" (to relative residual rtol per step); `step` (from state_step)
    reuses a step solver built once.
    """
    th, tau, D = p.theta, p.tau, p.dirichlet
    solve = step if step is not None else state_step(p, solver, rtol)
    R = (p.B - (1.0 - th) * tau * p.S).tocsr()
    C = np.zeros((p.L, p.N))
    if c0 is not None:
        C[0] = c0
    C[0, D] = 0.0
    for n in range(1, p.L):
        r = R @ C[n - 1] + tau * (p.B @ ((1.0 - th) * f[n - 1] + th * f[n]))
        if rhs_extra is not None:
            r = r + rhs_extra[n]
        r[D] = 0.0
        C[n] = solve(r, C[n - 1])
    return C


def adjoint_march(p: Problem, C: np.ndarray, c_obs: np.ndarray,
                  rhs_extra: np.ndarray | None = None, step=None) -> np.ndarray:
    """Adjoint G^0..G^M for state C (M+1, N) and observations c_obs (M+1, s); `step`
    (from adjoint_step) reuses a step solver built once (sparse LU by default)."""
    th, tau, D = p.theta, p.tau, p.dirichlet
    St = p.S.T.tocsr()
    solve = step if step is not None else adjoint_step(p)
    R = (p.B - (1.0 - th) * tau * St).tocsr()
    s = np.where(D, 0.0, p.s)
    G = np.zeros((p.L, p.N))
    for n in range(p.M - 1, -1, -1):
        mis = np.zeros((2, p.N))
        for q, m in enumerate((n, n + 1)):
            obs = np.zeros(p.N)
            np.add.at(obs, p.sensor_node, c_obs[m])
            mis[q] = s * C[m] - np.where(D, 0.0, obs)
        r = R @ G[n + 1] - tau * ((1.0 - th) * mis[0] + th * mis[1])
        if rhs_extra is not None:
            r = r + rhs_extra[n]
        r[D] = 0.0
        G[n] = solve(r, G[n + 1])
    return G


def observations(p: Problem, C: np.ndarray, r: np.ndarray, eps: float) -> np.ndarray:
    """C^eps at the sensors, shape (M+1, s): C + eps r C (Sec. 4)."""
    Cs = C[:, p.sensor_node]
    return Cs + eps * r * Cs


def observations_refined(p_fine: Problem, f_fine: np.ndarray, refine: int, r: np.ndarray,
                         eps: float, solver: str = "lu") -> np.ndarray:
    """C^eps at the sensors of p_fine on every refine-th level, shape (M_fine/refine + 1, s).

    p_fine is the problem on the refined mesh (its sensors at nodes of the coarse
    mesh), f_fine the true source at its nodes and levels, r the noise draws of
    the coarse samples.
    """
    if p_fine.M % refine:
        raise ValueError("the fine level count must be a multiple of the refinement")
    C = forward_march(p_fine, f_fine, solver=solver)
    Cs = C[::refine, p_fine.sensor_node]
    return Cs + eps * r * Cs
