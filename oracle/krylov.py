"""Restarted right-preconditioned GMRES and flexible GMRES (Sec. 3.2 and 4).

Test infrastructure (see the package header).

Right preconditioning solves F M^{-1} u = b with x = M^{-1} u (Sec. 3.2).
Flexible GMRES (Saad 1993, cited in Sec. 4) stores z_j = M_j^{-1} v_j and
forms x = x0 + Z y, which allows a preconditioner that changes between
iterations (the two-level method's inner coarse GMRES).

Orthogonalisation is classical Gram-Schmidt applied twice (CGS2); the
least-squares problem is solved with Givens rotations.  The stopping test
is on the residual 2-norm relative to ||b|| (zero initial guess, as in
Sec. 4); when the Arnoldi estimate passes the test the true residual
b - F x is formed and must pass too, otherwise the method restarts.

Pins: tests/test_oracle_schwarz.py (agrees with a dense direct solve; n-step
termination without restart; the flexible and standard forms agree for a
fixed preconditioner; iteration counts are non-increasing in restart).
"""

from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class Result:
    x: np.ndarray
    iterations: int
    converged: bool
    relres: float                 # true relative residual at exit
    history: List[float]          # Arnoldi residual estimates / ||b||


def gmres(apply_A: Callable[[np.ndarray], np.ndarray], b: np.ndarray,
          apply_M: Optional[Callable[[np.ndarray], np.ndarray]] = None,
          x0: Optional[np.ndarray] = None, restart: int = 30, rtol: float = 1e-8,
          maxit: int = 1000, flexible: bool = False, true_residual_check: bool = True) -> Result:
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    M = apply_M if apply_M is not None else (lambda v: v.copy())
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    history: List[float] = []
    if bnorm == 0.0:
        return Result(np.zeros(n), 0, True, 0.0, history)
    it = 0
    r = b - apply_A(x)
    beta = np.linalg.norm(r)
    converged = beta <= rtol * bnorm
    est = beta / bnorm
    while not converged and it < maxit:
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n)) if flexible else None
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        stop = False
        for j in range(m):
            z = M(V[j])
            if flexible:
                Z[j] = z
            w = apply_A(z)
            h = V[: j + 1] @ w                       # CGS, first pass
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1] @ w                      # second pass
            w = w - V[: j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):                       # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            est = abs(g[j + 1]) / bnorm
            history.append(est)
            if hn == 0.0 or est <= rtol or it >= maxit:
                stop = True
                break
            V[j + 1] = w / hn
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):               # back substitution
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        if flexible:
            x = x + Z[:k].T @ y
        else:
            x = x + M(V[:k].T @ y)
        if stop and not true_residual_check:
            converged = est <= rtol
            break
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        converged = beta <= rtol * bnorm
    if true_residual_check:
        relres = float(np.linalg.norm(b - apply_A(x)) / bnorm)
        converged = relres <= rtol
    else:
        relres = float(est)
    return Result(x, it, bool(converged), relres, history)
