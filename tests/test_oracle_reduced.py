"""Pins of the reduced-space oracle solve (oracle/reduced.py, the traditional method of Sec. 1).

* The KKT solution it assembles from marches and a Krylov solve on f agrees with a sparse direct
  solve of the assembled F_h (scipy's SuperLU) to 1e-10 relative, on small problems with both
  regularisers (Eq. 3 and Sec. 4's H1-L2) and both time schemes (Crank-Nicolson, implicit Euler),
  and its true KKT residual is at the Krylov tolerance.
* Its preconditioner is the regulariser: P^{-1} from the fast diagonalisation, multiplied by the
  assembled beta1 Lt (x) B + beta2 Mt (x) W2 + sigma Mt (x) B (the oracle's quadrature-built
  matrices), returns the input.  This checks the Kronecker structure, the 1D eigenvectors and the
  axis order of the transforms, which only affect the iteration count of the solve.
"""

import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import forward, kkt, reduced
from paper_1508_06103_gb300 import workloads as W

CASES = [((4, 4, 4), 6, "h1h1", 0.5), ((5, 4, 3), 5, "h1l2", 1.0), ((3, 5, 4), 7, "h1h1", 1.0),
         ((4, 3, 5), 4, "h1l2", 0.5)]


def _case(cells, M, reg, theta):
    w = W.mid(cells=cells, M=M, coarse_cells=None, coarse_M=None)
    w = dataclasses.replace(w, reg=reg, theta=theta)
    p = kkt.Problem.from_workload(w)
    C = forward.forward_march(p, w.true_source())
    cobs = forward.observations(p, C, w.noise(), w.noise_eps)
    return p, cobs, kkt.rhs(p, cobs)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}-{c[2]}-theta{c[3]}" for c in CASES])
def test_reduced_space_solve_matches_direct_solve(case):
    p, cobs, b = _case(*case)
    F = kkt.assemble(p)
    U = spla.spsolve(F.tocsc(), b)
    r = reduced.solve(p, cobs, rtol=1e-13)
    assert r.converged
    assert np.linalg.norm(r.U - U) <= 1e-10 * np.linalg.norm(U)
    assert np.linalg.norm(b - F @ r.U) <= 1e-12 * np.linalg.norm(b)
    assert np.array_equal(r.f, kkt.source(p, r.U))


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
def test_preconditioner_inverts_the_assembled_regulariser(reg):
    p, _, _ = _case((4, 3, 5), 6, reg, 0.5)
    P = reduced.RegularisationPreconditioner(p, sigma=0.37)
    W2 = p.K if reg == "h1h1" else p.B
    A = (p.beta1 * sp.kron(p.Lt, p.B) + p.beta2 * sp.kron(p.Mt, W2) + 0.37 * sp.kron(p.Mt, p.B)).tocsr()
    x = W.random_vector(p.L * p.N, 3)
    assert np.allclose(A @ P.apply(x), x, rtol=1e-10, atol=1e-10 * np.abs(x).max())
    assert np.allclose(P.apply(A @ x), x, rtol=1e-9, atol=1e-9 * np.abs(x).max())
