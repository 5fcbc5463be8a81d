"""Degenerate KKT systems that the GPU failure tests build on the host (no GPU needed).

A one-cell grid whose eight nodes all lie on Dirichlet faces, with beta1 = beta2 = 0: every C and
G row of F_h is an identity row (Dirichlet nodes, Appendix) and the f rows are -D G with W = 0
(Eq. 9 with no regularisation).  So
* F_h (0, 0, f) = 0 exactly for every f (each product that meets f has an exact zero factor), and
* the f diagonal of every f row is zero, and the first f row of the box (point 0, level 0) meets
  an exactly zero pivot under ILU(0) in point-block order: its L part holds only the own-point G
  column, whose pivot row (an identity row) has no f column, so nothing updates the diagonal.
  Later f rows divide by that zero, so their pivots are not finite.
The GPU tests (tests/test_gpu_failures.py) expect KKT_BREAKDOWN from GMRES on b = (0, 0, f) and
KKT_ERR_ZERO_PIVOT from the subdomain factorisation of this matrix.
"""

import numpy as np

from oracle import kkt, schwarz


def _problem():
    return kkt.Problem((1, 1, 1), (1.0, 1.0, 1.0), 0.75, 3, 0.5, 63, np.full(1, 0.1),
                       np.array([[1.0, 0.5, 0.0]]), np.zeros(0, dtype=np.int64), 0.0, 0.0)


def test_every_node_is_dirichlet_and_f_columns_are_a_null_space():
    p = _problem()
    assert p.dirichlet.all()
    F = kkt.assemble(p)
    x = np.zeros((p.L, p.N, 3))
    x[:, :, 2] = np.linspace(1.0, 2.0, p.N)
    y = F @ x.reshape(-1)
    assert np.count_nonzero(y) == 0
    assert np.count_nonzero(kkt.apply(p, x.reshape(-1))) == 0


def test_f_diagonal_is_zero_and_ilu0_meets_a_zero_pivot():
    p = _problem()
    F = kkt.assemble(p).tocsr()
    d = F.diagonal().reshape(p.L, p.N, 3)
    assert np.all(d[:, :, 2] == 0.0) and np.all(d[:, :, :2] == 1.0)
    b = schwarz.boxes(p, (1, 1, 1, 1), 0)[0]
    idx, _ = schwarz.box_unknowns(p, b)
    with np.errstate(all="ignore"):
        ilu = schwarz.ILU0(F[idx][:, idx].tocsr(), schwarz.local_pattern(p, idx))
    piv = ilu.diag.reshape(p.L, p.N, 3)
    assert piv[0, 0, 2] == 0.0 and np.all(piv[:, :, :2] == 1.0)
    assert not np.isfinite(piv[:, :, 2].ravel()[1:]).any()
