"""Failure paths of the library, made on the host: no GPU fault, trap or hang.

* Zero pivot: a one-cell problem whose eight nodes are all Dirichlet nodes
  and whose source regularisation is switched off (beta1 = beta2 = 0).  Every
  C and G row is then an identity row and the f rows read -D G only (Appendix
  block rows), so the f diagonal of the subdomain matrix is exactly zero and
  stays zero under ILU(0): ras_setup must return KKT_ERR_ZERO_PIVOT.  (The
  oracle's ILU(0) of the same matrix divides by zero:
  tests/test_oracle_degenerate.py.)
* Krylov breakdown: on the same problem F_h (0, 0, f) = 0 exactly (every
  coefficient that multiplies f is an exact zero), so unpreconditioned GMRES
  started on b = (0, 0, f) finds h_11 = h_21 = 0 with the residual unchanged:
  gmres_solve must return KKT_BREAKDOWN, not converge and not fail.
* Bounded waits: ras_selftest_wait makes the subdomain solve's own bounded
  mbarrier wait run out on a barrier that nothing completes (50 ms); the
  kernel returns, ras_status and gmres_solve report the error word, and after
  ras_refactor the handle works again with unchanged results.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_1508_06103_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1508_06103_gb300 import api as _api
    from paper_1508_06103_gb300 import build

    build.build()
    return _api


def _all_dirichlet_unregularised(api):
    return api.Problem((1, 1, 1), (1.0, 1.0, 1.0), 3, 0.25, np.full(1, 0.1), np.array([1.0, 0.5, 0.0]),
                       np.zeros(0, dtype=np.int32), 0.0, 0.0, 0.5, W.ALL_FACES)


def test_zero_pivot_is_reported(api):
    from paper_1508_06103_gb300._lib import KktError

    prob = _all_dirichlet_unregularised(api)
    for prec in (64, 32):
        with pytest.raises(KktError) as e:
            api.RAS(prob, (1, 1, 1, 1), 0, prec)
        assert e.value.status == -5 and "pivot" in str(e.value)


def test_breakdown_is_reported(api):
    prob = _all_dirichlet_unregularised(api)
    b = prob.zeros().view(prob.levels, prob.N, 3)
    b[:, :, 2] = torch.linspace(1.0, 2.0, prob.N, dtype=torch.float64, device="cuda")
    b = b.reshape(-1)
    assert torch.count_nonzero(prob.apply(b)).item() == 0   # F (0, 0, f) = 0 exactly
    x, st, its, rel = api.gmres_solve(prob, b, restart=10, rtol=1e-8, maxit=50)
    assert st == 2 and its == 1 and rel == pytest.approx(1.0)


def test_bounded_wait_gives_up_and_the_handle_recovers(api):
    from paper_1508_06103_gb300._lib import KktError

    w = W.random_small(41, cells=(5, 4, 3), M=5, nsens=4)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, (2, 2, 1, 2), 1, 32)
    r = torch.from_numpy(W.random_vector(prob.n, 3)).cuda()
    z0 = ras.apply(r).clone()
    assert ras.status() == 0
    ras.selftest_wait(50.0)
    with pytest.raises(KktError) as e:
        ras.status()
    assert e.value.status == -3 and "gave up" in str(e.value)
    with pytest.raises(KktError):
        api.gmres_solve(prob, r, ras=ras, restart=10, rtol=1e-6, maxit=20)
    ras.refactor()
    assert ras.status() == 0
    assert torch.equal(ras.apply(r), z0)


def test_selftest_rejects_bad_limits(api):
    from paper_1508_06103_gb300 import _lib

    lib = _lib.load()
    assert lib.ras_selftest_wait(None, 10.0, None) == -1
    w = W.random_small(42, cells=(3, 3, 3), M=3, nsens=2)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, (1, 1, 1, 1), 0, 64)
    assert lib.ras_selftest_wait(ras.h, 0.0, None) == -1
    assert lib.ras_selftest_wait(ras.h, 5000.0, None) == -1
    code = ctypes.c_int(7)
    assert lib.ras_status(ras.h, ctypes.byref(code), None) == 0 and code.value == 0


def test_overlapping_spans_are_rejected(api):
    from paper_1508_06103_gb300._lib import KktError

    w = W.random_small(43, cells=(3, 3, 2), M=3, nsens=2)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, (1, 1, 1, 1), 0, 64)
    buf = torch.zeros(prob.n + 8, dtype=torch.float64, device="cuda")
    r, z = buf[: prob.n], buf[8: 8 + prob.n]   # offset views share n - 8 values
    for fn in (ras.apply, ras.apply_static):
        with pytest.raises(KktError, match="overlap"):
            fn(r, out=z)
