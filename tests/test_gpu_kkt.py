"""GPU parity of the KKT matvec, right-hand side and source extraction against the oracle.

Tolerances (derived from the arithmetic):
* FP64 matvec: the stated bound 1e-12, applied per output as
  |y_gpu - y_ref| <= 1e-12 (|F| |x|)_i  -- each output is a sum of at most
  ~330 products, so the rounding of either side is below 330 u (|F||x|)_i
  with u = 1.1e-16, i.e. < 4e-14 (|F||x|)_i.
* FP32 matvec: (n + 3) u32 (|F||x|)_i with n ~ 330 terms, u32 = 6e-8,
  plus the rounding of x and the coefficients to FP32: bound 3e-5 (|F||x|)_i.
"""

import numpy as np
import pytest
import torch

from oracle import kkt as okkt
from paper_1508_06103_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1508_06103_gb300 import api as _api
    from paper_1508_06103_gb300 import build

    build.build()
    return _api


CASES = [
    dict(seed=1, cells=(5, 4, 3), M=6, theta=0.5, faces=W.FACE_X0 | W.FACE_Y1),
    dict(seed=2, cells=(7, 3, 5), M=5, theta=1.0, faces=W.ALL_FACES),
    dict(seed=3, cells=(1, 1, 1), M=1, theta=0.5, faces=0),
    dict(seed=4, cells=(9, 6, 4), M=9, theta=0.7, faces=W.FACE_Z0 | W.FACE_Z1),
]


def _case(c, reg="h1h1"):
    return W.random_small(c["seed"], cells=c["cells"], M=c["M"], theta=c["theta"], dirichlet_faces=c["faces"],
                          nsens=7, reg=reg)


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["cells"])) + f"x{c['M']}")
def test_matvec_fp64_matches_oracle_csr(api, case, reg):
    w = _case(case, reg)
    F = okkt.assemble(okkt.Problem.from_workload(w))
    prob = api.Problem.from_workload(w)
    assert prob.n == F.shape[0]
    for seed in (1, 2):
        # entries spread over six decades stress the per-output relative bound
        x = W.random_vector(prob.n, seed) * 10.0 ** np.random.default_rng(seed).uniform(-3, 3, prob.n)
        y = prob.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        bound = 1e-12 * (abs(F) @ np.abs(x))
        err = np.abs(y - F @ x)
        assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()


@pytest.mark.parametrize("case", CASES[:2], ids=["a", "b"])
def test_matvec_fp32_matches_oracle_within_rounding_bound(api, case):
    w = _case(case)
    F = okkt.assemble(okkt.Problem.from_workload(w))
    prob = api.Problem.from_workload(w)
    x = W.random_vector(prob.n, 3)
    y = prob.apply(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    bound = 3e-5 * (abs(F) @ np.abs(x))
    assert np.all(np.abs(y - F @ x) <= bound)


def test_residual_is_b_minus_matvec(api):
    w = _case(CASES[0])
    F = okkt.assemble(okkt.Problem.from_workload(w))
    prob = api.Problem.from_workload(w)
    x, b = W.random_vector(prob.n, 4), W.random_vector(prob.n, 5)
    r = prob.residual(torch.from_numpy(b).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    bound = 1e-12 * (abs(F) @ np.abs(x) + np.abs(b))
    assert np.all(np.abs(r - (b - F @ x)) <= bound)


def test_rhs_and_source_extraction_match_oracle(api):
    w = W.tiny(theta=0.5)
    p = okkt.Problem.from_workload(w)
    rng = np.random.default_rng(0)
    cobs = rng.normal(size=(p.L, len(p.sensor_node)))
    c0 = rng.normal(size=p.N)
    prob = api.Problem.from_workload(w)
    b = prob.rhs(torch.from_numpy(cobs).cuda(), torch.from_numpy(c0).cuda()).cpu().numpy()
    b_ref = okkt.rhs(p, cobs, c0)
    assert np.allclose(b, b_ref, rtol=1e-14, atol=1e-16)
    U = W.random_vector(prob.n, 9)
    f = prob.recover_source(torch.from_numpy(U).cuda()).cpu().numpy()
    assert np.array_equal(f, okkt.source(p, U))


def _abs_bound(p, x):
    """An upper bound of (|F| |x|)_i from the block rows with absolute spatial blocks."""
    X = np.abs(x).reshape(p.L, p.N, 3)
    C, G, f = X[:, :, 0], X[:, :, 1], X[:, :, 2]
    aB, aS, aST, aK = abs(p.B), abs(p.S), abs(p.S.T.tocsr()), abs(p.K)
    tau, M = p.tau, p.M
    Mt, Lt = abs(p.Mt).toarray(), abs(p.Lt).toarray()
    s = np.where(p.dirichlet, 0.0, p.s)
    Y = np.zeros_like(X)
    for n in range(p.L):
        m0, m1 = max(n - 1, 0), min(n + 1, M)
        yc = aB @ (C[n] + C[m0] + tau * (f[n] + f[m0])) + tau * (aS @ (C[n] + C[m0]))
        yg = aB @ (G[n] + G[m1]) + tau * (aST @ (G[n] + G[m1])) + tau * s * (C[n] + C[m1])
        Y[n, :, 0] = C[n] if n == 0 else np.where(p.dirichlet, C[n], yc)
        Y[n, :, 1] = G[n] if n == M else np.where(p.dirichlet, G[n], yg)
        acc = np.zeros(p.N)
        for m in range(max(0, n - 1), min(M, n + 1) + 1):
            acc += Mt[n, m] * (aB @ G[m]) + p.beta1 * Lt[n, m] * (aB @ f[m]) + p.beta2 * Mt[n, m] * (aK @ f[m])
        Y[n, :, 2] = acc
    return Y.reshape(-1)


def test_matvec_full_size_32cubed_x64_matches_levelwise_oracle(api):
    """Benchmark size (32^3 cells, 64 steps, 7.0M unknowns): every output checked
    against the oracle's level-wise product (the second construction of F_h)."""
    w = W.mid()
    p = okkt.Problem.from_workload(w)
    prob = api.Problem.from_workload(w)
    x = W.random_vector(prob.n, 21)
    y = prob.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref = okkt.apply(p, x)
    assert np.all(np.abs(y - y_ref) <= 1e-12 * _abs_bound(p, x))
