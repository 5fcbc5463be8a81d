"""GPU parity of the ILU(1) and 3x3 point-block ILU(0) subdomain solvers (ras_setup
local 2 and 3; Sec. 4 Table 1, Sec. 3.2) against the oracle's ILU(k) and block ILU(0).

Bars as for ILU(0) (tests/test_gpu_solve.py): both sides run the same IKJ
elimination on the same per-point pattern, so FP64 differs only by rounding
order and the reciprocal pivot: max|dz| <= 1e-9 max|z|; FP32 factors: 1e-3.
"""

import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from oracle import forward as ofwd
from oracle import kkt as okkt
from oracle import schwarz as osch
from paper_1508_06103_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1508_06103_gb300 import api as _api
    from paper_1508_06103_gb300 import build

    build.build()
    return _api


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


CASES = [
    dict(w=dict(seed=1, cells=(5, 4, 3), M=6, theta=0.5, dirichlet_faces=W.FACE_X0), nsub=(2, 2, 1, 2), ov=1),
    dict(w=dict(seed=2, cells=(4, 3, 4), M=5, theta=1.0, dirichlet_faces=W.ALL_FACES), nsub=(2, 1, 2, 2), ov=2),
]


@pytest.mark.parametrize("local", ["ilu1", "bilu0"])
@pytest.mark.parametrize("case", CASES, ids=["2x2x1x2", "2x1x2x2-ov2"])
def test_ras_apply_fp64_matches_oracle(api, case, local):
    w = W.random_small(nsens=6, **case["w"])
    p = okkt.Problem.from_workload(w)
    ref = osch.RAS(p, okkt.assemble(p), case["nsub"], case["ov"], local)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 64, local=local)
    for seed in (1, 2):
        r = W.random_vector(prob.n, seed)
        z = ras.apply(_dev(r)).cpu().numpy()
        zr = ref.apply(r)
        assert np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()


@pytest.mark.parametrize("local", ["ilu1", "bilu0"])
def test_ras_apply_fp32_close_to_oracle(api, local):
    case = CASES[0]
    w = W.random_small(nsens=6, **case["w"])
    p = okkt.Problem.from_workload(w)
    ref = osch.RAS(p, okkt.assemble(p), case["nsub"], case["ov"], local)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 32, local=local)
    r = W.random_vector(prob.n, 3)
    z = ras.apply(_dev(r)).cpu().numpy()
    zr = ref.apply(r)
    assert np.abs(z - zr).max() <= 1e-3 * np.abs(zr).max()


def test_h1l2_and_p1_with_ilu1(api):
    # the level-1 pattern is per point: the sensor couplings exist only where sensors sit
    case = CASES[0]
    w = dataclasses.replace(W.random_small(nsens=6, reg="h1l2", **case["w"]), element="p1")
    p = okkt.Problem.from_workload(w)
    ref = osch.RAS(p, okkt.assemble(p), case["nsub"], case["ov"], "ilu1")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 64, local="ilu1")
    r = W.random_vector(prob.n, 4)
    z = ras.apply(_dev(r)).cpu().numpy()
    zr = ref.apply(r)
    assert np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()


def test_fill_reduces_iterations_and_solves_match_direct(api):
    """Table 1's trend on one problem: ILU(1) and point-block ILU(0) take no more FGMRES
    iterations than ILU(0), and every local solver reaches the same solution."""
    w = W.mid(cells=(6, 6, 6), M=6, nsub=(2, 2, 2, 2), overlap=1, coarse_cells=(3, 3, 3), coarse_M=3)
    p = okkt.Problem.from_workload(w)
    F = okkt.assemble(p)
    C = ofwd.forward_march(p, w.true_source())
    cobs = ofwd.observations(p, C, w.noise(), w.noise_eps)
    U = spla.spsolve(F.tocsc(), okkt.rhs(p, cobs))
    prob = api.Problem.from_workload(w)
    b = prob.rhs(_dev(cobs))
    its = {}
    for local in ("ilu0", "ilu1", "bilu0"):
        ras = api.RAS(prob, w.nsub, w.overlap, 64, local=local)
        coarse = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.nsub, 1, 0.1, 4, 64)
        x, st, it, rel = api.gmres_solve(prob, b, ras=ras, coarse=coarse, restart=30, rtol=1e-13, maxit=3000)
        assert st == 0
        assert np.linalg.norm(x.cpu().numpy() - U) <= 1e-8 * np.linalg.norm(U)
        its[local] = it
    assert its["ilu1"] <= its["ilu0"] and its["bilu0"] <= its["ilu0"], its


def test_local_solver_arguments(api):
    w = W.random_small(nsens=6, **CASES[0]["w"])
    prob = api.Problem.from_workload(w)
    with pytest.raises(Exception):
        api.RAS(prob, CASES[0]["nsub"], 1, 16, local="ilu1")   # BF16 storage: ILU(0) only
