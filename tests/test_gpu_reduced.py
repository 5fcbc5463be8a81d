"""GPU parity of the reduced-space ("traditional") method of Sec. 1 (reduced_solve).

The reduced solve reaches the KKT solution by marching: it must return the
same U as a sparse direct solve of the assembled F_h.  Bar: relative 2-norm
error of U <= 1e-8 after the reduced system is solved to 1e-12 with step
solves to 1e-13 (the same bar as the all-at-once FP64 solve; both sides are
FP64 and the only differences are the iteration tolerances and rounding).
It must also agree with the all-at-once GPU solve of the same data.
"""

import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from oracle import forward as ofwd
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _data(w):
    p = okkt.Problem.from_workload(w)
    C = ofwd.forward_march(p, w.true_source())
    cobs = ofwd.observations(p, C, w.noise(), w.noise_eps)
    return p, cobs


CASES = {
    "mid-4x4x4x6": lambda: W.mid(cells=(4, 4, 4), M=6, coarse_cells=None, coarse_M=None),
    "mid-h1l2": lambda: dataclasses.replace(W.mid(cells=(4, 4, 4), M=6, coarse_cells=None, coarse_M=None),
                                            reg="h1l2"),
    "random-euler": lambda: W.random_small(5, cells=(5, 3, 4), M=5, theta=1.0,
                                           dirichlet_faces=W.FACE_X0 | W.FACE_Z1, nsens=6),
    "mid-p1": lambda: dataclasses.replace(W.mid(cells=(4, 4, 4), M=6, coarse_cells=None, coarse_M=None),
                                          element="p1"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_reduced_solve_matches_direct_kkt_solve(api, name):
    w = CASES[name]()
    p, cobs = _data(w)
    F = okkt.assemble(p)
    b = okkt.rhs(p, cobs)
    U = spla.spsolve(F.tocsc(), b)
    prob = api.Problem.from_workload(w)
    Ug, st, its, rel, stats = api.reduced_solve(prob, _dev(cobs), rtol=1e-12, maxit=500, step_rtol=1e-13)
    assert st == 0 and rel <= 1e-12, (st, its, rel, stats)
    Ue = Ug.cpu().numpy()
    err = np.linalg.norm(Ue - U) / np.linalg.norm(U)
    assert err <= 1e-8, err
    # the marches meet the C and G rows; the solve meets the f rows: the whole KKT residual is small
    assert np.linalg.norm(b - F @ Ue) <= 1e-9 * np.linalg.norm(b)
    # two marches per application of the reduced operator, M step solves each
    assert stats["step_solves"] == 2 * w.M * (stats["hess_applies"] + 2)


def test_reduced_and_all_at_once_gpu_solves_agree(api):
    w = W.mid(cells=(8, 8, 8), M=16, nsub=(2, 2, 2, 2), overlap=1, coarse_cells=(4, 4, 4), coarse_M=8)
    p, cobs = _data(w)
    prob = api.Problem.from_workload(w)
    c = _dev(cobs)
    Ur, st, its, rel, stats = api.reduced_solve(prob, c, rtol=1e-12, maxit=500, step_rtol=1e-13)
    assert st == 0
    ras = api.RAS(prob, w.nsub, w.overlap, 64)
    coarse = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.nsub, 1, 0.1, 4, 64)
    x, st2, its2, rel2 = api.gmres_solve(prob, prob.rhs(c), ras=ras, coarse=coarse, restart=30, rtol=1e-13,
                                         maxit=3000)
    assert st2 == 0
    fr = prob.recover_source(Ur).cpu().numpy()
    fa = prob.recover_source(x).cpu().numpy()
    assert np.linalg.norm(fr - fa) <= 1e-8 * np.linalg.norm(fa)


def test_reduced_solve_rejects_bad_arguments(api):
    w = CASES["mid-4x4x4x6"]()
    prob = api.Problem.from_workload(w)
    c = torch.zeros((w.M + 1, len(w.sensor_xyz)), dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        api.reduced_solve(prob, c, restart=0)
    with pytest.raises(Exception):
        api.reduced_solve(prob, c, step_rtol=0.0)
