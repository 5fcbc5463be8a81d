"""The 64^3 x 128 single solve (106,279,875 unknowns): FP32 subdomain and coarse solves inside FP64
FGMRES(40), two-level RAS with 8^4 subdomains, overlap 2, coarse 16^3 x 32.

Checked by what the oracle evaluates at this size: the right-hand side from the observations
(relative 1e-14, as in the small cases) and the true relative residual of the GPU solution,
||b - F_h U|| / ||b|| <= 1e-8 with the oracle's level-wise F_h (the stop test of the solve).
The layered diffusivity with a 100x contrast and the rotating velocity are the workload's own.
"""

import os

import numpy as np
import pytest
import torch

from oracle import kkt as okkt
from paper_1508_06103_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OBS = os.path.join(ROOT, "tests", "golden", "observations_large_64x64x64x128.txt")


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1508_06103_gb300 import api as _api
    from paper_1508_06103_gb300 import build

    build.build()
    return _api


def test_large_two_level_solve_true_residual(api):
    w = W.large()
    cobs = np.loadtxt(OBS, ndmin=2)
    prob = api.Problem.from_workload(w)
    assert prob.n == 106279875   # 65^3 nodes x 129 levels x 3
    ras = api.RAS(prob, w.nsub, w.overlap, 32)
    co = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.coarse_split, w.coarse_overlap, w.coarse_rtol,
                    w.coarse_maxit, 32)
    bd = prob.rhs(torch.from_numpy(cobs).cuda())
    x, st, its, rel = api.gmres_solve(prob, bd, ras=ras, coarse=co, restart=w.restart, rtol=w.rtol, maxit=2000)
    assert st == 0 and rel <= 1e-8
    xh = x.cpu().numpy()
    bh = bd.cpu().numpy()
    del x, bd, ras, co
    torch.cuda.empty_cache()
    p = okkt.Problem.from_workload(w)
    b = okkt.rhs(p, cobs)
    assert np.allclose(bh, b, rtol=1e-14, atol=1e-18)
    r = b - okkt.apply(p, xh)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b)
