"""ras_apply_static: the allocation-free RAS apply, for callers that cannot call cudaMalloc.

The entry point runs the same subdomain solve as ras_apply but keeps its
scratch (the padded local vectors of the subdomains) in a fixed array inside
the library instead of the handle.  Its output must match ras_apply's within
the tolerance the RAS parity tests use (max |dz| <= 1e-9 max |z|), on two
calls in a row, and after another handle has used the shared array.  The
solve reads the array only when it keeps the local vectors in global memory,
so the handles here are built with that placement (ras_setup_shape) and are
also compared with the oracle's RAS; a handle whose vectors live in shared
memory runs without the array.
This file is named to be collected last.
"""

import numpy as np
import pytest
import torch

from oracle import kkt as okkt
from oracle import schwarz as osch
from paper_1508_06103_gb300 import workloads as W

GLOBAL_VECTORS = (0, 0, 0, 2)   # ras_setup_shape: local vectors in global memory (the scratch)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1508_06103_gb300 import api as _api
    from paper_1508_06103_gb300 import build

    build.build()
    return _api


def _close(z, zr):
    return (z - zr).abs().max().item() <= 1e-9 * zr.abs().max().item()


@pytest.mark.parametrize("prec", [64, 32])
def test_static_scratch_apply_matches_ras_apply(api, prec):
    w = W.random_small(31, cells=(6, 5, 4), M=7, dirichlet_faces=W.FACE_X0, nsens=5)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, (2, 2, 1, 2), 1, prec, shape=GLOBAL_VECTORS)
    assert ras.solve_shape()["smem_vectors"] is False
    rn = W.random_vector(prob.n, 17)
    r = torch.from_numpy(rn).cuda()
    z_ref = ras.apply(r)
    for _ in range(2):
        z = ras.apply_static(r)
        torch.cuda.synchronize()
        assert _close(z, z_ref)
    # both against the oracle's ILU(0) RAS, at the RAS parity bars
    p = okkt.Problem.from_workload(w)
    zo = osch.RAS(p, okkt.assemble(p), (2, 2, 1, 2), 1, "ilu0").apply(rn)
    zs = z.cpu().numpy()
    if prec == 64:
        assert np.abs(zs - zo).max() <= 1e-9 * np.abs(zo).max()
    else:
        assert np.linalg.norm(zs - zo) <= 1e-3 * np.linalg.norm(zo)
    # another handle, with other box shapes, writes the shared array in between
    w2 = W.random_small(32, cells=(4, 4, 4), M=5, nsens=3)
    prob2 = api.Problem.from_workload(w2)
    ras2 = api.RAS(prob2, (1, 2, 2, 1), 2, prec, shape=GLOBAL_VECTORS)
    r2 = torch.from_numpy(W.random_vector(prob2.n, 18)).cuda()
    assert _close(ras2.apply_static(r2), ras2.apply(r2))
    z = ras.apply_static(r)
    torch.cuda.synchronize()
    assert _close(z, z_ref)


def test_static_apply_with_shared_memory_vectors_needs_no_scratch(api):
    w = W.random_small(33, cells=(5, 4, 4), M=6, nsens=4)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, (2, 2, 1, 2), 1, 32, shape=(0, 0, 0, 1))
    assert ras.solve_shape()["smem_vectors"] is True
    r = torch.from_numpy(W.random_vector(prob.n, 19)).cuda()
    assert _close(ras.apply_static(r), ras.apply(r))


def test_static_scratch_rejects_handles_beyond_its_size(api):
    from paper_1508_06103_gb300._lib import KktError

    w = W.mid(cells=(16, 16, 16), M=32, coarse_cells=None, coarse_M=None)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, w.nsub, w.overlap, 64)   # local vectors ~50 MB > 32 MiB
    r = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(KktError, match="static scratch"):
        ras.apply_static(r)
