"""Several independent problems solved together (ras_setup_batch, gmres_solve_batch, ras_autotune).

* The batched one-level RAS runs the boxes of all problems in one factorisation and one
  subdomain-solve launch; every box's work is the same as in the problem's own preconditioner
  with the same shape, so its apply equals the concatenation of the single-problem applies
  bit for bit.
* The batched FGMRES (all problems in lockstep, one captured graph per restart cycle, each
  problem with its own device-side rotations and stop test) matches, per problem, the sparse
  direct solution of that problem's F_h: FP64 factors, U within 1e-8 relative after a 1e-13
  solve (the bar of the single-problem solves); FP32 factors, the recovered source within 1e-5
  after a 1e-10 solve.
* A problem with a zero right-hand side stops at once with a zero solution while the others
  run; each problem reports its own iterations and true residual.
* ras_autotune returns a compiled shape and reads a cached result back for the same problems.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from oracle import forward as ofwd
from oracle import kkt as okkt
from paper_1508_06103_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NSUB = (2, 2, 1, 2)


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1508_06103_gb300 import api as _api
    from paper_1508_06103_gb300 import build

    build.build()
    return _api


def _members():
    return [W.mid(cells=(4, 4, 4), M=6, nsub=NSUB, overlap=1, coarse_cells=None, coarse_M=None),
            W.mid(cells=(5, 4, 6), M=8, nsub=NSUB, overlap=1, coarse_cells=None, coarse_M=None),
            W.mid(cells=(6, 5, 4), M=5, nsub=NSUB, overlap=1, coarse_cells=None, coarse_M=None)]


def _data(w):
    p = okkt.Problem.from_workload(w)
    C = ofwd.forward_march(p, w.true_source())
    cobs = ofwd.observations(p, C, w.noise(), w.noise_eps)
    b = okkt.rhs(p, cobs)
    return p, cobs, b, spla.spsolve(okkt.assemble(p).tocsc(), b)


@pytest.mark.parametrize("prec", [64, 32])
def test_batched_apply_equals_the_single_problem_applies(api, prec):
    ws = _members()
    probs = [api.Problem.from_workload(w) for w in ws]
    shape = (0, 2, 0, 2)   # same chunk choice and global-memory local vectors everywhere
    bras = api.BatchRAS(probs, NSUB, 1, prec, shape=shape)
    sh = bras.solve_shape()
    r = torch.from_numpy(W.random_vector(bras.n, 5)).cuda()
    z = bras.apply(r)
    for k, p in enumerate(probs):
        single = api.RAS(p, NSUB, 1, prec, shape=(sh["chunk_points"], 2, 0, 2))
        o0, o1 = bras.offsets[k], bras.offsets[k + 1]
        assert torch.equal(z[o0:o1], single.apply(r[o0:o1].contiguous()))


@pytest.mark.parametrize("prec", [64, 32])
def test_batched_solve_matches_direct_solves(api, prec):
    ws = _members()
    data = [_data(w) for w in ws]
    probs = [api.Problem.from_workload(w) for w in ws]
    bras = api.BatchRAS(probs, NSUB, 1, prec)
    b = torch.cat([p.rhs(torch.from_numpy(d[1]).cuda()) for p, d in zip(probs, data)])
    rtol = 1e-13 if prec == 64 else 1e-10
    x, st, sts, its, rel = api.gmres_solve_batch(probs, bras, b, restart=30, rtol=rtol, maxit=3000)
    assert st == 0 and all(s == 0 for s in sts) and all(r <= rtol for r in rel)
    for k, (p_ref, cobs, bh, U) in enumerate(data):
        xk = x[bras.offsets[k]:bras.offsets[k + 1]].cpu().numpy()
        assert np.allclose(b[bras.offsets[k]:bras.offsets[k + 1]].cpu().numpy(), bh, rtol=1e-14, atol=1e-18)
        if prec == 64:
            assert np.linalg.norm(xk - U) <= 1e-8 * np.linalg.norm(U)
        f, fr = okkt.source(p_ref, xk), okkt.source(p_ref, U)
        assert np.linalg.norm(f - fr) <= 1e-5 * np.linalg.norm(fr)


def test_zero_right_hand_side_stops_its_problem_alone(api):
    ws = _members()
    probs = [api.Problem.from_workload(w) for w in ws]
    bras = api.BatchRAS(probs, NSUB, 1, 64)
    b = torch.from_numpy(W.random_vector(bras.n, 9)).cuda()
    b[bras.offsets[1]:bras.offsets[2]] = 0.0
    x, st, sts, its, rel = api.gmres_solve_batch(probs, bras, b, restart=20, rtol=1e-9, maxit=2000)
    assert sts == [0, 0, 0] and its[1] == 0 and its[0] > 0 and its[2] > 0
    assert torch.count_nonzero(x[bras.offsets[1]:bras.offsets[2]]).item() == 0
    for k in (0, 2):
        o0, o1 = bras.offsets[k], bras.offsets[k + 1]
        r = probs[k].residual(b[o0:o1].contiguous(), x[o0:o1].contiguous())
        assert torch.linalg.norm(r).item() <= 1e-9 * torch.linalg.norm(b[o0:o1]).item() * 1.0001


def test_autotune_returns_a_compiled_shape_and_caches_it(api, tmp_path):
    probs = [api.Problem.from_workload(w) for w in _members()]
    cache = str(tmp_path / "tune.txt")
    shape, ms = api.autotune(probs, NSUB, 1, 32, reps=2, cache_path=cache)
    assert shape[0] in (52, 36, 20) and shape[1] in (2, 3) and shape[2] == 4 and ms > 0
    again, ms2 = api.autotune(probs, NSUB, 1, 32, reps=2, cache_path=cache)
    assert again == shape and abs(ms2 - ms) <= 1e-6 * ms
    assert len(open(cache).read().strip().splitlines()) == 1
    bras = api.BatchRAS(probs, NSUB, 1, 32, shape=shape)
    assert bras.solve_shape()["chunk_points"] == shape[0]
