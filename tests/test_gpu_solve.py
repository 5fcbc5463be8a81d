"""GPU parity of the Schwarz preconditioners and the (F)GMRES solves against the oracle.

Tolerances:
* one-level RAS with exact local LU: both sides solve the box matrices
  exactly; max|dz| <= 100 cond_1(M_ij) u max|z| (largest cond_1 of the boxes,
  computed in the test; 3e5 at most on these cases).
* one-level RAS, FP64 factors: the GPU and the oracle run the same ILU(0)
  (same pattern, same IKJ update order) and the same triangular sweeps, so
  they differ only by rounding order; relative to max|z| the difference is
  bounded by (number of terms per row ~ 330) x u x (growth of the factors).
  The check is max|dz| <= 1e-9 max|z|.
* two-level apply, FP64: also runs the 4-step coarse GMRES (CGS2) on both
  sides; same bound.
* FP64 solve: the stated bound, relative 2-norm error of U <= 1e-8
  against the oracle's sparse direct solve, after solving to rtol 1e-13 (the
  KKT matrix is ill-conditioned, so a 1e-8 residual alone does not give a
  1e-8 error).
* mixed solve (FP32 or BF16-stored factors, FP64 Krylov): recovered source f
  within 1e-5 relative L2 of the oracle's direct solve, after solving to
  rtol 1e-10.
* one-level RAS, BF16-stored factors: relative 2-norm difference to the
  oracle's FP64 ILU(0) apply <= 8 u_bf16 (u = 2^-8).
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


RAS_CASES = [
    dict(w=dict(seed=1, cells=(5, 4, 3), M=6, theta=0.5, dirichlet_faces=W.FACE_X0), nsub=(2, 2, 1, 2), ov=1),
    dict(w=dict(seed=2, cells=(7, 3, 5), M=5, theta=1.0, dirichlet_faces=W.ALL_FACES), nsub=(3, 2, 2, 3), ov=2),
    dict(w=dict(seed=3, cells=(4, 4, 2), M=3, theta=0.5, dirichlet_faces=0), nsub=(1, 1, 1, 1), ov=0),
]


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
@pytest.mark.parametrize("case", RAS_CASES, ids=["2x2x1x2", "3x2x2x3-ov2", "single"])
def test_ras_apply_fp64_matches_oracle(api, case, reg):
    w = W.random_small(nsens=6, reg=reg, **case["w"])
    p = okkt.Problem.from_workload(w)
    F = okkt.assemble(p)
    ref = osch.RAS(p, F, case["nsub"], case["ov"], "ilu0")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 64)
    for seed in (1, 2):
        r = W.random_vector(prob.n, seed)
        z = ras.apply(_dev(r)).cpu().numpy()
        zr = ref.apply(r)
        assert np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
@pytest.mark.parametrize("case", RAS_CASES, ids=["2x2x1x2", "3x2x2x3-ov2", "single"])
def test_ras_apply_exact_lu_matches_oracle(api, case, reg):
    # Both sides solve the same box matrices exactly (GPU: band LU with partial
    # pivoting; oracle: sparse LU), each backward stable, so each box's
    # solution differs by at most ~cond_1(M_ij) u times a modest growth factor:
    # bar 100 cond_1 u max|z| with the largest cond_1 of the boxes.
    w = W.random_small(nsens=6, reg=reg, **case["w"])
    p = okkt.Problem.from_workload(w)
    F = okkt.assemble(p)
    ref = osch.RAS(p, F, case["nsub"], case["ov"], "lu")
    kappa = max(np.linalg.cond(F[idx][:, idx].toarray(), 1) for idx in ref.idx)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 64, local="lu")
    for seed in (1, 2):
        r = W.random_vector(prob.n, seed)
        z = ras.apply(_dev(r)).cpu().numpy()
        zr = ref.apply(r)
        assert np.abs(z - zr).max() <= 100 * kappa * 2.0**-53 * np.abs(zr).max()


def test_exact_lu_rejects_other_precisions_and_static_apply(api):
    case = RAS_CASES[0]
    w = W.random_small(nsens=6, **case["w"])
    prob = api.Problem.from_workload(w)
    with pytest.raises(Exception, match="FP64 only"):
        api.RAS(prob, case["nsub"], case["ov"], 32, local="lu")
    ras = api.RAS(prob, case["nsub"], case["ov"], 64, local="lu")
    with pytest.raises(Exception, match="ILU"):
        ras.apply_static(_dev(W.random_vector(prob.n, 1)))


# Every compiled instance of the subdomain solve, as (factor precision, lanes per point,
# placement of the local vectors: 1 shared memory, 2 global memory, chunk points or 0 = the
# library's choice), with the smallest chunk size as well (a different row stride of the
# factor blocks).  The 32^3 x 64 benchmark runs (32, 4, 2) on its fine boxes and the FP64
# form (64, 4, 2); the small boxes of these cases would otherwise always get placement 1.
INSTANCES = [(64, 4, 1, 0), (64, 4, 2, 0), (64, 4, 2, 18), (32, 4, 1, 0), (32, 4, 2, 0), (32, 4, 2, 20),
             (32, 4, 1, 36), (16, 4, 1, 0), (16, 4, 2, 0), (16, 4, 2, 40)]


def _ras_bar_ok(prec, z, zr):
    if prec == 64:
        return np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()
    if prec == 32:
        return np.linalg.norm(z - zr) <= 1e-3 * np.linalg.norm(zr)
    return np.linalg.norm(z - zr) <= 8 * 2.0**-8 * np.linalg.norm(zr)


@pytest.mark.parametrize("inst", INSTANCES, ids=[f"fp{p}-l{l}-{'smem' if v == 1 else 'gmem'}-ch{c}"
                                                for p, l, v, c in INSTANCES])
@pytest.mark.parametrize("case", RAS_CASES, ids=["2x2x1x2", "3x2x2x3-ov2", "single"])
def test_ras_apply_every_solve_instance_matches_oracle(api, case, inst):
    prec, lanes, place, ch = inst
    w = W.random_small(nsens=6, **case["w"])
    p = okkt.Problem.from_workload(w)
    ref = osch.RAS(p, okkt.assemble(p), case["nsub"], case["ov"], "ilu0")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], prec, shape=(ch, 0, lanes, place))
    sh = ras.solve_shape()
    assert sh["lanes"] == lanes and sh["smem_vectors"] == (place == 1)
    assert ch == 0 or sh["chunk_points"] == ch
    for seed in (1, 2):
        r = W.random_vector(prob.n, seed)
        z = ras.apply(_dev(r)).cpu().numpy()
        assert _ras_bar_ok(prec, z, ref.apply(r))


def test_setup_shape_rejects_shapes_that_do_not_exist(api):
    from paper_1508_06103_gb300._lib import KktError

    case = RAS_CASES[0]
    prob = api.Problem.from_workload(W.random_small(nsens=6, **case["w"]))
    for prec, shape in ((64, (0, 0, 8, 0)), (32, (33, 0, 0, 0)), (16, (0, 5, 0, 0)), (32, (0, 0, 0, 3)),
                        (32, (28, 0, 0, 0))):
        with pytest.raises(KktError):
            api.RAS(prob, case["nsub"], case["ov"], prec, shape=shape)


def test_solve_shape_is_reported_and_valid(api):
    # the chunk size, copy-ring depth and vector placement chosen at set-up
    case = RAS_CASES[1]
    w = W.random_small(nsens=6, **case["w"])
    prob = api.Problem.from_workload(w)
    for prec, sizes in ((64, {34, 26, 18}), (32, {52, 36, 20}), (16, {72, 40, 8})):
        sh = api.RAS(prob, case["nsub"], case["ov"], prec).solve_shape()
        assert sh["chunk_points"] in sizes and 2 <= sh["stages"] <= 4 and isinstance(sh["smem_vectors"], bool)
        assert sh["lanes"] == 4


def test_ras_apply_fp32_close_to_oracle(api):
    case = RAS_CASES[0]
    w = W.random_small(nsens=6, **case["w"])
    p = okkt.Problem.from_workload(w)
    ref = osch.RAS(p, okkt.assemble(p), case["nsub"], case["ov"], "ilu0")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 32)
    r = W.random_vector(prob.n, 3)
    zr = ref.apply(r)
    z = ras.apply(_dev(r)).cpu().numpy()
    assert np.linalg.norm(z - zr) <= 1e-3 * np.linalg.norm(zr)


def test_ras_apply_bf16_close_to_oracle(api):
    # BF16 keeps 8 significant bits (unit roundoff u = 2^-8 = 3.9e-3); the
    # factors are rounded once after an FP32 factorisation and the sweeps
    # accumulate in FP32, so the preconditioned vector moves by a few u
    case = RAS_CASES[0]
    w = W.random_small(nsens=6, **case["w"])
    p = okkt.Problem.from_workload(w)
    ref = osch.RAS(p, okkt.assemble(p), case["nsub"], case["ov"], "ilu0")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 16)
    assert ras.info()["value_bytes"] == 2
    for seed in (3, 4):
        r = W.random_vector(prob.n, seed)
        zr = ref.apply(r)
        z = ras.apply(_dev(r)).cpu().numpy()
        assert np.linalg.norm(z - zr) <= 8 * 2.0**-8 * np.linalg.norm(zr)


def _two_level_case():
    return W.mid(cells=(4, 4, 4), M=8, nsub=(2, 2, 2, 2), overlap=1, coarse_cells=(2, 2, 2), coarse_M=4)


@pytest.mark.parametrize("place", [0, 1, 2], ids=["auto", "fine-smem", "fine-gmem"])
@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
def test_two_level_apply_fp64_matches_oracle(api, reg, place):
    # under H1-L2 this also checks that the coarse level takes the fine level's regularisation;
    # `place` forces the fine subdomain solve's local vectors into shared or global memory
    w = dataclasses.replace(_two_level_case(), reg=reg)
    p = okkt.Problem.from_workload(w)
    F = okkt.assemble(p)
    ref = osch.TwoLevel(p, F, w.nsub, w.overlap, w.coarse_cells, w.coarse_M, 1, 0.1, 4, "ilu0")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, w.nsub, w.overlap, 64, shape=None if place == 0 else (0, 0, 0, place))
    coarse = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.nsub, 1, 0.1, 4, 64)
    x = W.random_vector(prob.n, 5)
    z = coarse.apply(ras, _dev(x)).cpu().numpy()
    zr = ref.apply(x)
    assert np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()


def test_two_level_refactor_equals_separate_refactors(api):
    # the combined call runs the same factorisations, only on two streams
    w = _two_level_case()
    prob = api.Problem.from_workload(w)
    x = _dev(W.random_vector(prob.n, 7))
    outs = []
    for together in (False, True):
        ras = api.RAS(prob, w.nsub, w.overlap, 32)
        coarse = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.nsub, 1, 0.1, 4, 32)
        if together:
            coarse.refactor_with(ras)
        else:
            ras.refactor()
            coarse.refactor()
        outs.append(coarse.apply(ras, x).cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def _exact(w):
    p = okkt.Problem.from_workload(w)
    F = okkt.assemble(p)
    C = ofwd.forward_march(p, w.true_source())
    cobs = ofwd.observations(p, C, w.noise(), w.noise_eps)
    b = okkt.rhs(p, cobs)
    return p, F, cobs, b, spla.spsolve(F.tocsc(), b)


def test_one_level_fp64_solve_matches_direct_solve(api):
    w = W.mid(cells=(4, 4, 4), M=6, nsub=(2, 2, 1, 2), overlap=1, coarse_cells=None, coarse_M=None)
    p, F, cobs, b, U = _exact(w)
    prob = api.Problem.from_workload(w)
    bd = prob.rhs(_dev(cobs))
    assert np.allclose(bd.cpu().numpy(), b, rtol=1e-14, atol=1e-18)
    ras = api.RAS(prob, w.nsub, w.overlap, 64)
    x, st, its, rel = api.gmres_solve(prob, bd, ras=ras, restart=30, rtol=1e-13, maxit=2000)
    assert st == 0 and rel <= 1e-13
    xe = x.cpu().numpy()
    assert np.linalg.norm(xe - U) <= 1e-8 * np.linalg.norm(U)
    assert np.linalg.norm(b - F @ xe) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("prec", [64, 32, 16])
def test_two_level_solve_matches_direct_solve(api, prec):
    w = W.mid(cells=(6, 6, 6), M=6, nsub=(2, 2, 2, 2), overlap=1, coarse_cells=(3, 3, 3), coarse_M=3)
    p, F, cobs, b, U = _exact(w)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, w.nsub, w.overlap, prec)
    coarse = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.nsub, 1, 0.1, 4, prec)
    bd = prob.rhs(_dev(cobs))
    rtol = 1e-13 if prec == 64 else 1e-10
    x, st, its, rel = api.gmres_solve(prob, bd, ras=ras, coarse=coarse, restart=30, rtol=rtol, maxit=3000)
    assert st == 0 and rel <= rtol
    xe = x.cpu().numpy()
    if prec == 64:
        assert np.linalg.norm(xe - U) <= 1e-8 * np.linalg.norm(U)
    f = prob.recover_source(x).cpu().numpy()
    fr = okkt.source(p, U)
    assert np.linalg.norm(f - fr) <= 1e-5 * np.linalg.norm(fr)


def test_zero_rhs_gives_zero_solution_and_nan_is_reported(api):
    w = W.random_small(7, cells=(3, 3, 3), M=3)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, (1, 1, 1, 1), 0, 64)
    b = prob.zeros()
    x, st, its, rel = api.gmres_solve(prob, b, ras=ras)
    assert st == 0 and its == 0 and torch.count_nonzero(x).item() == 0
    b[5] = float("nan")
    from paper_1508_06103_gb300._lib import KktError
    with pytest.raises(KktError):
        api.gmres_solve(prob, b, ras=ras)


def test_maxit_exhaustion_reports_not_converged(api):
    w = W.random_small(8, cells=(4, 3, 3), M=4)
    prob = api.Problem.from_workload(w)
    b = _dev(W.random_vector(prob.n, 1))
    x, st, its, rel = api.gmres_solve(prob, b, restart=5, rtol=1e-12, maxit=7)
    assert st == 1 and its == 7 and rel > 1e-12


def test_captured_cycle_timing_launch_count_and_replay_determinism(api):
    # the outer FGMRES cycle is captured into a CUDA graph on the first solve and replayed;
    # the per-launch CUDA-event timing and the launch count go through the replays, and a
    # replay gives the first solve's result bit for bit
    w = W.mid(cells=(6, 6, 6), M=6, nsub=(2, 2, 2, 2), overlap=1, coarse_cells=(3, 3, 3), coarse_M=3)
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, w.nsub, w.overlap, 32)
    coarse = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.nsub, 1, 0.1, 4, 32)
    b = _dev(W.random_vector(prob.n, 13))
    xs = []
    api.timing_enable(True)
    try:
        for rep in range(3):
            api.timing_reset(prob, ras)
            n0 = api.launch_count()
            x, st, its, rel = api.gmres_solve(prob, b, ras=ras, coarse=coarse, restart=30, rtol=1e-10, maxit=300)
            assert st == 0 and rel <= 1e-10
            mv_ms, mv_n = api.matvec_timing(prob)
            rs_ms, rs_n = ras.timing(0)
            assert mv_n >= its + 1 and mv_ms > 0      # one matvec per step, one per true residual
            assert rs_n >= its and rs_ms > 0          # one fine subdomain solve per step
            assert api.launch_count() - n0 > 10 * its
            xs.append(x.clone())
    finally:
        api.timing_enable(False)
    assert torch.equal(xs[0], xs[1]) and torch.equal(xs[1], xs[2])
