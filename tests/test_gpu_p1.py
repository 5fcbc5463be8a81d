"""GPU parity of the P1 discretisation (linear tetrahedra on the Kuhn split of
every cell, Sec. 3.1) against the oracle.

The bars are those of the trilinear path (tests/test_gpu_kkt.py and
tests/test_gpu_solve.py): the FP64 matvec per output at 1e-12 (|F||x|)_i,
FP32 at 3e-5 (|F||x|)_i; the FP64 ILU(0) RAS and two-level applies at
1e-9 max|z| (same pattern, same update order, rounding only); the FP64
solve at 1e-8 relative error after rtol 1e-13 against a sparse direct
solve, the mixed solve's f at 1e-5 after rtol 1e-10.  The GPU forms the
P1 cell matrices in closed form, the oracle by inverting each tetrahedron's
vertex matrix and a 4-point rule, so the coefficients agree to rounding.
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
    dict(seed=1, cells=(5, 4, 3), M=6, theta=0.5, faces=W.FACE_X0 | W.FACE_Y1),
    dict(seed=2, cells=(7, 3, 5), M=5, theta=1.0, faces=W.ALL_FACES),
    dict(seed=3, cells=(1, 1, 1), M=1, theta=0.5, faces=0),
    dict(seed=4, cells=(9, 10, 5), M=17, theta=0.7, faces=W.FACE_Z0 | W.FACE_Z1),
]


def _case(c, reg="h1h1"):
    w = W.random_small(c["seed"], cells=c["cells"], M=c["M"], theta=c["theta"], dirichlet_faces=c["faces"],
                       nsens=7, reg=reg)
    return dataclasses.replace(w, element="p1")


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["cells"])) + f"x{c['M']}")
def test_p1_matvec_fp64_matches_oracle_csr(api, case, reg):
    w = _case(case, reg)
    F = okkt.assemble(okkt.Problem.from_workload(w))
    prob = api.Problem.from_workload(w)
    for seed in (1, 2):
        x = W.random_vector(prob.n, seed) * 10.0 ** np.random.default_rng(seed).uniform(-3, 3, prob.n)
        y = prob.apply(_dev(x)).cpu().numpy()
        bound = 1e-12 * (abs(F) @ np.abs(x))
        err = np.abs(y - F @ x)
        assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
def test_p1_matvec_fp32_matches_oracle_within_rounding_bound(api, reg):
    w = _case(CASES[3], reg)
    F = okkt.assemble(okkt.Problem.from_workload(w))
    prob = api.Problem.from_workload(w)
    x = W.random_vector(prob.n, 3)
    y = prob.apply(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    assert np.all(np.abs(y - F @ x) <= 3e-5 * (abs(F) @ np.abs(x)))


def test_element_switch_reassembles_and_switches_back(api):
    # P1 then Q1 again must give the trilinear operator exactly (a fresh Q1 handle)
    w = dataclasses.replace(_case(CASES[0]), element="q1")
    q1 = api.Problem.from_workload(w)
    sw = api.Problem.from_workload(w)
    x = _dev(W.random_vector(q1.n, 9))
    yq = q1.apply(x).cpu().numpy()
    sw.set_element("p1")
    yp = sw.apply(x).cpu().numpy()
    assert np.abs(yp - yq).max() > 1e-6 * np.abs(yq).max()
    sw.set_element("q1")
    assert np.array_equal(sw.apply(x).cpu().numpy(), yq)


RAS_CASES = [
    dict(w=dict(seed=1, cells=(5, 4, 3), M=6, theta=0.5, dirichlet_faces=W.FACE_X0), nsub=(2, 2, 1, 2), ov=1),
    dict(w=dict(seed=2, cells=(7, 3, 5), M=5, theta=1.0, dirichlet_faces=W.ALL_FACES), nsub=(3, 2, 2, 3), ov=2),
]


def _ras_workload(case, reg="h1h1"):
    return dataclasses.replace(W.random_small(nsens=6, reg=reg, **case["w"]), element="p1")


@pytest.mark.parametrize("place", [1, 2], ids=["smem", "gmem"])
@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
@pytest.mark.parametrize("case", RAS_CASES, ids=["2x2x1x2", "3x2x2x3-ov2"])
def test_p1_ras_apply_fp64_matches_oracle(api, case, reg, place):
    w = _ras_workload(case, reg)
    p = okkt.Problem.from_workload(w)
    F = okkt.assemble(p)
    ref = osch.RAS(p, F, case["nsub"], case["ov"], "ilu0")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 64, shape=(0, 0, 0, place))
    for seed in (1, 2):
        r = W.random_vector(prob.n, seed)
        z = ras.apply(_dev(r)).cpu().numpy()
        zr = ref.apply(r)
        assert np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()


def test_p1_ras_apply_fp32_close_to_oracle(api):
    case = RAS_CASES[0]
    w = _ras_workload(case)
    p = okkt.Problem.from_workload(w)
    ref = osch.RAS(p, okkt.assemble(p), case["nsub"], case["ov"], "ilu0")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, case["nsub"], case["ov"], 32)
    r = W.random_vector(prob.n, 4)
    z = ras.apply(_dev(r)).cpu().numpy()
    zr = ref.apply(r)
    assert np.abs(z - zr).max() <= 1e-3 * np.abs(zr).max()


def _two_level_case():
    w = W.mid(cells=(4, 4, 4), M=8, nsub=(2, 2, 2, 2), overlap=1, coarse_cells=(2, 2, 2), coarse_M=4)
    return dataclasses.replace(w, element="p1")


@pytest.mark.parametrize("reg", ["h1h1", "h1l2"])
def test_p1_two_level_apply_fp64_matches_oracle(api, reg):
    # the coarse level must take the fine level's element
    w = dataclasses.replace(_two_level_case(), reg=reg)
    p = okkt.Problem.from_workload(w)
    F = okkt.assemble(p)
    ref = osch.TwoLevel(p, F, w.nsub, w.overlap, w.coarse_cells, w.coarse_M, 1, 0.1, 4, "ilu0")
    prob = api.Problem.from_workload(w)
    ras = api.RAS(prob, w.nsub, w.overlap, 64)
    coarse = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.nsub, 1, 0.1, 4, 64)
    x = W.random_vector(prob.n, 5)
    z = coarse.apply(ras, _dev(x)).cpu().numpy()
    zr = ref.apply(x)
    assert np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()


@pytest.mark.parametrize("prec", [64, 32])
def test_p1_two_level_solve_matches_direct_solve(api, prec):
    w = dataclasses.replace(W.mid(cells=(6, 6, 6), M=6, nsub=(2, 2, 2, 2), overlap=1, coarse_cells=(3, 3, 3),
                                  coarse_M=3), element="p1")
    p = okkt.Problem.from_workload(w)
    F = okkt.assemble(p)
    C = ofwd.forward_march(p, w.true_source())
    cobs = ofwd.observations(p, C, w.noise(), w.noise_eps)
    b = okkt.rhs(p, cobs)
    U = spla.spsolve(F.tocsc(), b)
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


# ---------------------------------------------------------------------------
# benchmark size (32^3 cells x 64 steps, 7.0M unknowns) under P1
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def mid_p1(api):
    w = dataclasses.replace(W.mid(), element="p1")
    return w, okkt.Problem.from_workload(w), api.Problem.from_workload(w)


def test_p1_matvec_full_size_matches_levelwise_oracle(api, mid_p1):
    from test_gpu_kkt import _abs_bound   # (|F| |x|)_i from the block rows

    w, p, prob = mid_p1
    x = W.random_vector(prob.n, 22)
    y = prob.apply(_dev(x)).cpu().numpy()
    assert np.all(np.abs(y - okkt.apply(p, x)) <= 1e-12 * _abs_bound(p, x))


@pytest.mark.parametrize("prec", [64, 32])
def test_p1_fine_ras_full_size_interior_box_matches_oracle(api, mid_p1, prec):
    # the instance the benchmark's P1 form runs (local vectors in global memory, 4 lanes)
    w, p, prob = mid_p1
    r = W.random_vector(prob.n, 23)
    bxs = osch.boxes(p, w.nsub, w.overlap)
    bi = 1 + w.nsub[0] * (1 + w.nsub[1] * (1 + w.nsub[2] * 1))
    nodes, levels = osch.box_nodes_levels(p, bxs[bi])
    idx, owned = osch.box_unknowns(p, bxs[bi])
    zr = osch.ILU0(okkt.assemble_box(p, nodes, levels), osch.local_pattern(p, idx)).solve(r[idx])[owned]
    ras = api.RAS(prob, w.nsub, w.overlap, prec)
    sh = ras.solve_shape()
    assert not sh["smem_vectors"] and sh["lanes"] == 4
    z = ras.apply(_dev(r)).cpu().numpy()[idx[owned]]
    if prec == 64:
        assert np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()
    else:
        assert np.linalg.norm(z - zr) <= 1e-3 * np.linalg.norm(zr)


def test_p1_mixed_solve_full_size_true_residual(api, mid_p1):
    w, p, prob = mid_p1
    rng = np.random.default_rng(24)
    cobs = rng.standard_normal((w.M + 1, len(w.sensor_xyz)))
    ras = api.RAS(prob, w.nsub, w.overlap, 32)
    co = api.Coarse(prob, w.coarse_cells, w.coarse_M, w.nsub, w.coarse_overlap, w.coarse_rtol, w.coarse_maxit, 32)
    b = prob.rhs(_dev(cobs))
    x, st, its, rel = api.gmres_solve(prob, b, ras=ras, coarse=co, restart=w.restart, rtol=1e-8, maxit=2000)
    assert st == 0
    bo = okkt.rhs(p, cobs)
    assert np.linalg.norm(bo - okkt.apply(p, x.cpu().numpy())) <= 1e-8 * np.linalg.norm(bo)
