"""The paper's Examples 1-3 (Sec. 4.1) as synthetic workloads: sizes, boundary parts and
parameters as printed, and the source formulas checked at points worked out by hand."""

import math

import numpy as np

from oracle import forward, kkt
from paper_1508_06103_gb300 import workloads as W

GAMMA1 = W.FACE_X0 | W.FACE_X1 | W.FACE_Y0 | W.FACE_Y1    # |x| = 2 or |y| = 2


def test_example1_setup_and_source_at_t0():
    w = W.example1()
    assert w.cells == (40, 40, 40) and w.M == 39 and w.lengths == (4.0, 4.0, 4.0)
    assert len(w.sensor_xyz) == 14 ** 3 and (w.beta1, w.beta2) == (3.6e-5, 3.6e-3)
    assert w.dirichlet_faces == GAMMA1 and w.theta == 0.5 and w.nsub == (4, 4, 4, 4)
    # t = 0: centres (0, 2, 2) and (-2, 2, -2) in (-2, 2)^3, i.e. (2, 4, 4) and (0, 4, 0) here;
    # at the first centre f = 1 + exp(-|(2, 0, 4)|^2 / a^2) = 1 + exp(-20 / 4)
    f0 = w.true_source()[0]
    j = 20 + 41 * (40 + 41 * 40)                            # node (2.0, 4.0, 4.0), h = 0.1
    np.testing.assert_allclose(w.node_coords()[j], (2.0, 4.0, 4.0), atol=1e-12)
    assert abs(f0[j] - (1.0 + math.exp(-5.0))) < 1e-14


def test_example2_box_sources_count_and_amplitudes():
    # h = 1/3 keeps the cube faces (half-width 0.4) off the nodes
    for reg, b2 in (("h1h1", 1e-3), ("h1l2", 1e-8)):
        w = W.example2(reg, cells=12, M=2)
        assert (w.beta1, w.beta2, w.reg) == (1e-5, b2, reg)
        f = w.true_source()
        # t = 0: one source in each of four corners, 2^3 nodes each, amplitudes 2, 1, 1, 2
        assert np.count_nonzero(f[0]) == 32 and abs(f[0].sum() - 8 * 6.0) < 1e-12
        # t = 1/2: all four at the centre, 3^3 nodes with 2 + 1 + 1 + 2
        assert np.count_nonzero(f[1]) == 27 and np.allclose(f[1][f[1] > 0], 6.0)


def test_example3_sources_start_at_the_eight_corners():
    w = W.example3(9)
    assert w.cells == (64, 64, 64) and w.M == 47 and len(w.sensor_xyz) == 9 ** 3
    assert (w.beta1, w.beta2) == (3.6e-5, 3.6e-1) and len(W.example3(21).sensor_xyz) == 21 ** 3
    corners = {tuple(round(v, 12) for v in s.center(0.0)) for s in w.sources}
    assert corners == {(x, y, z) for x in (0.0, 4.0) for y in (0.0, 4.0) for z in (0.0, 4.0)}
    assert sorted(s.amp for s in w.sources) == [4.0] * 4 + [6.0] * 4


def test_reduced_example1_marches_to_finite_data():
    w = W.example1(cells=8, M=8)
    p = kkt.Problem.from_workload(w)
    C = forward.forward_march(p, w.true_source())
    obs = forward.observations(p, C, w.noise(), w.noise_eps)
    assert obs.shape == (9, 14 ** 3) and np.all(np.isfinite(obs)) and obs.max() > 0
    assert np.all(C[:, p.dirichlet] == 0.0)


def test_batch_members_are_seeded_and_in_range():
    a, b = W.batch(), W.batch()
    assert len(a) == 8 and [w.name for w in a] == [w.name for w in b]
    boxes = 0
    for w in a:
        assert 16 <= w.cells[0] <= 40 and w.cells[0] == w.cells[1] == w.cells[2] and 32 <= w.M <= 80
        assert round(len(w.sensor_xyz) ** (1 / 3)) ** 3 == len(w.sensor_xyz) and 27 <= len(w.sensor_xyz) <= 216
        assert 0.005 <= w.noise_eps <= 0.05 and 1 <= len(w.sources) <= 3
        assert np.allclose(w.beta2, 1e-3 * (32.0 / w.cells[0]) ** 2)
        boxes += int(np.prod(w.nsub))
    assert boxes == 512
