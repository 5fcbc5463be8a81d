"""Pins of the data generation on a finer mesh (Sec. 4: observations from a forward solve on a
finer mesh with a smaller time step).

* Refining by 1 reproduces the same-mesh observations exactly.
* On the 8^3 x 16 workload with the Crank-Nicolson scheme and no noise, the observations from
  meshes refined 1x, 2x and 4x in space and time converge at second order: the distance of the
  1x data to the 4x data is about (1 - 1/16) / (1/4 - 1/16) = 5 times that of the 2x data
  (first order would give 3).  This checks that every refinement discretises the same problem
  (coefficients, sensor positions, source, time levels).
"""

import dataclasses

import numpy as np

from oracle import forward, kkt
from paper_1508_06103_gb300 import workloads as W


def _data(w, r):
    wf = W.refined(w, r)
    pf = kkt.Problem.from_workload(wf)
    assert pf.M == w.M * r and len(pf.sensor_node) == len(w.sensor_xyz)
    return forward.observations_refined(pf, wf.true_source(), r, w.noise(), w.noise_eps)


def test_refinement_by_one_is_the_same_mesh_data():
    w = W.random_small(4, cells=(3, 4, 2), M=4)
    w = dataclasses.replace(w, noise_eps=0.02)
    p = kkt.Problem.from_workload(w)
    same = forward.observations(p, forward.forward_march(p, w.true_source()), w.noise(), w.noise_eps)
    np.testing.assert_array_equal(_data(w, 1), same)


def test_refined_sensors_sit_on_the_coarse_sensor_nodes():
    w = W.tiny()
    wf = W.refined(w, 3)
    xyz_c = w.node_coords()[w.sensor_nodes()]
    xyz_f = wf.node_coords()[wf.sensor_nodes()]
    np.testing.assert_allclose(xyz_f, xyz_c, atol=1e-14)


def test_refined_data_converge_at_second_order():
    w = dataclasses.replace(W.tiny(theta=0.5), noise_eps=0.0)
    d1, d2, d4 = (_data(w, r) for r in (1, 2, 4))
    e1, e2 = np.linalg.norm(d1 - d4), np.linalg.norm(d2 - d4)
    assert e1 < 0.1 * np.linalg.norm(d4)
    assert e1 / e2 > 3.8, e1 / e2


def test_iterative_step_solver_matches_sparse_lu():
    """The BiCGSTAB step solve (for refined meshes) reproduces the sparse-LU march."""
    w = W.tiny(theta=0.5)
    p = kkt.Problem.from_workload(w)
    f = w.true_source()
    a = forward.forward_march(p, f)
    b = forward.forward_march(p, f, solver="bicgstab")
    assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()
