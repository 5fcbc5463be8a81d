"""Pins of the data generation on a finer mesh (Sec. 4: observations from a forward solve on a
finer mesh with a smaller time step).

* Refining by 1 reproduces the same-mesh observations exactly.
* On the 8^3 x 16 workload with the Crank-Nicolson scheme and no noise, the observations from
  meshes refined 1x, 2x and 4x in space and time converge at second order: the distance of the
  1x data to the 4x data is about (1 - 1/16) / (1/4 - 1/16) = 5 times that of the 2x data
  (first order would give 3).  This checks that every refinement discretises the same problem
  (coefficients, sensor positions, source, time levels).
* The noise model of Sec. 4, C^eps = C + eps r C with r standard Gaussian, fixed by what the
  paper states about it rather than by its formula: the noise is relative (a sensor whose state
  is zero reads exactly zero, and scaling C scales the data by the same factor for fixed draws),
  its level is eps (over many samples the relative perturbation (C^eps - C) / (eps C) has mean 0
  and standard deviation 1, drawn with the workload's own generator), and without noise the data
  are C at the sensor locations: for a state that is the nodal interpolant of a known function,
  the function's values at the sensors' (node-snapped) coordinates.
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


def _noise_case():
    w = W.random_small(6, cells=(4, 3, 3), M=8, nsens=7)
    p = kkt.Problem.from_workload(w)
    xyz = w.node_coords()
    t = np.arange(p.L)[:, None] * p.tau
    C = np.sin(1.0 + xyz[:, 0])[None, :] * np.cos(0.5 + xyz[:, 1] - xyz[:, 2])[None, :] * (1.0 + t)
    return w, p, C


def test_noise_is_relative_and_of_degree_one_in_the_state():
    w, p, C = _noise_case()
    r = np.random.default_rng(3).standard_normal((p.L, len(p.sensor_node)))
    obs = forward.observations(p, C, r, 0.05)
    assert np.array_equal(forward.observations(p, np.zeros_like(C), r, 0.05), np.zeros_like(obs))
    assert np.allclose(forward.observations(p, 3.0 * C, r, 0.05), 3.0 * obs, rtol=1e-15, atol=0)
    Cz = C.copy()
    Cz[:, p.sensor_node[0]] = 0.0
    assert np.all(forward.observations(p, Cz, r, 0.05)[:, 0] == 0.0)


def test_noise_level_is_eps_with_the_workloads_own_draws():
    w = W.random_small(7, cells=(6, 6, 6), M=40, nsens=120)
    w = dataclasses.replace(w, noise_eps=0.02)
    p = kkt.Problem.from_workload(w)
    C = 1.0 + np.abs(W.random_vector(p.L * p.N, 9)).reshape(p.L, p.N)
    obs = forward.observations(p, C, w.noise(), w.noise_eps)
    rel = (obs - C[:, p.sensor_node]) / (w.noise_eps * C[:, p.sensor_node])
    assert rel.size > 4000
    assert abs(rel.mean()) < 4.0 / np.sqrt(rel.size) and abs(rel.std() - 1.0) < 0.05


def test_noise_free_data_are_the_state_at_the_sensor_locations():
    w, p, C = _noise_case()
    obs = forward.observations(p, C, np.zeros((p.L, len(p.sensor_node))), 0.0)
    hx, hy, hz = w.h
    snapped = np.rint(w.sensor_xyz / np.array([hx, hy, hz])) * np.array([hx, hy, hz])
    t = np.arange(p.L)[:, None] * p.tau
    expect = (np.sin(1.0 + snapped[:, 0])[None, :] * np.cos(0.5 + snapped[:, 1] - snapped[:, 2])[None, :]
              * (1.0 + t))
    assert np.allclose(obs, expect, rtol=1e-14, atol=1e-14)
