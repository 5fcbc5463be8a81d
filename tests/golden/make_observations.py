"""Write the noisy sensor observations of the 32^3 x 64 workload (oracle only).

The data follow Sec. 4 of the paper: the forward problem is solved with the
true source (here on the same mesh and scheme; the paper uses a finer mesh)
and the sensor values get multiplicative Gaussian noise C + eps r C.  The
forward solve is the oracle's time march; the seeded inputs (grid,
coefficients, sensors, source, noise draws r) come from the workload module.
The benchmark reads the resulting text file so that it never runs the oracle
outside its CPU-baseline leg.

    python tests/golden/make_observations.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import forward, kkt  # noqa: E402
from paper_1508_06103_gb300 import workloads as W  # noqa: E402


def write(w, path):
    p = kkt.Problem.from_workload(w)
    C = forward.forward_march(p, w.true_source())
    obs = forward.observations(p, C, w.noise(), w.noise_eps)
    header = (f"noisy observations C + eps r C at {len(p.sensor_node)} sensors x {p.L} levels, "
              f"workload {w.name}, eps {w.noise_eps}, noise seed {w.noise_seed}; row = time level")
    np.savetxt(path, obs, fmt="%.17g", header=header)


if __name__ == "__main__":
    w = W.mid()
    write(w, os.path.join(HERE, f"observations_{w.name}.txt"))
