"""Write the noisy sensor observations of the 32^3 x 64 workload (oracle only).

The data follow Sec. 4 of the paper: the forward problem is solved with the
true source (by default on the same mesh and scheme; with --refine R on a mesh
R times finer in space and time, as the paper does) and the sensor values get
multiplicative Gaussian noise C + eps r C.  The
forward solve is the oracle's time march; the seeded inputs (grid,
coefficients, sensors, source, noise draws r) come from the workload module.
The benchmark reads the resulting text file so that it never runs the oracle
outside its CPU-baseline leg.

    python tests/golden/make_observations.py              # observations_mid_32x32x32x64.txt
    python tests/golden/make_observations.py --refine 2   # ..._refined2.txt (not used by default)
    python tests/golden/make_observations.py --workload large   # observations_large_64x64x64x128.txt
    python tests/golden/make_observations.py --workload batch   # observations_batch4_<k>_*.txt, 8 problems
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import forward, kkt  # noqa: E402
from paper_1508_06103_gb300 import workloads as W  # noqa: E402


def write(w, path, refine=1, solver="lu"):
    if refine == 1:
        p = kkt.Problem.from_workload(w)
        C = forward.forward_march(p, w.true_source(), solver=solver)
        obs = forward.observations(p, C, w.noise(), w.noise_eps)
    else:
        wf = W.refined(w, refine)
        # the refined 3D step matrix is too large for sparse LU: BiCGSTAB to 1e-13 per step
        obs = forward.observations_refined(kkt.Problem.from_workload(wf), wf.true_source(), refine, w.noise(),
                                           w.noise_eps, solver="bicgstab")
    fine = "" if refine == 1 else f", forward solve on a mesh refined {refine}x"
    header = (f"noisy observations C + eps r C at {obs.shape[1]} sensors x {obs.shape[0]} levels, "
              f"workload {w.name}, eps {w.noise_eps}, noise seed {w.noise_seed}{fine}; row = time level")
    np.savetxt(path, obs, fmt="%.17g", header=header)


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("--refine", type=int, default=1)
    ap.add_argument("--workload", choices=["mid", "large", "batch"], default="mid")
    a = ap.parse_args()
    if a.workload == "batch":
        for wk in W.batch():
            # iterative steps above ~25^3 nodes, where sparse LU fill grows large
            write(wk, os.path.join(HERE, f"observations_{wk.name}.txt"), 1,
                  "lu" if wk.cells[0] <= 24 else "bicgstab")
        sys.exit(0)
    w = W.mid() if a.workload == "mid" else W.large()
    suffix = "" if a.refine == 1 else f"_refined{a.refine}"
    # the 65^3-node step matrix is too large for sparse LU: iterative steps to 1e-13
    write(w, os.path.join(HERE, f"observations_{w.name}{suffix}.txt"), a.refine,
          "lu" if a.workload == "mid" else "bicgstab")
