"""Write the KKT solution of the 8^3 x 16 implicit-Euler workload by a sparse direct solve (oracle only).

F_h is assembled by the oracle (oracle/kkt.py) and solved with scipy's sparse LU (SuperLU, a library
routine used as one step); the observations are the oracle's forward march of the true source with
the workload's seeded noise.  The file holds the solution's norms and its values at 4096 seeded
sample indices; the GPU test of that workload compares its solution with them.

    python tests/golden/make_direct_solution.py     # direct_solution_tiny_8x8x8x16.txt (a few minutes)
"""

import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import forward, kkt  # noqa: E402
from paper_1508_06103_gb300 import workloads as W  # noqa: E402

SAMPLES = 4096
SAMPLE_SEED = 20152


def write(w, path):
    p = kkt.Problem.from_workload(w)
    C = forward.forward_march(p, w.true_source())
    cobs = forward.observations(p, C, w.noise(), w.noise_eps)
    b = kkt.rhs(p, cobs)
    F = kkt.assemble(p)
    t0 = time.time()
    U = spla.spsolve(F.tocsc(), b)
    wall = time.time() - t0
    res = np.linalg.norm(b - F @ U) / np.linalg.norm(b)
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    idx = np.sort(rng.choice(p.n, size=SAMPLES, replace=False))
    header = (f"sparse direct solution of workload {w.name} ({p.n} unknowns), theta {w.theta}: "
              f"true relres {res:.3e}, {wall:.0f} s\n"
              f"norm2_U {np.linalg.norm(U):.17e}\n"
              f"sample seed {SAMPLE_SEED}: {SAMPLES} indices over U\ncolumns: point-block index, value")
    np.savetxt(path, np.stack([idx.astype(np.float64), U[idx]], axis=1), fmt=["%d", "%.17e"], header=header)
    print(header, flush=True)


def read(path):
    """(norm of U, sample indices, values) of a written file."""
    norm = None
    for ln in open(path):
        if not ln.startswith("#"):
            break
        parts = ln[1:].split()
        if parts and parts[0] == "norm2_U":
            norm = float(parts[1])
    d = np.loadtxt(path, ndmin=2)
    return norm, d[:, 0].astype(np.int64), d[:, 1]


if __name__ == "__main__":
    w = W.tiny(theta=1.0)
    write(w, os.path.join(HERE, f"direct_solution_{w.name}.txt"))
