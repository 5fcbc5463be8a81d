"""Write a sample of the KKT solution of the 32^3 x 64 workload, computed by the oracle's
reduced-space method (oracle only).

The solution is the one of F_h U = b for the committed observations
(observations_mid_32x32x32x64.txt), computed without any part of the all-at-once
machinery: forward and adjoint time marches with Jacobi-BiCGSTAB steps (relative
residual 1e-14 per step) and GMRES on the source to a relative residual of 1e-13
(oracle/reduced.py, Sec. 1's traditional method).  The file holds the solution's
norms and the values of U at seeded sample indices: 4096 drawn over all unknowns and
4096 over the f components (the recovered source).  The GPU tests compare the FP64
form's U and the mixed forms' f with these values.

    python tests/golden/make_reduced_solution.py      # reduced_solution_mid_32x32x32x64.txt (~15-25 min)
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import kkt, reduced  # noqa: E402
from paper_1508_06103_gb300 import workloads as W  # noqa: E402

SAMPLES = 4096
SAMPLE_SEED = 20151


def sample_indices(P: int, n: int):
    """Seeded sample: n indices over all 3P unknowns and n over the f components (sorted)."""
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    u = np.sort(rng.choice(3 * P, size=n, replace=False))
    f = np.sort(3 * rng.choice(P, size=n, replace=False) + 2)
    return u, f


def write(w, obs_path, path, solver="bicgstab"):
    p = kkt.Problem.from_workload(w)
    cobs = np.loadtxt(obs_path, ndmin=2)
    b = kkt.rhs(p, cobs)
    t0 = time.time()
    r = reduced.solve(p, cobs, rtol=1e-13, solver=solver, step_rtol=1e-14, log=lambda s: print(s, flush=True))
    wall = time.time() - t0
    kres = np.linalg.norm(b - kkt.apply(p, r.U)) / np.linalg.norm(b)
    U = r.U.reshape(p.L, p.N, 3)
    iu, jf = sample_indices(p.P, SAMPLES)
    header = (f"reduced-space oracle solution of workload {w.name} ({p.n} unknowns) for "
              f"{os.path.basename(obs_path)}: GMRES {r.iterations} iterations, reduced relres {r.relres:.3e}, "
              f"KKT true relres {kres:.3e}, {wall:.0f} s\n"
              f"norm2_U {np.linalg.norm(r.U):.17e}\nnorm2_C {np.linalg.norm(U[..., 0]):.17e}\n"
              f"norm2_G {np.linalg.norm(U[..., 1]):.17e}\nnorm2_f {np.linalg.norm(U[..., 2]):.17e}\n"
              f"sample seed {SAMPLE_SEED}: {SAMPLES} indices over U then {SAMPLES} over its f components\n"
              f"columns: point-block index, value")
    idx = np.concatenate([iu, jf])
    np.savetxt(path, np.stack([idx.astype(np.float64), r.U[idx]], axis=1), fmt=["%d", "%.17e"], header=header)
    print(header, flush=True)


def read(path):
    """(norms dict, U sample indices, values, f sample indices, values) of a written file."""
    norms = {}
    for ln in open(path):
        if not ln.startswith("#"):
            break
        parts = ln[1:].split()
        if parts and parts[0].startswith("norm2_"):
            norms[parts[0][6:]] = float(parts[1])
    d = np.loadtxt(path, ndmin=2)
    idx = d[:, 0].astype(np.int64)
    return norms, idx[:SAMPLES], d[:SAMPLES, 1], idx[SAMPLES:], d[SAMPLES:, 1]


if __name__ == "__main__":
    w = W.mid()
    write(w, os.path.join(HERE, f"observations_{w.name}.txt"), os.path.join(HERE, f"reduced_solution_{w.name}.txt"))
