"""Seeded synthetic inputs for the space-time inverse source problem.

This module only *describes* problems: the grid, the coefficient fields a(x)
and v(x) sampled at cell centroids, the sensor positions (snapped to nodes),
the true source f(x, t) used to make observation data, and the standard
normal draws r of the multiplicative noise model C^eps = C + eps r C
(Section 4, data generation).  It holds none of the method's arithmetic
(no discretisation, no solver), so that both the CPU oracle and the CUDA
path can take their inputs from here without sharing any computation.

Conventions
-----------
* Domain [0, lx] x [0, ly] x [0, lz], uniform hexahedral cells
  ``cells = (cx, cy, cz)``; nodes per axis ``n = c + 1``.
* Node id ``j = ix + nx * (iy + ny * iz)``; cell id ``e = ex + cx * (ey + cy * ez)``.
* Time levels ``t^n = n * T / M`` for ``n = 0..M``.
* ``dirichlet_faces`` is a bit mask of the faces carrying the Dirichlet part
  Gamma_1 of the boundary: bit 0 x=0, bit 1 x=lx, bit 2 y=0, bit 3 y=ly,
  bit 4 z=0, bit 5 z=lz.  The other faces form the Neumann part Gamma_2.
* ``beta`` of a workload maps to (beta1, beta2) = (beta / 100, beta): the
  ratio the paper uses in its Examples 1 and 2 (Section 4.1).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Sequence, Tuple

import numpy as np

FACE_X0, FACE_X1, FACE_Y0, FACE_Y1, FACE_Z0, FACE_Z1 = 1, 2, 4, 8, 16, 32
ALL_FACES = 63


@dataclasses.dataclass
class Source:
    """One source times a switch w(t), centred at c(t): a Gaussian
    amp * exp(-|x - c(t)|^2 / (2 sigma^2)), or with shape "box" the constant amp
    on the cube max_k |x_k - c_k(t)| < half_width."""

    center: Callable[[float], Tuple[float, float, float]]
    sigma: float = 0.1
    amp: float = 1.0
    switch: Callable[[float], float] = lambda t: 1.0
    shape: str = "gaussian"
    half_width: float = 0.4


@dataclasses.dataclass
class Workload:
    name: str
    cells: Tuple[int, int, int]
    lengths: Tuple[float, float, float]
    T: float
    M: int
    theta: float
    dirichlet_faces: int
    a_cell: np.ndarray          # (ncell,)   diffusivity at cell centroids
    v_cell: np.ndarray          # (ncell, 3) velocity at cell centroids
    sensor_xyz: np.ndarray      # (s, 3)     sensor positions
    beta1: float
    beta2: float
    sources: List[Source]
    noise_eps: float
    noise_seed: int
    # solver settings (paper Section 4 / Table 3 defaults where the workload is silent)
    nsub: Tuple[int, int, int, int] = (2, 2, 2, 2)
    overlap: int = 1
    local: str = "ilu0"
    coarse_cells: Tuple[int, int, int] | None = None
    coarse_M: int | None = None
    coarse_overlap: int = 1
    coarse_nsub: Tuple[int, int, int, int] | None = None   # split of the coarse level (None: as nsub)
    coarse_rtol: float = 1e-1
    coarse_maxit: int = 4
    restart: int = 30
    rtol: float = 1e-8
    # regularisation: "h1h1" (N_beta, Eq. 3) or "h1l2" (beta2 |grad f|^2 -> beta2 f^2, Sec. 4 Example 2)
    reg: str = "h1h1"
    # spatial element: "q1" (trilinear hexahedra) or "p1" (linear tetrahedra, Kuhn split of each cell)
    element: str = "q1"

    # ---- derived sizes -------------------------------------------------
    @property
    def nodes(self) -> Tuple[int, int, int]:
        return tuple(c + 1 for c in self.cells)

    @property
    def N(self) -> int:
        nx, ny, nz = self.nodes
        return nx * ny * nz

    @property
    def P(self) -> int:
        return self.N * (self.M + 1)

    @property
    def unknowns(self) -> int:
        return 3 * self.P

    @property
    def coarse_split(self) -> Tuple[int, int, int, int]:
        """Subdomains of the coarse level's one-level RAS."""
        return self.coarse_nsub if self.coarse_nsub is not None else self.nsub

    @property
    def tau(self) -> float:
        return self.T / self.M

    @property
    def h(self) -> Tuple[float, float, float]:
        return tuple(l / c for l, c in zip(self.lengths, self.cells))

    def node_coords(self) -> np.ndarray:
        """(N, 3) coordinates of the nodes in node-id order."""
        nx, ny, nz = self.nodes
        hx, hy, hz = self.h
        iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        return np.stack([ix.ravel() * hx, iy.ravel() * hy, iz.ravel() * hz], axis=1)

    def sensor_nodes(self) -> np.ndarray:
        return snap_to_nodes(self.sensor_xyz, self.cells, self.lengths)

    def noise(self) -> np.ndarray:
        """Standard normal draws r, shape (M+1, s), one per sensor sample."""
        rng = np.random.Generator(np.random.PCG64(self.noise_seed))
        return rng.standard_normal((self.M + 1, len(self.sensor_xyz)))

    def true_source(self) -> np.ndarray:
        """Nodal values of the true source, shape (M+1, N)."""
        xyz = self.node_coords()
        out = np.zeros((self.M + 1, self.N))
        for n in range(self.M + 1):
            t = n * self.tau
            for s in self.sources:
                c = np.asarray(s.center(t))
                if s.shape == "box":
                    inside = (np.abs(xyz - c) < s.half_width).all(axis=1)
                    out[n] += s.amp * s.switch(t) * inside
                else:
                    r2 = ((xyz - c) ** 2).sum(axis=1)
                    out[n] += s.amp * s.switch(t) * np.exp(-r2 / (2.0 * s.sigma ** 2))
        return out


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def cell_centroids(cells: Sequence[int], lengths: Sequence[float]) -> np.ndarray:
    cx, cy, cz = cells
    hx, hy, hz = (l / c for l, c in zip(lengths, cells))
    ez, ey, ex = np.meshgrid(np.arange(cz), np.arange(cy), np.arange(cx), indexing="ij")
    return np.stack([(ex.ravel() + 0.5) * hx, (ey.ravel() + 0.5) * hy, (ez.ravel() + 0.5) * hz], axis=1)


def snap_to_nodes(xyz: np.ndarray, cells: Sequence[int], lengths: Sequence[float]) -> np.ndarray:
    """Nearest node of each point; a tie goes to the lower index."""
    nx, ny, nz = (c + 1 for c in cells)
    idx = []
    for d, (c, l) in enumerate(zip(cells, lengths)):
        u = xyz[:, d] * c / l
        # round half down: ceil(u - 0.5)
        k = np.ceil(u - 0.5 - 1e-12).astype(np.int64)
        idx.append(np.clip(k, 0, c))
    return (idx[0] + nx * (idx[1] + ny * idx[2])).astype(np.int32)


def sensor_lattice(m: int, lengths: Sequence[float]) -> np.ndarray:
    """m^3 sensors at ((k+1)/(m+1)) * L along each axis."""
    g = [(np.arange(m) + 1.0) / (m + 1.0) * l for l in lengths]
    z, y, x = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def smooth_random_field(xyz: np.ndarray, seed: int, modes: int = 8, kmax: int = 3) -> np.ndarray:
    """Sum of `modes` seeded Fourier modes (wave numbers <= kmax), min-max scaled to [0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    val = np.zeros(len(xyz))
    for _ in range(modes):
        k = rng.integers(0, kmax + 1, size=3)
        phase = rng.uniform(0.0, 2.0 * math.pi, size=3)
        amp = rng.uniform(0.5, 1.0)
        val += amp * np.prod(np.cos(math.pi * k[None, :] * xyz + phase[None, :]), axis=1)
    lo, hi = val.min(), val.max()
    return (val - lo) / (hi - lo) if hi > lo else np.zeros_like(val)


def circular_path(k: int, K: int, T: float, z: float, radius: float = 0.25):
    def c(t: float):
        ang = 2.0 * math.pi * t / T + 2.0 * math.pi * k / K
        return (0.5 + radius * math.cos(ang), 0.5 + radius * math.sin(ang), z)
    return c


def linear_path(p0, p1, T: float):
    def c(t: float):
        s = t / T
        return tuple(a + s * (b - a) for a, b in zip(p0, p1))
    return c


def switching(windows: Sequence[Tuple[float, float]]):
    def w(t: float) -> float:
        return 1.0 if any(a <= t < b for a, b in windows) else 0.0
    return w


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def tiny(theta: float = 1.0, reg: str = "h1h1") -> Workload:
    """8^3 cells x 16 implicit-Euler steps, one source moving on a line, 27 sensors."""
    cells, L = (8, 8, 8), (1.0, 1.0, 1.0)
    ncell = 8 ** 3
    beta = 1e-3
    return Workload(
        name="tiny_8x8x8x16", cells=cells, lengths=L, T=1.0, M=16, theta=theta,
        dirichlet_faces=ALL_FACES,
        a_cell=np.full(ncell, 0.1), v_cell=np.tile([1.0, 0.5, 0.0], (ncell, 1)),
        sensor_xyz=sensor_lattice(3, L), beta1=beta / 100, beta2=beta,
        sources=[Source(center=linear_path((0.3, 0.3, 0.5), (0.7, 0.7, 0.5), 1.0))],
        noise_eps=0.01, noise_seed=1,
        nsub=(2, 2, 2, 2), overlap=1, local="lu", restart=30, rtol=1e-8, reg=reg,
    )


def mid(cells=(32, 32, 32), M: int = 64, nsub=(4, 4, 4, 4), overlap: int = 2,
        coarse_cells=(16, 16, 16), coarse_M: int = 32, name: str | None = None) -> Workload:
    """32^3 cells x 64 Crank-Nicolson steps, two sources on circles, 125 sensors.

    a = 0.05 + 0.05 rho(x) with rho a seeded smooth field; v = (1, 1, 0) sin(pi z);
    Dirichlet on x = 0 only; beta = 1e-3 at 32 cells per axis.  Smaller `cells`/`M`
    give the same problem family at sizes the oracle solves in seconds; there beta
    is scaled with h^2 so that the ratio of the source-equation diagonal
    beta2 (grad g, grad g) to the mass coupling (g, g), about 9 beta2 / h^2, stays
    what it is at 32 cells (the balance that decides how well ILU(0) works).
    """
    L = (1.0, 1.0, 1.0)
    cen = cell_centroids(cells, L)
    a = 0.05 + 0.05 * smooth_random_field(cen, seed=2)
    v = np.stack([np.sin(math.pi * cen[:, 2]), np.sin(math.pi * cen[:, 2]), np.zeros(len(cen))], axis=1)
    beta = 1e-3 * (32.0 / cells[0]) ** 2
    srcs = [Source(center=circular_path(k, 2, 1.0, z)) for k, z in enumerate((0.6, 0.4))]
    return Workload(
        name=name or f"mid_{cells[0]}x{cells[1]}x{cells[2]}x{M}", cells=tuple(cells), lengths=L,
        T=1.0, M=M, theta=0.5, dirichlet_faces=FACE_X0, a_cell=a, v_cell=v,
        sensor_xyz=sensor_lattice(5, L), beta1=beta / 100, beta2=beta, sources=srcs,
        noise_eps=0.01, noise_seed=2, nsub=tuple(nsub), overlap=overlap, local="ilu0",
        coarse_cells=tuple(coarse_cells) if coarse_cells else None, coarse_M=coarse_M,
        coarse_overlap=1, coarse_rtol=1e-1, coarse_maxit=4, restart=30, rtol=1e-8,
    )


def large() -> Workload:
    """64^3 cells x 128 steps, layered a with 100x contrast, rotating v, 3 switching sources."""
    cells, L = (64, 64, 64), (1.0, 1.0, 1.0)
    cen = cell_centroids(cells, L)
    band = np.floor(cen[:, 2] * 8).astype(int)
    a = np.where(band % 2 == 0, 0.01, 1.0)
    v = np.stack([-(cen[:, 1] - 0.5), cen[:, 0] - 0.5, np.full(len(cen), 0.2)], axis=1)
    beta = 1e-3
    srcs = [
        Source(center=circular_path(0, 3, 1.0, 0.5), switch=switching([(0.0, 0.4), (0.7, 1.01)])),
        Source(center=circular_path(1, 3, 1.0, 0.35), switch=switching([(0.2, 0.8)])),
        Source(center=circular_path(2, 3, 1.0, 0.65), switch=switching([(0.0, 0.3), (0.5, 0.9)])),
    ]
    return Workload(
        name="large_64x64x64x128", cells=cells, lengths=L, T=1.0, M=128, theta=0.5,
        dirichlet_faces=FACE_X0, a_cell=a, v_cell=v, sensor_xyz=sensor_lattice(8, L),
        beta1=beta / 100, beta2=beta, sources=srcs, noise_eps=0.02, noise_seed=5,
        nsub=(8, 8, 8, 8), overlap=2, local="ilu0", coarse_cells=(16, 16, 16), coarse_M=32,
        coarse_overlap=1, coarse_nsub=(4, 4, 4, 4), restart=40, rtol=1e-8,
    )


def batch(seed: int = 4, count: int = 8) -> List[Workload]:
    """Independent inverse problems solved together (one launch per kernel for all of them).

    Each member is drawn from `seed`: a grid of c^3 cells with c in [16, 40] and M in [32, 80]
    Crank-Nicolson steps, an m^3 sensor lattice with m in [3, 6], noise of 0.5-5 %, and 1-3
    Gaussian sources on circular paths at seeded heights; a(x) = 0.05 + 0.05 rho(x) with rho a
    seeded smooth field, v = (1, 1, 0) sin(pi z), Dirichlet on x = 0, beta scaled with h^2 from
    1e-3 at 32 cells (as the 32^3 x 64 family).  Each problem is split into 4 x 4 x 2 x 2
    space-time subdomains with overlap 1 (64 per problem, 512 for eight), FP32 local solves.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    L = (1.0, 1.0, 1.0)
    for k in range(count):
        c = int(rng.integers(16, 41))
        M = int(rng.integers(32, 81))
        m = int(rng.integers(3, 7))
        eps = float(rng.uniform(0.005, 0.05))
        nsrc = int(rng.integers(1, 4))
        zs = rng.uniform(0.3, 0.7, nsrc)
        cells = (c, c, c)
        cen = cell_centroids(cells, L)
        a = 0.05 + 0.05 * smooth_random_field(cen, seed=seed * 100 + k)
        v = np.stack([np.sin(math.pi * cen[:, 2]), np.sin(math.pi * cen[:, 2]), np.zeros(len(cen))], axis=1)
        beta = 1e-3 * (32.0 / c) ** 2
        srcs = [Source(center=circular_path(i, nsrc, 1.0, float(z))) for i, z in enumerate(zs)]
        out.append(Workload(
            name=f"batch{seed}_{k}_{c}x{c}x{c}x{M}", cells=cells, lengths=L, T=1.0, M=M, theta=0.5,
            dirichlet_faces=FACE_X0, a_cell=a, v_cell=v, sensor_xyz=sensor_lattice(m, L),
            beta1=beta / 100, beta2=beta, sources=srcs, noise_eps=eps, noise_seed=seed * 100 + k,
            nsub=(4, 4, 2, 2), overlap=1, local="ilu0", restart=30, rtol=1e-8,
        ))
    return out


# ---------------------------------------------------------------------------
# the paper's Examples 1-3 (Sec. 4.1) as synthetic workloads
# ---------------------------------------------------------------------------
# Domain (-2, 2)^3 (here [0, 4]^3, paper coordinates shifted by +2), T = 1,
# C(., 0) = 0, a = 1, v = (1, 1, 1); Dirichlet on |x| = 2 and |y| = 2, Neumann
# on |z| = 2; Crank-Nicolson.  Sensors: an m^3 lattice inside the domain.  The
# paper runs these with np = 256 subdomains (4^4 here), overlap 1, ILU(0),
# one level.  L = S = H = 2 are the half-widths used in the source traces.
_HALF = 2.0


def _paper_example(name, cells, M, sources, sensors, beta1, beta2, noise_eps=0.01, reg="h1h1"):
    L = (2 * _HALF,) * 3
    ncell = cells ** 3
    return Workload(
        name=name, cells=(cells,) * 3, lengths=L, T=1.0, M=M, theta=0.5,
        dirichlet_faces=FACE_X0 | FACE_X1 | FACE_Y0 | FACE_Y1,
        a_cell=np.full(ncell, 1.0), v_cell=np.tile([1.0, 1.0, 1.0], (ncell, 1)),
        sensor_xyz=sensor_lattice(sensors, L), beta1=beta1, beta2=beta2, sources=sources,
        noise_eps=noise_eps, noise_seed=11, nsub=(4, 4, 4, 4), overlap=1, local="ilu0",
        restart=30, rtol=1e-8, reg=reg,
    )


def _shifted(f):
    """A trace in the paper's coordinates on (-2, 2)^3, moved to [0, 4]^3."""
    def c(t: float):
        return tuple(v + _HALF for v in f(t))
    return c


def example1(cells: int = 40, M: int = 39, noise_eps: float = 0.01) -> Workload:
    """Two moving Gaussians exp(-|x - x_i(t)|^2 / a^2), a = 2 (so sigma = a / sqrt 2);
    40^3 mesh, tau = 1/39, 14^3 sensors, beta1 = 3.6e-5, beta2 = 3.6e-3."""
    L = S = H = _HALF
    tr1 = _shifted(lambda t: (L * math.sin(2 * math.pi * t), S * math.cos(2 * math.pi * t),
                              H * math.cos(4 * math.pi * t)))
    tr2 = _shifted(lambda t: (L - 2 * L * abs(math.cos(4 * t)), -S + 2 * S * abs(math.cos(4 * t)),
                              -H + 2 * H * t * t))
    sig = 2.0 / math.sqrt(2.0)
    return _paper_example(f"example1_{cells}x{M}", cells, M, [Source(tr1, sig), Source(tr2, sig)], 14,
                          3.6e-5, 3.6e-3, noise_eps)


def example2(reg: str = "h1h1", cells: int = 40, M: int = 39) -> Workload:
    """Four constant cube sources of half-width 0.4 moving along the diagonals to the far
    corners, amplitudes 2, 1, 1, 2; mesh, sensors as Example 1; beta1 = 1e-5 and beta2 = 1e-3
    (H1-H1) or 1e-8 (H1-L2)."""
    L = S = H = _HALF
    traces = [
        lambda t: (-L + 2 * L * t, -S + 2 * S * t, H - 2 * H * t),
        lambda t: (L - 2 * L * t, S - 2 * S * t, -H + 2 * H * t),
        lambda t: (L - 2 * L * t, -S + 2 * S * t, -H + 2 * H * t),
        lambda t: (-L + 2 * L * t, S - 2 * S * t, H - 2 * H * t),
    ]
    amps = (2.0, 1.0, 1.0, 2.0)
    srcs = [Source(_shifted(tr), amp=a, shape="box", half_width=0.4) for tr, a in zip(traces, amps)]
    beta2 = 1e-3 if reg == "h1h1" else 1e-8
    return _paper_example(f"example2_{reg}_{cells}x{M}", cells, M, srcs, 14, 1e-5, beta2, reg=reg)


def example3(sensors: int = 21, cells: int = 64, M: int = 47) -> Workload:
    """Eight Gaussians a_i exp(-|x - x_i(t)|^2) starting at the corners (the printed exponent's
    parentheses are garbled; read as -|x - x_i|^2, so sigma = 1/sqrt 2), a = 4 (i <= 4), 6;
    64^3 mesh, tau = 1/47, 21^3 or 9^3 sensors, beta1 = 3.6e-5, beta2 = 3.6e-1."""
    L = S = H = _HALF
    c2, s2 = (lambda t, k=1.0: math.cos(k * math.pi * t) ** 2), (lambda t: math.sin(math.pi * t) ** 2)
    ch, sh = (lambda t: math.cos(math.pi / 2 * t)), (lambda t: math.sin(math.pi / 2 * t))
    traces = [
        lambda t: (-L + 2 * L * (1 - t), -S + 2 * S * (1 - t), -H + 2 * H * (1 - t)),
        lambda t: (-L + 2 * L * t, -S + 2 * S * t, -H + 2 * H * t),
        lambda t: (-L + 2 * L * c2(t) * (1 - t), -S + 2 * S * s2(t) * t, -H + 2 * H * c2(t) * (1 - t)),
        lambda t: (-L + 2 * L * c2(t) * (1 - t), -S + 2 * S * c2(t) * (1 - t), -H + 2 * H * s2(t) * t),
        lambda t: (-L + 2 * L * c2(t, 2.0) * ch(t), -S + 2 * S * s2(t) * sh(t), -H + 2 * H * s2(t) * sh(t)),
        lambda t: (-L + 2 * L * s2(t) * sh(t), -S + 2 * S * c2(t, 2.0) * ch(t), -H + 2 * H * s2(t) * sh(t)),
        lambda t: (-L + 2 * L * s2(t) * sh(t), -S + 2 * S * s2(t) * sh(t), -H + 2 * H * c2(t, 2.0) * ch(t)),
        lambda t: (-L + 2 * L * s2(t) * sh(t), -S + 2 * S * c2(t, 2.0) * ch(t), -H + 2 * H * c2(t, 2.0) * ch(t)),
    ]
    amps = (4.0,) * 4 + (6.0,) * 4
    sig = 1.0 / math.sqrt(2.0)
    srcs = [Source(_shifted(tr), sig, a) for tr, a in zip(traces, amps)]
    return _paper_example(f"example3_s{sensors}_{cells}x{M}", cells, M, srcs, sensors, 3.6e-5, 3.6e-1)


def random_small(seed: int, cells=(5, 4, 3), M: int = 5, theta: float = 0.5,
                 dirichlet_faces: int = FACE_X0 | FACE_Y1, nsens: int = 6, reg: str = "h1h1") -> Workload:
    """Small problem with random coefficients, for parity tests on ragged sizes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = (1.0, 0.8, 0.6)
    ncell = int(np.prod(cells))
    a = rng.uniform(0.05, 0.2, ncell)
    v = rng.uniform(-1.0, 1.0, (ncell, 3))
    xyz = rng.uniform(0.0, 1.0, (nsens, 3)) * np.asarray(L)
    return Workload(
        name=f"random_{seed}", cells=tuple(cells), lengths=L, T=1.0, M=M, theta=theta,
        dirichlet_faces=dirichlet_faces, a_cell=a, v_cell=v, sensor_xyz=xyz,
        beta1=1e-4, beta2=1e-2, sources=[Source(center=lambda t: (0.5, 0.4, 0.3))],
        noise_eps=0.0, noise_seed=seed, reg=reg,
    )


def refined(w: Workload, r: int) -> Workload:
    """The same problem on a mesh r times finer in space and time, for data generation.

    Sec. 4 generates the observations by a forward solve "on a finer mesh with a
    smaller time step".  Each fine cell keeps the diffusivity and velocity of the
    cell it lies in (so every refinement discretises the same coefficients), the
    sensors sit at the coordinates of the nodes the coarse mesh snaps them to
    (nodes of every refinement), and the sources, noise draws and the rest are
    unchanged; the coarse levels are the fine levels 0, r, 2r, ...
    """
    if r < 1:
        raise ValueError("refinement factor must be >= 1")
    cx, cy, cz = w.cells
    fx, fy, fz = cx * r, cy * r, cz * r
    kz, ky, kx = np.meshgrid(np.arange(fz) // r, np.arange(fy) // r, np.arange(fx) // r, indexing="ij")
    parent = (kx + cx * (ky + cy * kz)).ravel()
    sens = w.node_coords()[w.sensor_nodes()]
    return dataclasses.replace(w, name=f"{w.name}_refined{r}", cells=(fx, fy, fz), M=w.M * r,
                               a_cell=np.asarray(w.a_cell)[parent], v_cell=np.asarray(w.v_cell)[parent],
                               sensor_xyz=sens)


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded standard normal vector."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)
