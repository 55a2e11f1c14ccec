"""Seeded synthetic inputs for the heat-stencil workloads.

This module only draws random fields; it holds none of the stencil's arithmetic.
Both the CPU oracle (through the tests) and the CUDA path (through the tests and
the benchmark) take their inputs from here, so the two sides see identical bytes.

Generator: numpy ``default_rng(seed)`` (PCG64).  Every field is drawn as float32
in the fixed order u, kappa, s, then any extras.  The time step is
``dt = fl32(r / max(kappa))``: the ratio is formed in float64 from the float32
maximum and rounded once to float32, so ``r = dt * max(kappa)`` is the stated
stability number up to one float32 rounding.

Workloads (sizes and distributions follow the stencil-class workloads the paper
evaluates: Rodinia hotspot 1024^2 and srad 8192^2 in its evaluation; their data
files are not used -- these seeded fields stand in at the same scale):

* ``plain_small``      512 x 512, u~U[0,1), kappa~U[0.5,1), s~U[0,1e-3),
                       Dirichlet, r = 0.2, 100 steps, seed 0.
* ``plain_scale``      8192 x 8192, kappa = clip(exp(0.5 N(0,1)), 0.1, 4),
                       s~U[0,1e-3) (or 0), periodic, r = 0.24, 1000 steps.
* ``precision``        16384 x 16384, distributions of ``plain_small``,
                       Dirichlet, r = 0.2, 2000 steps.
* ``batching``         4096 grids, nx and ny independently round(exp(U[ln 32,
                       ln 1024])), steps uniform in {10..500}, per-grid
                       kappa~U[0.5,1), s~U[0,1e-3), u~U[0,1), Dirichlet,
                       per-grid dt with r = 0.2.
* ``differentiation``  2048 x 2048, kappa~U[0.5,1), u0~U[0,1), s = 0,
                       Dirichlet, r = 0.2, 200 steps, checkpoint every 20;
                       target = sum of 8 seeded sinusoidal modes.
* ``volume``           the 3-D 7-point variant (the paper's hotspot3D class,
                       512 x 512 in its evaluation, layer count unstated):
                       512 x 512 x 512, distributions of ``plain_small``,
                       Dirichlet, r = 0.15 (six faces: r <= 1/6 keeps the
                       update a convex combination), 100 steps, seed 5.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DIRICHLET = 0
PERIODIC = 1


def dt_for(kappa: np.ndarray, r: float) -> np.float32:
    """fl32(r / max kappa), ratio formed in float64 from the float32 maximum."""
    kmax = float(np.max(kappa)) if kappa.size else 1.0
    return np.float32(r / kmax)


@dataclass
class Grid:
    """One grid problem.  Fields are row-major (ny, nx) float32, x fastest."""
    u: np.ndarray
    kappa: np.ndarray
    src: np.ndarray
    dt: np.float32
    steps: int
    bc: int
    name: str = ""
    extras: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return int(self.u.shape[1])

    @property
    def ny(self) -> int:
        return int(self.u.shape[0])

    @property
    def updates(self) -> int:
        return self.nx * self.ny * self.steps


def _uniform(rng, shape, lo, hi):
    return (rng.random(shape, dtype=np.float32) * np.float32(hi - lo) + np.float32(lo)).astype(np.float32)


def random_grid(seed: int, nx: int, ny: int, steps: int, bc: int, r: float = 0.2,
                kappa_lo: float = 0.5, kappa_hi: float = 1.0, src_hi: float = 1e-3,
                zero_source: bool = False) -> Grid:
    """A grid with the plain-small distributions at any size (parity cases)."""
    rng = np.random.default_rng(seed)
    u = rng.random((ny, nx), dtype=np.float32)
    kappa = _uniform(rng, (ny, nx), kappa_lo, kappa_hi)
    src = rng.random((ny, nx), dtype=np.float32) * np.float32(src_hi)
    if zero_source:
        src = np.zeros_like(src)
    return Grid(u, kappa, src.astype(np.float32), dt_for(kappa, r), steps, bc,
                name=f"random-{nx}x{ny}-seed{seed}")


@dataclass
class Grid3:
    """One 3-D grid problem.  Fields are (nz, ny, nx) float32, x fastest."""
    u: np.ndarray
    kappa: np.ndarray
    src: np.ndarray
    dt: np.float32
    steps: int
    bc: int
    name: str = ""

    @property
    def nx(self) -> int:
        return int(self.u.shape[2])

    @property
    def ny(self) -> int:
        return int(self.u.shape[1])

    @property
    def nz(self) -> int:
        return int(self.u.shape[0])

    @property
    def updates(self) -> int:
        return self.nx * self.ny * self.nz * self.steps


def random_grid3(seed: int, nx: int, ny: int, nz: int, steps: int, bc: int, r: float = 0.15,
                 kappa_lo: float = 0.5, kappa_hi: float = 1.0, src_hi: float = 1e-3,
                 zero_source: bool = False) -> Grid3:
    """A 3-D grid with the plain-small distributions (u, kappa, s drawn in that order)."""
    rng = np.random.default_rng(seed)
    u = rng.random((nz, ny, nx), dtype=np.float32)
    kappa = _uniform(rng, (nz, ny, nx), kappa_lo, kappa_hi)
    src = rng.random((nz, ny, nx), dtype=np.float32) * np.float32(src_hi)
    if zero_source:
        src = np.zeros_like(src)
    return Grid3(u, kappa, src.astype(np.float32), dt_for(kappa, r), steps, bc,
                 name=f"random3-{nx}x{ny}x{nz}-seed{seed}")


def volume(seed: int = 5, n: int = 512, steps: int = 100) -> Grid3:
    g = random_grid3(seed, n, n, n, steps, DIRICHLET, r=0.15)
    g.name = f"volume-{n}x{n}x{n}-dirichlet-{steps}steps"
    return g


def plain_small(seed: int = 0, n: int = 512, steps: int = 100) -> Grid:
    g = random_grid(seed, n, n, steps, DIRICHLET, r=0.2)
    g.name = f"plain-{n}x{n}-dirichlet-{steps}steps"
    return g


def lognormal_kappa(rng, shape) -> np.ndarray:
    z = rng.standard_normal(shape, dtype=np.float32)
    return np.clip(np.exp(np.float32(0.5) * z), np.float32(0.1), np.float32(4.0)).astype(np.float32)


def plain_scale(seed: int = 1, n: int = 8192, steps: int = 1000, zero_source: bool = False) -> Grid:
    rng = np.random.default_rng(seed)
    u = rng.random((n, n), dtype=np.float32)
    kappa = lognormal_kappa(rng, (n, n))
    src = rng.random((n, n), dtype=np.float32) * np.float32(1e-3)
    if zero_source:
        src = np.zeros_like(src)
    g = Grid(u, kappa, src.astype(np.float32), dt_for(kappa, 0.24), steps, PERIODIC,
             name=f"plain-{n}x{n}-periodic-{steps}steps" + ("-s0" if zero_source else ""))
    return g


def precision(seed: int = 2, n: int = 16384, steps: int = 2000) -> Grid:
    g = random_grid(seed, n, n, steps, DIRICHLET, r=0.2)
    g.name = f"precision-{n}x{n}-dirichlet-{steps}steps"
    return g


@dataclass
class Batch:
    """Many independent grids packed back to back in flat float32 arrays."""
    nx: np.ndarray          # int32 [G]
    ny: np.ndarray          # int32 [G]
    steps: np.ndarray       # int32 [G]
    dt: np.ndarray          # float32 [G]
    offset: np.ndarray      # int64 [G] element offset of each grid in the flat arrays
    u: np.ndarray           # float32 [total]
    kappa: np.ndarray
    src: np.ndarray
    bc: int = DIRICHLET

    @property
    def ngrids(self) -> int:
        return int(self.nx.shape[0])

    @property
    def cells(self) -> int:
        return int(self.u.shape[0])

    @property
    def updates(self) -> int:
        return int(np.sum(self.nx.astype(np.int64) * self.ny.astype(np.int64) * self.steps.astype(np.int64)))

    def grid(self, g: int) -> Grid:
        o, nx, ny = int(self.offset[g]), int(self.nx[g]), int(self.ny[g])
        sl = slice(o, o + nx * ny)
        return Grid(self.u[sl].reshape(ny, nx), self.kappa[sl].reshape(ny, nx),
                    self.src[sl].reshape(ny, nx), np.float32(self.dt[g]), int(self.steps[g]), self.bc,
                    name=f"batch-grid{g}")


def batching(seed: int = 3, ngrids: int = 4096, side_lo: int = 32, side_hi: int = 1024,
             steps_lo: int = 10, steps_hi: int = 500) -> Batch:
    """Uneven grids: sides log-uniform in [side_lo, side_hi], drawn separately."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(side_lo), math.log(side_hi)
    nx = np.rint(np.exp(rng.uniform(lo, hi, ngrids))).astype(np.int32)
    ny = np.rint(np.exp(rng.uniform(lo, hi, ngrids))).astype(np.int32)
    steps = rng.integers(steps_lo, steps_hi + 1, ngrids).astype(np.int32)
    cells = nx.astype(np.int64) * ny.astype(np.int64)
    offset = np.zeros(ngrids, dtype=np.int64)
    if ngrids > 1:
        offset[1:] = np.cumsum(cells)[:-1]
    total = int(cells.sum())
    u = rng.random(total, dtype=np.float32)
    kappa = _uniform(rng, total, 0.5, 1.0)
    src = (rng.random(total, dtype=np.float32) * np.float32(1e-3)).astype(np.float32)
    dt = np.empty(ngrids, dtype=np.float32)
    for g in range(ngrids):
        o = int(offset[g])
        dt[g] = dt_for(kappa[o:o + int(cells[g])], 0.2)
    return Batch(nx, ny, steps, dt, offset, u, kappa, src, DIRICHLET)


def smooth_target(rng, nx: int, ny: int, modes: int = 8) -> np.ndarray:
    """Sum of `modes` sinusoids a sin(2 pi (f i/nx + g j/ny) + phi), float32."""
    a = rng.random(modes) / modes
    f = rng.integers(1, 9, modes)
    g = rng.integers(1, 9, modes)
    phi = rng.uniform(0.0, 2.0 * math.pi, modes)
    i = np.arange(nx, dtype=np.float64)[None, :]
    j = np.arange(ny, dtype=np.float64)[:, None]
    t = np.zeros((ny, nx), dtype=np.float64)
    for m in range(modes):
        t += a[m] * np.sin(2.0 * math.pi * (f[m] * i / nx + g[m] * j / ny) + phi[m])
    return t.astype(np.float32)


def differentiation(seed: int = 4, n: int = 2048, steps: int = 200, ckpt: int = 20,
                    ny: int | None = None) -> Grid:
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    u0 = rng.random((ny, n), dtype=np.float32)
    kappa = _uniform(rng, (ny, n), 0.5, 1.0)
    src = np.zeros((ny, n), dtype=np.float32)
    target = smooth_target(rng, n, ny)
    g = Grid(u0, kappa, src, dt_for(kappa, 0.2), steps, DIRICHLET,
             name=f"adjoint-{n}x{ny}-dirichlet-{steps}steps-ckpt{ckpt}")
    g.extras = {"target": target, "ckpt": ckpt}
    return g


def unit_directions(seed: int, count: int, shape) -> np.ndarray:
    """`count` seeded random unit vectors (float64) of the given shape."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((count,) + tuple(shape))
    norms = np.sqrt(np.sum(d.reshape(count, -1) ** 2, axis=1))
    return d / norms.reshape((count,) + (1,) * len(shape))


WORKLOADS = {
    "plain_small": plain_small,
    "plain_scale": plain_scale,
    "precision": precision,
    "batching": batching,
    "differentiation": differentiation,
}
