"""Seeded synthetic inputs for the multi-source Helmholtz solve.

This module builds problem data only: squared-slowness models m = 1/v^2,
the absorbing-layer profile gamma, angular frequencies and point-source
right-hand sides.  It contains none of the solver's arithmetic (no operator,
no transfer, no Krylov step), so both the CPU oracle's tests and the GPU path
may draw their inputs from it.

Conventions
-----------
* A grid of ``n1 x n2 (x n3)`` *cells* has ``N_k = n_k + 1`` nodes per axis;
  the unknowns live on the nodes (Sec. 2.4, second-order finite differences
  on a regular grid).
* Arrays are numpy C-order with the first spatial axis x1 fastest, i.e.
  shape ``(N2, N1)`` in 2D and ``(N3, N2, N1)`` in 3D.  The last spatial axis
  (x2 in 2D, x3 in 3D; numpy axis 0) is depth; node row 0 is the free
  surface, where no absorbing layer is placed (Sec. 5.1 and 5.2 pad every
  side but the top).
* The velocity models stand in for the SEG/EAGE salt model of Sec. 5, which
  is not available: layered media with 1.5--4.5 km/s (the range of the
  paper's figures), optional dipping faults, a salt-like 4.5 km/s ellipse and
  smooth Gaussian anomalies.  Every generator is driven by
  ``numpy.random.Generator(PCG64(seed))``.
* Sources are unit point sources discretised as a finite-volume delta
  (Sec. 2.1, Eq. helm): value ``1/h^d`` at the source node.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.ndimage import gaussian_filter

V_MIN = 1500.0   # m/s, lowest velocity of the synthetic media
V_MAX = 4500.0   # m/s, salt velocity / highest layer velocity


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def node_shape(cells) -> tuple:
    """numpy shape of the node grid for ``cells = (n1, n2[, n3])``."""
    return tuple(int(c) + 1 for c in reversed(tuple(cells)))


def omega_for_ppw(h: float, v_min: float = V_MIN, ppw: float = 10.0) -> float:
    """Angular frequency with ``ppw`` points per wavelength at ``v_min``
    (the rule of Sec. 2.4; Sec. 5.3 uses omega*h/v_min = 2*pi/10)."""
    return 2.0 * math.pi * v_min / (ppw * h)


# --------------------------------------------------------------------------
# velocity models
# --------------------------------------------------------------------------

def _layer_velocity(depth_index: np.ndarray, nz: int, rng, nlayers: int):
    """Piecewise-constant layered velocity as a function of (fractional)
    depth index; interfaces at sorted U(0.1, 0.9) * depth, velocities sorted
    ascending U[1.5, 4.5] km/s."""
    interfaces = np.sort(rng.uniform(0.1, 0.9, nlayers - 1)) * (nz - 1)
    vel = np.sort(rng.uniform(V_MIN, V_MAX, nlayers))
    layer = np.searchsorted(interfaces, depth_index, side="right")
    return vel[layer]


def _smooth_noise(rng, shape, sigma: float) -> np.ndarray:
    """White noise smoothed by a Gaussian of ``sigma`` cells, scaled to
    max |n| = 1."""
    n = gaussian_filter(rng.standard_normal(shape), sigma, mode="nearest")
    return n / np.max(np.abs(n))


def layered_velocity_2d(seed: int, cells=(128, 64), nlayers: int = 4,
                        faults: int = 0, salt: bool = False,
                        noise: float = 0.05) -> np.ndarray:
    """2D layered model (x1 = lateral, x2 = depth), node values in m/s.

    Layers: ``nlayers`` with Gaussian-smoothed interfaces (sigma = 2 cells).
    ``faults`` dipping faults, each with dip U(30, 70) degrees and throw
    U(5, 15)% of the depth, displace the layering on their hanging wall.
    ``salt`` adds a 4.5 km/s ellipse (semi-axes U(40, 90) x U(20, 50) cells,
    centre in the middle third).  The result is multiplied by
    ``1 + noise * n`` with ``n`` smoothed noise (sigma = 3 cells) and clipped to
    [1.5, 4.5] km/s.
    """
    rng = rng_for(seed)
    nz, nx = node_shape(cells)
    z, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")
    zeff = z.copy()
    for _ in range(faults):
        dip = math.radians(rng.uniform(30.0, 70.0))
        throw = rng.uniform(0.05, 0.15) * (nz - 1)
        x0 = rng.uniform(0.2, 0.8) * (nx - 1)
        hanging = x > x0 + z / math.tan(dip)
        zeff = np.where(hanging, zeff - throw, zeff)
    v = _layer_velocity(zeff, nz, rng, nlayers)
    v = gaussian_filter(v, 2.0, mode="nearest")
    if salt:
        a = rng.uniform(40.0, 90.0)
        b = rng.uniform(20.0, 50.0)
        cx = rng.uniform(1.0 / 3.0, 2.0 / 3.0) * (nx - 1)
        cz = rng.uniform(1.0 / 3.0, 2.0 / 3.0) * (nz - 1)
        inside = ((x - cx) / a) ** 2 + ((z - cz) / b) ** 2 <= 1.0
        v = np.where(inside, V_MAX, v)
    if noise:
        v = v * (1.0 + noise * _smooth_noise(rng, v.shape, 3.0))
    return np.clip(v, V_MIN, V_MAX)


def layered_velocity_3d(seed: int, cells=(128, 128, 64), nlayers: int = 4,
                        anomalies: int = 3) -> np.ndarray:
    """3D layered model (x3 = depth) plus ``anomalies`` smooth Gaussian
    anomalies of +-15% with sigma U(8, 16) cells; clipped to [1.5, 4.5] km/s."""
    rng = rng_for(seed)
    nz, ny, nx = node_shape(cells)
    z = np.arange(nz, dtype=np.float64)[:, None, None] * np.ones((1, ny, nx))
    v = _layer_velocity(z, nz, rng, nlayers)
    v = gaussian_filter(v, 2.0, mode="nearest")
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                             indexing="ij")
    for _ in range(anomalies):
        amp = 0.15 * (1.0 if rng.uniform() < 0.5 else -1.0)
        sig = rng.uniform(8.0, 16.0)
        c = [rng.uniform(0.2, 0.8) * (n - 1) for n in (nz, ny, nx)]
        r2 = (zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2
        v = v * (1.0 + amp * np.exp(-r2 / (2.0 * sig * sig)))
    return np.clip(v, V_MIN, V_MAX)


# --------------------------------------------------------------------------
# absorbing layer
# --------------------------------------------------------------------------

def absorbing_gamma(shape, width: int, gamma0: float = 0.0,
                    free_surface: bool = True) -> np.ndarray:
    """Dimensionless attenuation profile on the node grid.

    Inside the boundary layer of ``width`` cells gamma ramps quadratically to
    1 at the outermost node: per axis ``((L - d) / L)^2`` for a node at
    distance ``d < L`` (in nodes) from the outer boundary, maximised over the
    axes, plus the background ``gamma0``.  The top of the depth axis (numpy
    axis 0, index 0) is a free surface without layer.
    """
    g = np.zeros(shape, dtype=np.float64)
    L = float(width)
    for ax, n in enumerate(shape):
        idx = np.arange(n, dtype=np.float64)
        lo = np.where(idx < L, ((L - idx) / L) ** 2, 0.0)
        hi = np.where(n - 1 - idx < L, ((L - (n - 1 - idx)) / L) ** 2, 0.0)
        if ax == 0 and free_surface:
            lo = np.zeros_like(lo)
        prof = np.maximum(lo, hi)
        view = [1] * len(shape)
        view[ax] = n
        g = np.maximum(g, prof.reshape(view))
    return g + gamma0


# --------------------------------------------------------------------------
# sources
# --------------------------------------------------------------------------

def point_sources(shape, positions, h: float) -> np.ndarray:
    """Right-hand sides for unit point sources, ABI layout: float64 complex
    array of shape (s, N) (one contiguous column per source, x1 fastest).
    ``positions`` are numpy node indices (depth index first)."""
    d = len(shape)
    N = int(np.prod(shape))
    q = np.zeros((len(positions), N), dtype=np.complex128)
    for k, p in enumerate(positions):
        q[k, np.ravel_multi_index(tuple(int(c) for c in p), shape)] = 1.0 / h ** d
    return q


def line_positions(shape, count: int, row: int, width: int):
    """``count`` node positions on depth row ``row``, evenly spaced over the
    lateral interior outside the absorbing layer (2D)."""
    nx = shape[-1]
    xs = np.rint(np.linspace(width, nx - 1 - width, count)).astype(int)
    return [(row, int(x)) for x in xs]


def surface_grid_positions(shape, per_axis: int, spacing: int, row: int = 0):
    """``per_axis`` x ``per_axis`` surface grid of node positions, centred,
    ``spacing`` cells apart, on depth row ``row`` (3D)."""
    _, ny, nx = shape
    off_y = (ny - 1) // 2 - spacing * (per_axis - 1) // 2
    off_x = (nx - 1) // 2 - spacing * (per_axis - 1) // 2
    return [(row, off_y + spacing * j, off_x + spacing * i)
            for j in range(per_axis) for i in range(per_axis)]


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclass
class Problem:
    """One Helmholtz problem: model, layer, frequency and sources."""
    name: str
    cells: tuple
    h: float
    omega: float
    m: np.ndarray            # squared slowness on the nodes, numpy node shape
    gamma: np.ndarray        # dimensionless attenuation (layer) on the nodes
    sources: list            # node positions
    shift: float = 0.5       # imaginary shift beta of the preconditioner
    levels: int = 3
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.m.shape

    @property
    def dim(self):
        return len(self.cells)

    @property
    def n_nodes(self):
        return int(self.m.size)

    def rhs(self, columns=None) -> np.ndarray:
        pos = self.sources if columns is None else [self.sources[c] for c in columns]
        return point_sources(self.shape, pos, self.h)


def layered2d_problem(seed: int = 0, cells=(128, 64), h: float = 25.0,
                      width: int = 10, nsrc: int = 8, src_row: int = 2,
                      freq_hz: float | None = None) -> Problem:
    """Small 2D workload: 128x64 cells, h = 25 m, 4 smoothed layers with 5%
    noise, 10-cell layer, 8 sources on node row 2, 10 points per wavelength
    at 1.5 km/s (omega = 37.70 rad/s, 6 Hz), shift 0.5, 3 levels."""
    v = layered_velocity_2d(seed, cells)
    shape = node_shape(cells)
    omega = omega_for_ppw(h) if freq_hz is None else 2 * math.pi * freq_hz
    return Problem("layered2d_%dx%d" % tuple(cells), tuple(cells), h, omega,
                   1.0 / v ** 2, absorbing_gamma(shape, width),
                   line_positions(shape, nsrc, src_row, width), levels=3)


SALT2D_FREQS_HZ = (2.0, 3.5, 5.0, 6.5, 8.0)


def salt2d_problem(seed: int = 0, freq_hz: float = 5.0, cells=(512, 256),
                   h: float = 12.5, width: int = 20, nsrc: int = 64,
                   levels: int = 4) -> Problem:
    """2D faulted layered model with a salt ellipse: 512x256 cells,
    h = 12.5 m, 20-cell layer, 64 sources on the top node row, 4 levels."""
    v = layered_velocity_2d(seed, cells, faults=3, salt=True)
    shape = node_shape(cells)
    return Problem("salt2d_%dx%d" % tuple(cells), tuple(cells), h,
                   2 * math.pi * freq_hz, 1.0 / v ** 2,
                   absorbing_gamma(shape, width),
                   line_positions(shape, nsrc, 0, width), levels=levels,
                   extra={"freq_hz": freq_hz})


def layered3d_problem(seed: int = 0, cells=(128, 128, 64), h: float = 20.0,
                      width: int = 12, freq_hz: float = 4.0, per_axis: int = 16,
                      spacing: int = 8, levels: int = 4) -> Problem:
    """3D layered model with Gaussian anomalies: 128x128x64 cells,
    h = 20 m, 12-cell layer, 16x16 surface sources 8 cells apart, 4 Hz,
    4 levels (coarsest 17x17x9)."""
    v = layered_velocity_3d(seed, cells)
    shape = node_shape(cells)
    return Problem("layered3d_%dx%dx%d" % tuple(cells), tuple(cells), h,
                   2 * math.pi * freq_hz, 1.0 / v ** 2,
                   absorbing_gamma(shape, width),
                   surface_grid_positions(shape, per_axis, spacing), levels=levels)


def random_problem_2d(seed: int, cells, h: float, freq_hz: float,
                      nsrc: int, width: int = 20, levels: int | None = None,
                      salt: bool = True) -> Problem:
    """A 2D faulted/salt problem of any size (used by the uneven batch and
    for the learned stage's training data)."""
    v = layered_velocity_2d(seed, cells, faults=3, salt=salt)
    shape = node_shape(cells)
    if levels is None:
        levels = default_levels(cells)
    w = min(width, min(cells) // 4)
    return Problem("faulted2d_%dx%d" % tuple(cells), tuple(cells), h,
                   2 * math.pi * freq_hz, 1.0 / v ** 2,
                   absorbing_gamma(shape, w),
                   line_positions(shape, nsrc, 0, w), levels=levels,
                   extra={"freq_hz": freq_hz})


def default_levels(cells, max_coarsest: int = 9000) -> int:
    """Fewest levels whose coarsest grid has at most ``max_coarsest`` nodes
    (each coarsening halves the cells per axis)."""
    L = 1
    c = list(cells)
    while np.prod([x + 1 for x in c]) > max_coarsest and all(x % 2 == 0 for x in c):
        c = [x // 2 for x in c]
        L += 1
    return L


def constant_problem(cells, h: float, omega: float, m0: float = 1.0,
                     gamma0: float = 0.0, sources=None, levels: int = 2) -> Problem:
    """Constant medium, uniform gamma, no layer (closed-form test cases)."""
    shape = node_shape(cells)
    m = np.full(shape, m0)
    g = np.full(shape, gamma0)
    if sources is None:
        sources = [tuple(n // 2 for n in shape)]
    return Problem("constant_" + "x".join(map(str, cells)), tuple(cells), h,
                   omega, m, g, sources, levels=levels)
