"""Seeded synthetic dam-break inputs (the test case of the paper's Section 2, Fig. 2).

This module builds INPUT DATA only: particle positions, initial velocities, the
hydrostatic initial density and the run constants.  It is shared by the FP64
oracle (``oracle/``) and by the CUDA library (``paper_1110_3711_gb300``) and holds
none of the method's arithmetic (no neighbour search, kernel, equation of state
for the update, integration or time step).

The paper does not print its geometry, so the recipe below is a stated reading:

* Tank interior ``[0, Lx] x [0, Ly] x [0, Lz]`` with ``Lx = round(1.6/dp)*dp``,
  ``Ly = floor(0.67/dp)*dp`` and ``Lz = round(0.4/dp)*dp``; no lid.
* Water column ``0.4 x 0.67 x 0.3`` m against the ``x = 0`` wall, filled with a
  cubic lattice ``((i+1/2)dp, (j+1/2)dp, (k+1/2)dp)``.
* Two staggered layers of fixed ("dynamic", Table 1) boundary particles on the
  floor and the four walls: layer 1 on the wall planes at integer multiples of
  ``dp``; layer 2 shifted by ``dp/2`` in the plane and ``dp/2`` outwards.  Points
  shared by two planes are kept once (built on an exact half-``dp`` integer grid).
* Mass ``m = rho0 * dp**3`` for every particle.
* Initial density is hydrostatic for fluid and submerged boundary particles:
  ``rho(z) = rho0 * (1 + rho0*g*(H - z)/B)**(1/gamma)`` with ``H = nz*dp`` (top of
  the lattice), ``B = c0**2 rho0 / gamma`` and depth clipped at 0, so that the
  Tait pressure of the initial state is ``rho0*g*depth``.
* Velocities are zero, plus (optionally) a seeded ``N(0, sigma)`` perturbation on
  every fluid component.

Run constants follow Table 1 and the dam-break configuration: cubic spline with
``h = 0.866*sqrt(3)*dp`` (support and cell size ``2h``), Tait ``gamma = 7``,
``c0 = 10*sqrt(g*0.3)``, artificial viscosity ``alpha = 0.1`` (Table 1 prints 0.25,
kept as a variant), ``eta^2 = 0.01 h^2``, CFL 0.2, Verlet with an Euler step every
40 steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

G = 9.81


@dataclass
class RunParams:
    """Flat run constants (SI).  Field order is the C-ABI's ``sph_params``."""
    dp: float
    h: float
    cell_size: float
    rho0: float = 1000.0
    gamma: float = 7.0
    c0: float = 10.0 * math.sqrt(G * 0.3)
    alpha: float = 0.1
    eta2_coef: float = 0.01
    cfl: float = 0.2
    mass: float = 0.0
    g: tuple = (0.0, 0.0, -G)
    dom_min: tuple = (0.0, 0.0, 0.0)
    dom_max: tuple = (0.0, 0.0, 0.0)
    verlet_euler_every: int = 40
    fixed_dt: float = 0.0
    clamp_boundary_rho: int = 1
    tensile_eps: float = 0.0     # tensile correction for negative pressures (0: off)
    tensile_pos: float = 0.0     # ... for two positive pressures
    tensile_n: int = 4           # exponent of W(r)/W(dp)

    def as_dict(self):
        return asdict(self)


@dataclass
class Case:
    """One synthetic input: fluid particles first, then boundary particles."""
    params: RunParams
    n_f: int
    n_b: int
    pos: np.ndarray          # [N, 3] float64
    vel: np.ndarray          # [N, 3] float64 (boundary rows are zero)
    rho: np.ndarray          # [N] float64
    tank: tuple = (0.0, 0.0, 0.0)
    column: tuple = (0, 0, 0)  # fluid lattice counts (nx, ny, nz)
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.n_f + self.n_b


def _count(length: float, dp: float) -> int:
    """floor(length/dp) that is robust to the rounding of the quotient."""
    return int(math.floor(length / dp + 1e-9))


def _boundary_half_units(X: int, Y: int, Z: int) -> np.ndarray:
    """Boundary points in units of dp/2 (exact integers), duplicates removed."""
    pts = []
    # layer 1: on the planes, integer multiples of dp  -> even half-units
    i = np.arange(X + 1)
    j = np.arange(Y + 1)
    k = np.arange(Z + 1)
    I, J = np.meshgrid(i, j, indexing="ij")
    pts.append(np.stack([2 * I, 2 * J, 0 * I], -1).reshape(-1, 3))          # floor
    J2, K2 = np.meshgrid(j, k, indexing="ij")
    pts.append(np.stack([0 * J2, 2 * J2, 2 * K2], -1).reshape(-1, 3))       # x = 0
    pts.append(np.stack([0 * J2 + 2 * X, 2 * J2, 2 * K2], -1).reshape(-1, 3))  # x = Lx
    I3, K3 = np.meshgrid(i, k, indexing="ij")
    pts.append(np.stack([2 * I3, 0 * I3, 2 * K3], -1).reshape(-1, 3))       # y = 0
    pts.append(np.stack([2 * I3, 0 * I3 + 2 * Y, 2 * K3], -1).reshape(-1, 3))  # y = Ly
    # layer 2: shifted by dp/2 in plane and dp/2 outwards -> odd half-units
    i2 = np.arange(-1, X + 1)
    j2 = np.arange(-1, Y + 1)
    k2 = np.arange(-1, Z)
    I, J = np.meshgrid(i2, j2, indexing="ij")
    pts.append(np.stack([2 * I + 1, 2 * J + 1, 0 * I - 1], -1).reshape(-1, 3))
    J2, K2 = np.meshgrid(j2, k2, indexing="ij")
    pts.append(np.stack([0 * J2 - 1, 2 * J2 + 1, 2 * K2 + 1], -1).reshape(-1, 3))
    pts.append(np.stack([0 * J2 + 2 * X + 1, 2 * J2 + 1, 2 * K2 + 1], -1).reshape(-1, 3))
    I3, K3 = np.meshgrid(i2, k2, indexing="ij")
    pts.append(np.stack([2 * I3 + 1, 0 * I3 - 1, 2 * K3 + 1], -1).reshape(-1, 3))
    pts.append(np.stack([2 * I3 + 1, 0 * I3 + 2 * Y + 1, 2 * K3 + 1], -1).reshape(-1, 3))
    allp = np.concatenate(pts, 0).astype(np.int64)
    # unique rows, then a deterministic order: z, then y, then x (x fastest)
    allp = np.unique(allp, axis=0)
    order = np.lexsort((allp[:, 0], allp[:, 1], allp[:, 2]))
    return allp[order]


def dam_break(dp: float, *, seed: int = 0, vel_sigma: float = 0.0,
              alpha: float = 0.1, fixed_dt: float = 0.0,
              tank=(1.6, 0.67, 0.4), column=(0.4, 0.67, 0.3),
              h_coef: float = 0.866 * math.sqrt(3.0)) -> Case:
    """Build the 3D dam break at lattice spacing ``dp`` (see the module docstring)."""
    rho0, gamma = 1000.0, 7.0
    c0 = 10.0 * math.sqrt(G * 0.3)
    h = h_coef * dp
    s = 2.0 * h
    X = int(round(tank[0] / dp))
    Y = _count(tank[1], dp)
    Z = int(round(tank[2] / dp))
    Lx, Ly, Lz = X * dp, Y * dp, Z * dp
    nx, ny, nz = _count(column[0], dp), _count(column[1], dp), _count(column[2], dp)
    ny = min(ny, Y)
    # fluid lattice, x fastest
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    fpos = np.stack([(ii + 0.5) * dp, (jj + 0.5) * dp, (kk + 0.5) * dp], -1).reshape(-1, 3)
    bpos = _boundary_half_units(X, Y, Z).astype(np.float64) * (0.5 * dp)
    pos = np.concatenate([fpos, bpos], 0)
    n_f, n_b = fpos.shape[0], bpos.shape[0]
    H = nz * dp
    B = c0 * c0 * rho0 / gamma
    depth = np.clip(H - pos[:, 2], 0.0, None)
    rho = rho0 * (1.0 + rho0 * G * depth / B) ** (1.0 / gamma)
    vel = np.zeros_like(pos)
    if vel_sigma > 0.0:
        rng = np.random.default_rng(seed)
        vel[:n_f] = rng.normal(0.0, vel_sigma, size=(n_f, 3))
    params = RunParams(
        dp=dp, h=h, cell_size=s, rho0=rho0, gamma=gamma, c0=c0, alpha=alpha,
        mass=rho0 * dp ** 3, g=(0.0, 0.0, -G),
        dom_min=(-2.0 * s, -2.0 * s, -2.0 * s),
        dom_max=(Lx + 2.0 * s, Ly + 2.0 * s, 2.0 * Lz),
        fixed_dt=fixed_dt)
    return Case(params=params, n_f=n_f, n_b=n_b, pos=pos, vel=vel, rho=rho,
                tank=(Lx, Ly, Lz), column=(nx, ny, nz),
                meta=dict(dp=dp, H=H, seed=seed, vel_sigma=vel_sigma))


def wall_sensors(case: Case, *, wall: str = "back", n_y: int = 8, n_z: int = 8,
                 z_top: float = 0.3, inset: float = 1.5) -> np.ndarray:
    """Sensor points ``inset*dp`` inside a wall, on an ``n_y x n_z`` grid.

    ``wall="back"`` is the ``x = 0`` wall behind the column; ``wall="far"`` is the
    ``x = Lx`` wall the front moves towards.
    """
    Lx, Ly, _ = case.tank
    dp = case.params.dp
    x = inset * dp if wall == "back" else Lx - inset * dp
    ys = (np.arange(n_y) + 0.5) * Ly / n_y
    zs = (np.arange(n_z) + 0.5) * z_top / n_z
    Z, Yg = np.meshgrid(zs, ys, indexing="ij")
    return np.stack([np.full(Z.size, x), Yg.reshape(-1), Z.reshape(-1)], -1)


def still_tank(dp: float, *, depth: float = 0.1, width=(0.2, 0.2)) -> Case:
    """A small tank filled to ``depth`` over its whole floor (no dam), for the
    hydrostatic pin."""
    return dam_break(dp, tank=(width[0], width[1], 2.0 * depth),
                     column=(width[0], width[1], depth))


def uniform_block(n_side: int, dp: float, *, seed: int = 0, vel_sigma: float = 0.0,
                  rho_sigma: float = 0.0, jitter: float = 0.0) -> Case:
    """A cube of ``n_side**3`` fluid particles, no boundaries and no gravity."""
    h = 0.866 * math.sqrt(3.0) * dp
    s = 2.0 * h
    rng = np.random.default_rng(seed)
    kk, jj, ii = np.meshgrid(*(np.arange(n_side),) * 3, indexing="ij")
    pos = np.stack([(ii + 0.5) * dp, (jj + 0.5) * dp, (kk + 0.5) * dp], -1).reshape(-1, 3)
    if jitter > 0.0:
        pos = pos + rng.uniform(-jitter * dp, jitter * dp, size=pos.shape)
    n = pos.shape[0]
    vel = rng.normal(0.0, vel_sigma, size=(n, 3)) if vel_sigma > 0 else np.zeros((n, 3))
    rho = np.full(n, 1000.0)
    if rho_sigma > 0:
        rho = rho * (1.0 + rng.normal(0.0, rho_sigma, size=n))
    L = n_side * dp
    params = RunParams(dp=dp, h=h, cell_size=s, mass=1000.0 * dp ** 3,
                       g=(0.0, 0.0, 0.0),
                       dom_min=(-2.0 * s, -2.0 * s, -2.0 * s),
                       dom_max=(L + 2.0 * s, L + 2.0 * s, L + 2.0 * s))
    return Case(params=params, n_f=n, n_b=0, pos=pos, vel=vel, rho=rho,
                tank=(L, L, L), column=(n_side, n_side, n_side))


def random_cloud(n: int, *, box: float = 0.1, dp: float = 0.01, n_b: int = 0,
                 seed: int = 0, vel_sigma: float = 0.1, rho_sigma: float = 0.01) -> Case:
    """Uniformly random particles in a cube (the last ``n_b`` are boundary)."""
    h = 0.866 * math.sqrt(3.0) * dp
    s = 2.0 * h
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, box, size=(n, 3))
    vel = rng.normal(0.0, vel_sigma, size=(n, 3))
    vel[n - n_b:] = 0.0
    rho = 1000.0 * (1.0 + np.abs(rng.normal(0.0, rho_sigma, size=n)))
    params = RunParams(dp=dp, h=h, cell_size=s, mass=1000.0 * dp ** 3,
                       dom_min=(-s, -s, -s), dom_max=(box + s, box + s, box + s))
    return Case(params=params, n_f=n - n_b, n_b=n_b, pos=pos, vel=vel, rho=rho,
                tank=(box, box, box))


# The five run configurations (dam break at several resolutions).
CONFIGS = {
    "dam10k": dict(dp=0.02, steps=100, precision="fp64"),
    "dam1m": dict(dp=0.005, steps=1000, precision="fp32"),
    "dam5m": dict(dp=0.0025, steps=200, precision="fp32"),
    "damgrad": dict(dp=0.01, steps=400, precision="fp64", fixed_dt=1e-4,
                    vel_sigma=0.05, checkpoint_every=20),
    "dam20m": dict(dp=0.0016, steps=500, precision="fp32"),
}


def small_dam(dp: float = 0.02, *, seed: int = 0, vel_sigma: float = 0.05) -> Case:
    """A small dam break (tank 0.3 x 0.12 x 0.24 m, column 0.1 x 0.12 x 0.12 m)
    with a seeded velocity perturbation: the case the gradient oracle runs."""
    return dam_break(dp, seed=seed, vel_sigma=vel_sigma, tank=(0.3, 0.12, 0.24),
                     column=(0.1, 0.12, 0.12))
