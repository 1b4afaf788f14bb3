"""Seeded synthetic workloads (the only module both the CUDA path and the CPU oracle consume).

This module holds geometry, loads and random draws only -- none of the peridynamic arithmetic.  Every
quantity the method derives (A, K, G, m_i, s0 from G0, the stable time step) is computed by each
implementation itself; ``s0`` is left to the caller (``Workload.Gc`` is the input), and the time steps
below are literals whose derivation is pinned by the oracle tests.

Geometry conventions: particles sit at cell centres of a uniform grid, x = (i + 1/2) dx, caller order
is i fastest, then j, then k.  2D volumes are dx^2 (unit thickness; the thickness cancels from u, v
and damage), 3D volumes dx^3.  The recipes follow the paper's workloads in shape (Section 4: plane
stress plates with a pre-crack under edge traction, Section 4.2; a notched 3D block under torsion,
Section 4.4) with the sizes of the five benchmark configurations.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

MODEL_3D, MODEL_PLANE_STRESS, MODEL_PLANE_STRAIN = 0, 1, 2
FREE, FIXED, PRESCRIBED = 0, 1, 2


@dataclass
class Workload:
    name: str
    model: int
    E: float
    nu: float
    rho: float
    dx: float
    delta: float
    dt: float
    nsteps: int
    x: np.ndarray
    y: np.ndarray
    z: Optional[np.ndarray]
    vol: np.ndarray
    Gc: Optional[float] = None            # critical energy release rate; None -> no bond breaking
    cracks: List[tuple] = field(default_factory=list)   # 9 doubles each (p0, p1, p2)
    flag: Optional[np.ndarray] = None     # uint8 per particle: 0 free, 1 fixed, 2 prescribed
    b: Optional[np.ndarray] = None        # (dim, n) body-force density [N/m^3]
    axis_point: Optional[np.ndarray] = None
    axis_dir: Optional[np.ndarray] = None
    twist_in_s0: float = 0.0              # prescribed total rotation angle, in units of s0
    u0: Optional[np.ndarray] = None       # (dim, n)
    v0: Optional[np.ndarray] = None
    vp: Optional[np.ndarray] = None       # (dim, n) prescribed velocity of the prescribed particles

    @property
    def n(self) -> int:
        return int(self.x.size)

    @property
    def dim(self) -> int:
        return 3 if self.z is not None else 2

    def rotation_rate(self, s0: float) -> float:
        """Angular rate so that the prescribed end reaches ``twist_in_s0 * s0`` radians at the end."""
        if self.twist_in_s0 == 0.0:
            return 0.0
        return self.twist_in_s0 * s0 / (self.nsteps * self.dt)

    def initial_u(self) -> np.ndarray:
        return np.zeros((self.dim, self.n)) if self.u0 is None else self.u0

    def initial_v(self) -> np.ndarray:
        return np.zeros((self.dim, self.n)) if self.v0 is None else self.v0


def grid_2d(nx: int, ny: int, dx: float):
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    x = (i.reshape(-1) + 0.5) * dx
    y = (j.reshape(-1) + 0.5) * dx
    return x.astype(np.float64), y.astype(np.float64)


def grid_3d(nx: int, ny: int, nz: int, dx: float):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x = (i.reshape(-1) + 0.5) * dx
    y = (j.reshape(-1) + 0.5) * dx
    z = (k.reshape(-1) + 0.5) * dx
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


# ---- material of configurations 1, 2, 4 (soda-lime glass) and 3, 5 (concrete-like) -------------
GLASS = dict(E=72e9, nu=0.22, rho=2440.0)
CONCRETE = dict(E=30e9, nu=0.2, rho=2400.0)


def plate_vibration(nx: int = 40, ny: int = 40, dx: float = 1e-3, ratio: float = 3.015,
                    seed: int = 0, amp: float = 1e-6, nsteps: int = 1000,
                    dt: float = 2.6954e-7) -> Workload:
    """Configuration 1: plane-stress square plate, free vibration from a random displacement.

    u0 ~ N(0, amp) per component (numpy default_rng(seed)); no constraints, loads or breaking.
    dt = 0.8 x the stable bound 2/sqrt(lambda_max(M^-1 K)) for 40x40, ratio 3.015, nu = 0.22 (the
    literal is pinned by tests/test_oracle_pins.py::test_stable_dt_config1).
    """
    x, y = grid_2d(nx, ny, dx)
    rng = np.random.default_rng(seed)
    u0 = rng.normal(0.0, amp, size=(2, x.size))
    return Workload("plate_vibration_%dx%d" % (nx, ny), MODEL_PLANE_STRESS, dx=dx, delta=ratio * dx,
                    dt=dt, nsteps=nsteps, x=x, y=y, z=None, vol=np.full(x.size, dx * dx), u0=u0,
                    **GLASS)


def cracked_plate(nx: int = 400, ny: int = 160, dx: float = 2.5e-4, ratio: float = 3.015,
                  sigma: float = 1e6, Gc: float = 3.8, crack_cells: float = 200.125,
                  nsteps: int = 5000, dt: float = 6.7385e-8) -> Workload:
    """Configuration 2: plane-stress plate with a central edge pre-crack under edge traction.

    The crack lies on y = (ny/2) dx (between two particle rows) from outside the left edge to
    x = crack_cells * dx (0.05003 m for the defaults; the 1/8-cell offset keeps every bond crossing
    point at least dx/24 away from the tip).  The traction sigma acts on the outermost rows as the
    body-force density +-sigma/dx (top +y, bottom -y), constant from t = 0 (Section 4.2 keeps the
    traction constant).
    """
    x, y = grid_2d(nx, ny, dx)
    n = x.size
    yc = 0.5 * ny * dx
    crack = (-dx, yc, 0.0, crack_cells * dx, yc, 0.0, 0.0, 0.0, 0.0)
    b = np.zeros((2, n))
    j = np.arange(n) // nx
    b[1, j == ny - 1] = sigma / dx
    b[1, j == 0] = -sigma / dx
    return Workload("cracked_plate_%dx%d" % (nx, ny), MODEL_PLANE_STRESS, dx=dx, delta=ratio * dx,
                    dt=dt, nsteps=nsteps, x=x, y=y, z=None, vol=np.full(n, dx * dx), Gc=Gc,
                    cracks=[crack], b=b, **GLASS)


def kalthoff(nx: int = 402, ny: int = 201, dx: float = 5e-4, ratio: float = 3.015, v_imp: float = 22.0,
             notch_cells: float = 100.125, gap_cells: int = 100, layers: int = 3, Gc: float = 6.9e4,
             nsteps: int = 5000, dt: float = 2e-8) -> Workload:
    """Kalthoff-Winkler-like plane-strain impact (Section 4.3's workload in shape; the figure with its
    geometry is not in the text): steel (E 190 GPa, nu 0.25, rho 7800, G0 6.9e4 J/m^2), delta =
    3.015 dx (the paper's 3 dx puts lattice points exactly on the horizon, where membership would
    depend on rounding), nx x ny particles (402 x 201 = 80,802 for the defaults, the paper's node
    count).  Two edge notches
    run from outside the left edge to x = notch_cells * dx on the lattice lines y = yc +- gap_cells/2 dx
    (yc the lattice line nearest the centre; particles sit at cell centres, so no particle lies on a
    notch); the first `layers` columns between the notches move at the constant velocity v_imp along +x
    from t = 0 (prescribed velocity); everything else is free.
    """
    x, y = grid_2d(nx, ny, dx)
    n = x.size
    jc = ny // 2
    ylo, yhi = (jc - gap_cells // 2) * dx, (jc + gap_cells // 2) * dx
    cracks = [(-dx, yl, 0.0, notch_cells * dx, yl, 0.0, 0.0, 0.0, 0.0) for yl in (ylo, yhi)]
    i = np.arange(n) % nx
    hit = (i < layers) & (y > ylo) & (y < yhi)
    flag = np.where(hit, PRESCRIBED, FREE).astype(np.uint8)
    vp = np.zeros((2, n))
    vp[0, hit] = v_imp
    return Workload("kalthoff_%dx%d" % (nx, ny), MODEL_PLANE_STRAIN, E=190e9, nu=0.25, rho=7800.0, dx=dx,
                    delta=ratio * dx, dt=dt, nsteps=nsteps, x=x, y=y, z=None, vol=np.full(n, dx * dx), Gc=Gc,
                    cracks=cracks, flag=flag, axis_point=np.zeros(3), axis_dir=np.array([0.0, 0.0, 1.0]), vp=vp)


def notched_block(nx: int = 200, ny: int = 100, nz: int = 50, dx: float = 1e-3,
                  ratio: float = 3.015, Gc: float = 50.0, nsteps: int = 2000,
                  dt: float = 3.790e-7, seed: Optional[int] = None, amp: float = 0.0,
                  notch_cells: Optional[float] = None) -> Workload:
    """Configurations 3 and 5: 3D block, 45-degree through-notch, one end clamped, the other twisted.

    Notch: the plane (x - z) = c dx with c = notch_cells, a half-integer (default
    floor(0.3775 nx) + 0.5: 75.5 for nx = 200, 151.5 for nx = 400) so no particle lies on it; it
    runs through the whole
    thickness z and from y = ny dx down to y = 0.7537 ny dx (a quarter of the height, the 0.0037
    offset keeps every crossing point away from the notch front).  Clamp: the 3 particle layers
    i < 3 are fixed.  Twist: the 3 layers i >= nx - 3 rotate rigidly about the x axis through the
    section centre; total angle 24 s0 reached at the last step (linearized rotation).
    Optional random initial displacement (seed, amp) for parity tests.
    """
    x, y, z = grid_3d(nx, ny, nz, dx)
    n = x.size
    c = float(np.floor(0.3775 * nx) + 0.5) if notch_cells is None else float(notch_cells)
    ylo = 0.7537 * ny
    p0 = np.array([(c - 1.0) * dx, ylo * dx, -dx])
    e1 = np.array([(nz + 2.0) * dx, 0.0, (nz + 2.0) * dx])
    e2 = np.array([0.0, (ny + 1.0 - ylo) * dx, 0.0])
    crack = tuple(p0) + tuple(p0 + e1) + tuple(p0 + e2)
    i = np.arange(n) % nx
    flag = np.zeros(n, dtype=np.uint8)
    flag[i < 3] = FIXED
    flag[i >= nx - 3] = PRESCRIBED
    u0 = None
    if seed is not None:
        u0 = np.random.default_rng(seed).normal(0.0, amp, size=(3, n))
        u0[:, flag != FREE] = 0.0
    return Workload("notched_block_%dx%dx%d" % (nx, ny, nz), MODEL_3D, dx=dx, delta=ratio * dx,
                    dt=dt, nsteps=nsteps, x=x, y=y, z=z, vol=np.full(n, dx ** 3), Gc=Gc,
                    cracks=[crack], flag=flag, axis_point=np.array([0.0, 0.5 * ny * dx, 0.5 * nz * dx]),
                    axis_dir=np.array([1.0, 0.0, 0.0]), twist_in_s0=24.0, u0=u0, **CONCRETE)


def config1() -> Workload:
    return plate_vibration()


def config2() -> Workload:
    return cracked_plate()


def config3() -> Workload:
    return notched_block()


def config5() -> Workload:
    return notched_block(nx=400, ny=200, nz=100, dx=5e-4, nsteps=1000, dt=1.895e-7)


# ---- configuration 4: batch of independent plates ------------------------------------------------
# Lower bound of the stable-step coefficient C in dt_crit = C dx sqrt(rho/E) over nu in [0.1, 0.45]
# for plane stress at horizon ratios 3.015 and 4.015 (pinned against the oracle's lambda_max by
# tests/test_oracle_pins.py::test_batch_dt_coefficients).
BATCH_DT_COEF = {3.015: 1.70, 4.015: 2.20}


@dataclass
class BatchWorkload:
    name: str
    model: int
    bodies: List[Workload]
    offsets: np.ndarray          # int64[nbodies + 1]

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    def concat(self, attr: str):
        return np.concatenate([getattr(w, attr) for w in self.bodies])


def plate_batch(nplates: int = 256, seed: int = 1, dx: float = 2.5e-4, side_lo: int = 20,
                side_hi: int = 200, Gc: float = 3.8, nsteps: int = 1000) -> BatchWorkload:
    """Configuration 4: independent plane-stress plates with uneven sizes and materials.

    Per plate (numpy default_rng(seed), drawn in this order): nx, ny ~ U{side_lo..side_hi};
    E ~ U[20, 200] GPa; nu ~ U[0.1, 0.45]; horizon ratio 3.015 or 4.015 (p = 1/2); edge traction
    sigma ~ U[0.5, 5] MPa on the top and bottom rows.  No pre-crack; rho = 2440; G0 = Gc.
    dt = 0.8 BATCH_DT_COEF[ratio] dx sqrt(rho / E).
    """
    rng = np.random.default_rng(seed)
    bodies = []
    offsets = [0]
    for p in range(nplates):
        nx = int(rng.integers(side_lo, side_hi + 1))
        ny = int(rng.integers(side_lo, side_hi + 1))
        E = float(rng.uniform(20e9, 200e9))
        nu = float(rng.uniform(0.1, 0.45))
        ratio = 3.015 if rng.random() < 0.5 else 4.015
        sigma = float(rng.uniform(0.5e6, 5e6))
        rho = 2440.0
        dt = 0.8 * BATCH_DT_COEF[ratio] * dx * np.sqrt(rho / E)
        x, y = grid_2d(nx, ny, dx)
        n = x.size
        b = np.zeros((2, n))
        j = np.arange(n) // nx
        b[1, j == ny - 1] = sigma / dx
        b[1, j == 0] = -sigma / dx
        bodies.append(Workload("plate%d" % p, MODEL_PLANE_STRESS, E=E, nu=nu, rho=rho, dx=dx,
                               delta=ratio * dx, dt=dt, nsteps=nsteps, x=x, y=y, z=None,
                               vol=np.full(n, dx * dx), Gc=Gc, b=b))
        offsets.append(offsets[-1] + n)
    return BatchWorkload("plate_batch_%d" % nplates, MODEL_PLANE_STRESS, bodies,
                         np.asarray(offsets, dtype=np.int64))


def config4() -> BatchWorkload:
    return plate_batch()
