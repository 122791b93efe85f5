"""Seeded synthetic inputs shared by the GPU path's tests, the oracle's tests and
bench.py.

This module only *draws* inputs: grid and material descriptions of the five
workloads, initial magnetisation states, replica sizes and per-replica
currents.  It holds none of the method's arithmetic (no fields, torques,
integrators or transforms), so the oracle and the CUDA path stay independent.

Every array is float64, shaped (3, nz, ny, nx) for vector fields (component
major, x fastest), matching the state layout described in Methods, "Replica
batching" (replica-outermost, component-major, x-fastest indexing).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    pbc: tuple = (0, 0, 0)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self) -> tuple:
        return (self.nz, self.ny, self.nx)


@dataclass(frozen=True)
class Material:
    """Scalar material parameters (SI).  ``cell`` optionally holds per-cell
    float64 arrays of shape (nz, ny, nx) (``u`` is (3, nz, ny, nx)) that
    override the scalars."""
    Ms: float
    A: float
    alpha: float
    Ku1: float = 0.0
    u: tuple = (0.0, 0.0, 1.0)
    D: float = 0.0
    cell: dict = field(default_factory=dict)
    Db: float = 0.0         # bulk DMI constant (J/m^2)
    Kc1: float = 0.0        # cubic anisotropy (J/m^3)
    Kc2: float = 0.0
    c1: tuple = (1.0, 0.0, 0.0)   # cubic axes (c3 = c1 x c2)
    c2: tuple = (0.0, 1.0, 0.0)
    Ks: float = 0.0         # surface anisotropy at free z faces (J/m^2)
    B1: float = 0.0         # magnetoelastic coupling constants (J/m^3)
    B2: float = 0.0


@dataclass(frozen=True)
class Workload:
    name: str
    grid: Grid
    mat: Material
    B_ext: tuple            # tesla
    integrator: str         # "rk45" | "heun"
    t_end: float            # seconds of simulated time
    rtol: float = 1e-6
    dt: float = 1e-14
    demag: bool = True
    T: float = 0.0
    seed: int = 0


# ---------------------------------------------------------------------------
# The five workloads (sizes and parameters as stated for each benchmark case)
# ---------------------------------------------------------------------------

def film_128x32() -> Workload:
    """Thin-film rectangle 128x32x1 of 3.90625x3.90625x3 nm, FP64, RK45."""
    return Workload(
        name="film_128x32x1_rk45_fp64",
        grid=Grid(128, 32, 1, 3.90625e-9, 3.90625e-9, 3.0e-9),
        mat=Material(Ms=8.0e5, A=1.3e-11, alpha=0.02),
        B_ext=(-24.6e-3, 4.3e-3, 0.0), integrator="rk45", t_end=0.5e-9,
        rtol=1e-6, seed=1)


def dmi_256x256x16() -> Workload:
    """256x256x16 grid of 2 nm cubes with Ku, interfacial DMI, RK45 relaxation."""
    return Workload(
        name="dmi_256x256x16_rk45",
        grid=Grid(256, 256, 16, 2e-9, 2e-9, 2e-9),
        mat=Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0.0, 0.0, 1.0), D=3e-3),
        B_ext=(0.0, 0.0, 0.0), integrator="rk45", t_end=2e-9, rtol=1e-6, seed=2)


def replicas_perp(R: int = 1024) -> list:
    """Perpendicular free layers with sizes drawn from {32..128}^2 x 1, T=300 K,
    damping-like SOT with J per replica in [1e11, 3e11] A/m^2, Heun dt=1e-14."""
    sizes = replica_sizes(R, seed=3)
    J = replica_currents(R)
    out = []
    for r in range(R):
        n = sizes[r]
        out.append(Workload(
            name=f"perp_replica_{r}",
            grid=Grid(n, n, 1, 2e-9, 2e-9, 1e-9),
            mat=Material(Ms=1.1e6, A=2e-11, alpha=0.01, Ku1=9e5, u=(0.0, 0.0, 1.0)),
            B_ext=(0.0, 0.0, 0.0), integrator="heun", t_end=5e-9, dt=1e-14,
            demag=True, T=300.0, seed=3))
    return out, J


def skyrmion_512() -> Workload:
    """512x512x1 film of 2x2x1 nm cells with a DMI skyrmion lattice."""
    return Workload(
        name="skyrmion_512x512x1",
        grid=Grid(512, 512, 1, 2e-9, 2e-9, 1e-9),
        mat=Material(Ms=5.8e5, A=1.5e-11, alpha=0.3, Ku1=8e5, u=(0.0, 0.0, 1.0), D=3.5e-3),
        B_ext=(0.0, 0.0, 0.2), integrator="rk45", t_end=1e-9, rtol=1e-6, seed=4)


def vortex_512x512x64() -> Workload:
    """512x512x64 cells of 3 nm cubes (16.7 M cells), RK45 for 0.2 ns."""
    return Workload(
        name="vortex_512x512x64_rk45",
        grid=Grid(512, 512, 64, 3e-9, 3e-9, 3e-9),
        mat=Material(Ms=8.0e5, A=1.3e-11, alpha=0.02),
        B_ext=(0.0, 0.0, 0.0), integrator="rk45", t_end=0.2e-9, rtol=1e-6, seed=5)


# ---------------------------------------------------------------------------
# Initial states
# ---------------------------------------------------------------------------

def _unit(v: np.ndarray) -> np.ndarray:
    n = np.sqrt((v * v).sum(axis=0, keepdims=True))
    return v / np.where(n > 0, n, 1.0)


def m_uniform_perturbed(grid: Grid, direction=(1.0, 1.0, 1.0), amp=0.05, seed=1) -> np.ndarray:
    """Uniform direction plus a seeded uniform perturbation of amplitude
    ``amp`` on every component, then renormalised."""
    rng = np.random.default_rng(seed)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    m = np.broadcast_to(d[:, None, None, None], (3,) + grid.shape).copy()
    m += amp * rng.uniform(-1.0, 1.0, size=m.shape)
    return _unit(m)


def m_random_sphere(grid: Grid, seed=2) -> np.ndarray:
    """Independent unit vectors uniform on the sphere (z ~ U(-1,1), phi ~ U(0,2pi))."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1.0, 1.0, size=grid.shape)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=grid.shape)
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z])


def m_vortex(grid: Grid, seed=5, core_radius=10e-9, noise=0.01) -> np.ndarray:
    """One vortex at a seeded centre in the middle half of the film, seeded
    chirality and polarity, identical in every layer, plus seeded noise."""
    rng = np.random.default_rng(seed)
    Lx, Ly = grid.nx * grid.dx, grid.ny * grid.dy
    cx = rng.uniform(0.25, 0.75) * Lx
    cy = rng.uniform(0.25, 0.75) * Ly
    chir = rng.choice([-1.0, 1.0])
    pol = rng.choice([-1.0, 1.0])
    x = (np.arange(grid.nx) + 0.5) * grid.dx - cx
    y = (np.arange(grid.ny) + 0.5) * grid.dy - cy
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X, Y)
    mz = pol * np.exp(-(r / core_radius) ** 2)
    inplane = np.sqrt(np.clip(1.0 - mz * mz, 0.0, 1.0))
    phi = np.arctan2(Y, X)
    mx = -chir * np.sin(phi) * inplane
    my = chir * np.cos(phi) * inplane
    m = np.stack([np.broadcast_to(c, grid.shape) for c in (mx, my, mz)]).copy()
    m += noise * rng.uniform(-1.0, 1.0, size=m.shape)
    return _unit(m)


def m_skyrmion_lattice(grid: Grid, seed=4, spacing=40e-9, radius=8e-9) -> np.ndarray:
    """Background +z with reversed (-z) seeded bubbles on a jittered
    triangular lattice: a starting point from which DMI relaxes skyrmions."""
    rng = np.random.default_rng(seed)
    x = (np.arange(grid.nx) + 0.5) * grid.dx
    y = (np.arange(grid.ny) + 0.5) * grid.dy
    X, Y = np.meshgrid(x, y)
    mz = np.ones_like(X)
    mx = np.zeros_like(X)
    my = np.zeros_like(X)
    Lx, Ly = grid.nx * grid.dx, grid.ny * grid.dy
    row = 0
    yc = spacing / 2
    while yc < Ly:
        xc = spacing / 2 + (spacing / 2 if row % 2 else 0.0)
        while xc < Lx:
            jx, jy = rng.uniform(-0.2, 0.2, size=2) * spacing
            dxp, dyp = X - (xc + jx), Y - (yc + jy)
            r = np.hypot(dxp, dyp)
            theta = math.pi * np.exp(-(r / radius) ** 2)   # pi at the core, 0 far away
            sel = r < 3 * radius
            mz = np.where(sel, np.cos(theta), mz)
            mx = np.where(sel, np.sin(theta) * dxp / np.maximum(r, 1e-30), mx)
            my = np.where(sel, np.sin(theta) * dyp / np.maximum(r, 1e-30), my)
            xc += spacing
        yc += spacing * math.sqrt(3) / 2
        row += 1
    m = np.stack([np.broadcast_to(c, grid.shape) for c in (mx, my, mz)]).copy()
    m += 0.01 * rng.uniform(-1.0, 1.0, size=m.shape)
    return _unit(m)


def m_perp(grid: Grid, seed=0, tilt=0.05) -> np.ndarray:
    """Perpendicular (+z) state with a small seeded tilt on every cell."""
    return m_uniform_perturbed(grid, direction=(0.0, 0.0, 1.0), amp=tilt, seed=seed)


def replica_sizes(R: int, seed=3) -> list:
    """Square edge lengths drawn uniformly from {32, 48, 64, 96, 128}."""
    rng = np.random.default_rng(seed)
    choices = np.array([32, 48, 64, 96, 128])
    return [int(v) for v in rng.choice(choices, size=R)]


def replica_currents(R: int, lo=1e11, hi=3e11) -> np.ndarray:
    """Current density per replica, linear in replica index over [lo, hi]."""
    if R == 1:
        return np.array([lo])
    return lo + (hi - lo) * np.arange(R) / (R - 1)


def replica_seeds(R: int, base=3) -> np.ndarray:
    """Distinct 64-bit Philox seeds per replica, drawn from one seeded stream."""
    rng = np.random.default_rng(base)
    return rng.integers(0, 2**63 - 1, size=R, dtype=np.int64).astype(np.uint64)


def random_m(grid: Grid, seed: int) -> np.ndarray:
    return m_random_sphere(grid, seed=seed)


def random_material_cells(grid: Grid, seed: int, n_regions=3, with_holes=True) -> dict:
    """Per-cell material arrays drawn from a handful of seeded materials (a
    granular film), optionally with Ms=0 holes (absent cells)."""
    rng = np.random.default_rng(seed)
    region = rng.integers(0, n_regions, size=grid.shape)
    Ms = rng.uniform(4e5, 1.2e6, size=n_regions)
    A = rng.uniform(0.8e-11, 2e-11, size=n_regions)
    alpha = rng.uniform(0.01, 0.3, size=n_regions)
    Ku = rng.uniform(0.0, 8e5, size=n_regions)
    D = rng.uniform(0.0, 3e-3, size=n_regions)
    u = rng.normal(size=(3, n_regions))
    u /= np.linalg.norm(u, axis=0, keepdims=True)
    cells = {
        "Ms": Ms[region], "A": A[region], "alpha": alpha[region],
        "Ku1": Ku[region], "D": D[region], "u": u[:, region],
    }
    if with_holes:
        hole = rng.uniform(size=grid.shape) < 0.08
        cells["Ms"] = np.where(hole, 0.0, cells["Ms"])
    return cells


def with_cells(mat: Material, cells: dict) -> Material:
    return replace(mat, cell=dict(cells))
