"""Seeded synthetic inputs for the microscale kinetic step.

This module is the only code shared by the CUDA path and the CPU oracle. It
holds no arithmetic of the method itself: it draws random numbers, lays out
initial filament densities and prescribed velocity fields, and picks ensemble
parameters. Both sides receive what it produces as plain float64 arrays.

Layouts (row-major, C order):
    psi  [ny][nx][ntheta]        filament density Psi(x, theta) (Sec. 2, Eq. 1)
    u    [2][ny][nx]             in-plane fluid velocity u_2 at cell centres
    mtot [ny][nx]                total motor density M (Eq. 6)

The generator is splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014); a uniform double in [0, 1) is
the top 53 bits of one 64-bit draw times 2**-53.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """Counter-based splitmix64 stream (state += golden gamma, then mix)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        """n uniforms in [0,1), vectorised splitmix64 (same sequence as uniform())."""
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(self.GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * self.GAMMA) & _MASK
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass(frozen=True)
class Grid:
    """Uniform grid of the unit periodic square, orientation circle and arclength."""

    nx: int
    ny: int
    ntheta: int
    ns: int
    L: float = 1.0

    @property
    def ncells(self) -> int:
        return self.nx * self.ny

    @property
    def micro_cells(self) -> int:
        return self.nx * self.ny * self.ntheta * self.ns


@dataclass(frozen=True)
class Rates:
    """Nondimensional rates and couplings (defaults: the workloads' values).

    glide = 0.05 and v_sp = 0 make the gliding speed depend on the bound-motor
    number per filament; force_scale and ell scale the motor force and force
    dipole (Eq. 10).
    """

    v_walk: float = 1.0
    k_on: float = 1.0
    k_off: float = 0.5
    glide: float = 0.05
    v_sp: float = 0.0
    force_scale: float = 1.0
    ell: float = 1.0
    cfl: float = 0.4


def cell_centres(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def psi_isotropic_perturbed(grid: Grid, seed: int, amp: float = 0.05) -> np.ndarray:
    """psi = psibar (1 + amp xi), xi ~ U(-1,1) i.i.d. in [iy][ix][k] order,
    then rescaled so that sum(psi) dx dy dtheta = 1 (total filament number 1)."""
    rng = SplitMix64(seed)
    xi = 2.0 * rng.uniforms(grid.ny * grid.nx * grid.ntheta) - 1.0
    psibar = 1.0 / (2.0 * math.pi)
    psi = psibar * (1.0 + amp * xi)
    vol = (1.0 / grid.nx) * (1.0 / grid.ny) * (2.0 * math.pi / grid.ntheta)
    psi = psi / (psi.sum() * vol)
    return psi.reshape(grid.ny, grid.nx, grid.ntheta)


def psi_uniform(grid: Grid) -> np.ndarray:
    return np.full((grid.ny, grid.nx, grid.ntheta), 1.0 / (2.0 * math.pi))


def cellular_flow(grid: Grid, amp: float = 0.1) -> np.ndarray:
    """u = amp (sin 2pi x cos 2pi y, -cos 2pi x sin 2pi y) at cell centres."""
    x = cell_centres(grid.nx)[None, :]
    y = cell_centres(grid.ny)[:, None]
    u = np.empty((2, grid.ny, grid.nx))
    u[0] = amp * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y)
    u[1] = -amp * np.cos(2 * math.pi * x) * np.sin(2 * math.pi * y)
    return u


def random_divfree_flow(grid: Grid, seed: int, n_modes: int, amp: float) -> np.ndarray:
    """Divergence-free field from a random stream function.

    phi_s = sum_m sin(2 pi k_m . x + phase_m), k_m integer in [-4,4]^2 \\ {0},
    phase_m ~ U[0, 2 pi); u = (d phi_s/dy, -d phi_s/dx) evaluated analytically
    at cell centres, scaled so that max over cells of |u| equals amp.
    """
    rng = SplitMix64(seed)
    modes = []
    while len(modes) < n_modes:
        kx = int(rng.uniform() * 9.0) - 4
        ky = int(rng.uniform() * 9.0) - 4
        ph = 2.0 * math.pi * rng.uniform()
        if kx == 0 and ky == 0:
            continue
        modes.append((kx, ky, ph))
    x = cell_centres(grid.nx)[None, :]
    y = cell_centres(grid.ny)[:, None]
    u = np.zeros((2, grid.ny, grid.nx))
    for kx, ky, ph in modes:
        c = np.cos(2 * math.pi * (kx * x + ky * y) + ph)
        u[0] += 2 * math.pi * ky * c
        u[1] -= 2 * math.pi * kx * c
    mag = np.sqrt(u[0] ** 2 + u[1] ** 2).max()
    if mag > 0:
        u *= amp / mag
    return u


def velocity_seed(seed: int, macro_step: int) -> int:
    """Seed of the velocity field drawn for a given macro step."""
    return (seed * 1_000_003 + 7919 * (macro_step + 1)) & _MASK


def uniform_mtot(grid: Grid, value: float = 1.0) -> np.ndarray:
    return np.full((grid.ny, grid.nx), value)


@dataclass(frozen=True)
class Member:
    grid: Grid
    rates: Rates
    seed: int


def ensemble_members(n: int = 64, base: int = 1000) -> list[Member]:
    """Detachment-rate sweep: per member m (seed 1..n), draw from
    splitmix64(base + m): N in {32,48,64,96,128}, Ntheta in {16,32},
    Ns in {16,32}, k_off log-uniform in [0.05, 5], v_walk uniform in [0.5, 2]."""
    out = []
    for m in range(1, n + 1):
        rng = SplitMix64(base + m)
        N = (32, 48, 64, 96, 128)[min(4, int(rng.uniform() * 5))]
        nth = (16, 32)[min(1, int(rng.uniform() * 2))]
        ns = (16, 32)[min(1, int(rng.uniform() * 2))]
        k_off = math.exp(math.log(0.05) + rng.uniform() * (math.log(5.0) - math.log(0.05)))
        v_w = 0.5 + 1.5 * rng.uniform()
        out.append(Member(Grid(N, N, nth, ns), Rates(v_walk=v_w, k_off=k_off), m))
    return out


# Workload shapes (sizes, substeps and flows) used by the tests and the bench.
WORKLOADS = {
    "cellular32": dict(grid=Grid(32, 32, 16, 16), substeps=200, macro=1, flow="cellular",
                       amp=0.1, seed=0),
    "precision128": dict(grid=Grid(128, 128, 32, 32), substeps=50, macro=10, flow="random",
                         modes=8, amp=0.1, seed=0),
    "adjoint64": dict(grid=Grid(64, 64, 32, 32), substeps=100, macro=1, flow="random",
                      modes=8, amp=0.1, seed=0),
    "large512": dict(grid=Grid(512, 512, 64, 64), substeps=100, macro=20, flow="random",
                     modes=16, amp=0.2, seed=0),
    # 64 members of ensemble_members(); each starts from its own perturbed
    # isotropic psi (seed = member seed) under its own 8-mode random flow
    "ensemble64": dict(members=64, substeps=500, macro=1, flow="random", modes=8, amp=0.1),
}


def member_inputs(m: Member, modes: int = 8, amp: float = 0.1) -> tuple[np.ndarray, np.ndarray]:
    """Initial psi and velocity of an ensemble member (from its seed)."""
    psi0 = psi_isotropic_perturbed(m.grid, m.seed)
    u = random_divfree_flow(m.grid, velocity_seed(m.seed, 0), modes, amp)
    return psi0, u


def workload_velocity(name: str, macro_step: int) -> np.ndarray:
    w = WORKLOADS[name]
    if w["flow"] == "cellular":
        return cellular_flow(w["grid"], w["amp"])
    return random_divfree_flow(w["grid"], velocity_seed(w["seed"], macro_step), w["modes"], w["amp"])
