"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module only builds inputs: frequency grids, direction grids and analytic
particle trajectories (position r, normalised velocity beta, its time
derivative beta_dot, weighting w) in SI units, float64, SoA [3][N].  It holds
none of the radiation arithmetic.  The paper's LWFA run (PIConGPU, Sec. 4) is
not available, so LWFA-shaped bunches with analytic betatron motion stand in
for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

C = 299792458.0
Q_E = 1.602176634e-19
M_E = 9.1093837015e-31
EPS0 = 8.8541878128e-12


# ----------------------------------------------------------------- grids
def omega_linear(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n, dtype=np.float64)


def omega_log(lo: float, hi: float, n: int) -> np.ndarray:
    if n == 1:
        return np.array([lo], dtype=np.float64)
    j = np.arange(n, dtype=np.float64)
    return lo * (hi / lo) ** (j / (n - 1))


def dirs_theta_line(theta_max: float, n: int) -> np.ndarray:
    """n directions (sin th, 0, cos th), th = linspace(0, theta_max): [n][3]."""
    th = np.linspace(0.0, theta_max, n)
    return np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], axis=1)


def dirs_grid(half_angle: float, nx: int, ny: int) -> np.ndarray:
    """Cartesian angle grid, n = (sin tx cos ty, sin ty, cos tx cos ty): [ny*nx][3]."""
    tx = np.linspace(-half_angle, half_angle, nx)
    ty = np.linspace(-half_angle, half_angle, ny)
    TY, TX = np.meshgrid(ty, tx, indexing="ij")
    d = np.stack([np.sin(TX) * np.cos(TY), np.sin(TY), np.cos(TX) * np.cos(TY)], axis=-1)
    return d.reshape(-1, 3)


# ----------------------------------------------------------- trajectories
@dataclass
class Step:
    """One time step's particle arrays (float64): r, beta, beta_dot SoA [3][N], w [N]."""

    r: np.ndarray
    beta: np.ndarray
    beta_dot: np.ndarray
    w: np.ndarray
    t: float
    dt: float

    @property
    def n(self) -> int:
        return self.w.shape[0]


class HelixBunch:
    """Macro-particles on identical helices about z with seeded phases.

    Undulator-like strength K = gamma beta_perp = 1, radius rho, helix angular
    frequency w_h = beta_perp c / rho, beta_z from |beta| = sqrt(1 - 1/gamma^2).
    """

    def __init__(self, n: int, gamma: float = 50.0, radius: float = 1e-6, seed: int = 1,
                 weight: float = 1.0, k_strength: float = 1.0):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.n = n
        self.phase = rng.uniform(0.0, 2.0 * math.pi, n)
        self.rho = radius
        self.bperp = k_strength / gamma
        self.wh = self.bperp * C / radius
        self.bz = math.sqrt(1.0 - 1.0 / gamma**2 - self.bperp**2)
        self.w = np.full(n, float(weight))

    def step(self, t: float, dt: float) -> Step:
        ph = self.wh * t + self.phase
        cp, sp = np.cos(ph), np.sin(ph)
        z = np.full(self.n, self.bz * C * t)
        r = np.concatenate([self.rho * cp, self.rho * sp, z])
        beta = np.concatenate([-self.bperp * sp, self.bperp * cp, np.full(self.n, self.bz)])
        bdot = np.concatenate([-self.bperp * self.wh * cp, -self.bperp * self.wh * sp,
                               np.zeros(self.n)])
        return Step(r, beta, bdot, self.w.copy(), float(t), float(dt))


def plasma_omega(n_e_cm3: float) -> float:
    n_e = n_e_cm3 * 1e6
    return math.sqrt(n_e * Q_E**2 / (EPS0 * M_E))


class BetatronBunch:
    """LWFA-shaped bunch: Gaussian in space, log-normal gamma, betatron motion.

    x(t) = x0 cos(k_b c t + phi_x), y likewise, with k_b = (w_p / c) / sqrt(2 gamma)
    (w_p from the plasma density n_e); beta_z follows from |beta| = const, and z
    carries the matching second-order longitudinal oscillation.  Weightings are
    uniform in [w_lo, w_hi] electrons.
    """

    def __init__(self, n: int, seed: int = 2, sigma_z: float = 1e-6, sigma_r: float = 2e-6,
                 gamma0: float = 300.0, sigma_ln_gamma: float = 0.1, n_e_cm3: float = 1e18,
                 w_lo: float = 1e3, w_hi: float = 1e5, gamma_range: tuple | None = None):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.n = n
        self.z0 = rng.normal(0.0, sigma_z, n)
        self.x0 = rng.normal(0.0, sigma_r, n)
        self.y0 = rng.normal(0.0, sigma_r, n)
        if gamma_range is None:
            self.gamma = gamma0 * np.exp(sigma_ln_gamma * rng.normal(0.0, 1.0, n))
        else:
            lo, hi = gamma_range
            self.gamma = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
        self.phx = rng.uniform(0.0, 2.0 * math.pi, n)
        self.phy = rng.uniform(0.0, 2.0 * math.pi, n)
        self.w = rng.uniform(w_lo, w_hi, n)
        self.kb = plasma_omega(n_e_cm3) / C / np.sqrt(2.0 * self.gamma)
        self.inv_g2 = 1.0 / self.gamma**2

    def step(self, t: float, dt: float) -> Step:
        kb, x0, y0 = self.kb, self.x0, self.y0
        px = kb * C * t + self.phx
        py = kb * C * t + self.phy
        cx, sx, cy, sy = np.cos(px), np.sin(px), np.cos(py), np.sin(py)
        x, y = x0 * cx, y0 * cy
        bx, by = -x0 * kb * sx, -y0 * kb * sy
        bz = np.sqrt(1.0 - self.inv_g2 - bx * bx - by * by)
        # z = z0 + c * integral of beta_z, beta_z to second order in the transverse motion
        ax2, ay2 = (x0 * kb) ** 2, (y0 * kb) ** 2
        osc = (ax2 * (t / 2 - (np.sin(2 * px) - np.sin(2 * self.phx)) / (4 * kb * C))
               + ay2 * (t / 2 - (np.sin(2 * py) - np.sin(2 * self.phy)) / (4 * kb * C)))
        z = self.z0 + C * t * (1.0 - 0.5 * self.inv_g2) - 0.5 * C * osc
        bdx, bdy = -x0 * kb * kb * C * cx, -y0 * kb * kb * C * cy
        bdz = -(bx * bdx + by * bdy) / bz
        r = np.concatenate([x, y, z])
        beta = np.concatenate([bx, by, bz])
        bdot = np.concatenate([bdx, bdy, bdz])
        return Step(r, beta, bdot, self.w.copy(), float(t), float(dt))


# ----------------------------------------------------------- workloads
@dataclass
class Workload:
    name: str
    omega: np.ndarray
    dirs: np.ndarray
    bunch: object
    n_steps: int
    dt: float
    ff_kind: int
    ff_width: float

    def step(self, s: int) -> Step:
        return self.bunch.step(s * self.dt, self.dt)

    @property
    def n_particles(self) -> int:
        return self.bunch.n

    def updates_per_step(self) -> int:
        return self.bunch.n * self.omega.shape[0] * self.dirs.shape[0]


FF_POINT, FF_CIC, FF_TSC, FF_QSC, FF_GAUSS = 0, 1, 2, 3, 4


def tiny_helix(n_particles: int = 64, n_steps: int = 1000, n_omega: int = 128,
               n_dir: int = 16, seed: int = 1) -> Workload:
    """Plain method, tiny: 64 point macro-particles (w = 1) on gamma = 50 helices of
    radius 1 um, 1000 steps of 1e-17 s, 128 linear omega in [1e15, 1e18] rad/s,
    16 directions on a theta line 0..20 mrad."""
    return Workload("helix_tiny", omega_linear(1e15, 1e18, n_omega), dirs_theta_line(0.02, n_dir),
                    HelixBunch(n_particles, gamma=50.0, radius=1e-6, seed=seed), n_steps, 1e-17,
                    FF_POINT, 0.0)


def lwfa_bunch(n_particles: int = 100_000, n_steps: int = 2048, n_omega: int = 512,
               n_side: int = 16, seed: int = 2) -> Workload:
    """LWFA-shaped bunch: 1e5 macro-particles, Gaussian sigma_z = 1 um,
    sigma_r = 2 um, gamma log-normal about 300, betatron motion at n_e = 1e18 cm^-3,
    w uniform in [1e3, 1e5], Gaussian form factor with sigma = 0.1 um, 2048 steps
    of 1e-16 s, 512 log omega in [1e14, 1e20] rad/s, 16 x 16 directions +-10 mrad."""
    return Workload("lwfa_bunch", omega_log(1e14, 1e20, n_omega), dirs_grid(0.01, n_side, n_side),
                    BetatronBunch(n_particles, seed=seed), n_steps, 1e-16, FF_GAUSS, 0.1e-6)


@dataclass
class JobSpec:
    seed: int
    n_particles: int
    n_omega: int
    n_side: int
    n_steps: int
    gamma_lo: float
    gamma_hi: float
    sigma: float

    def workload(self) -> Workload:
        bunch = BetatronBunch(self.n_particles, seed=self.seed, sigma_z=self.sigma,
                              sigma_r=self.sigma, gamma_range=(self.gamma_lo, self.gamma_hi))
        return Workload(f"job{self.seed}", omega_log(1e14, 1e20, self.n_omega),
                        dirs_grid(0.01, self.n_side, self.n_side), bunch, self.n_steps, 1e-16,
                        FF_GAUSS, 0.1e-6)

    def updates_per_step(self) -> int:
        return self.n_particles * self.n_omega * self.n_side * self.n_side


def job_mix(n_jobs: int = 64, base_seed: int = 4000, n_lo: float = 1e3, n_hi: float = 1e6,
            steps: tuple = (200, 200), log2_omega: tuple = (6, 10),
            log2_side: tuple = (2, 5)) -> list[JobSpec]:
    """Batched-jobs mix: N log-uniform in [n_lo, n_hi] (default 1e3..1e6), omega
    grids 2^6..2^10 = 64..1024 and square direction grids (2^2)^2..(2^5)^2 =
    4^2..32^2 by default (powers of two, inclusive ranges of exponents), gamma
    log-uniform in [50, 1000] (each job's bunch), sigma uniform in [0.5, 5] um."""
    out = []
    for j in range(n_jobs):
        rng = np.random.Generator(np.random.PCG64(base_seed + j))
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        n_omega = int(2 ** rng.integers(log2_omega[0], log2_omega[1] + 1))
        n_side = int(2 ** rng.integers(log2_side[0], log2_side[1] + 1))
        g = math.exp(rng.uniform(math.log(50.0), math.log(1000.0)))
        sigma = rng.uniform(0.5e-6, 5e-6)
        n_steps = int(rng.integers(steps[0], steps[1] + 1))
        out.append(JobSpec(base_seed + j, n, n_omega, n_side, n_steps, 0.9 * g, 1.1 * g, sigma))
    return out
