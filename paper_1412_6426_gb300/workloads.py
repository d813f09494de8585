"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only unit conversions and initial conditions (particle
positions, momenta, weights, ids; field parameters; time steps).  It contains
none of the method's arithmetic and is the one module both the CUDA path and
the CPU oracle's tests draw their inputs from.

All quantities are in Compton units: length hbar/(m c), time hbar/(m c^2),
momentum m c, fields E_S = m^2 c^3/(e hbar).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# CODATA 2018
C_LIGHT = 299792458.0
HBAR = 1.054571817e-34
M_E = 9.1093837015e-31
Q_E = 1.602176634e-19
LAMBDA_C_BAR = HBAR / (M_E * C_LIGHT)          # m
TAU_C = HBAR / (M_E * C_LIGHT ** 2)            # s
E_S = M_E ** 2 * C_LIGHT ** 3 / (Q_E * HBAR)   # V/m
MC2_EV = M_E * C_LIGHT ** 2 / Q_E

FIELD_GRID, FIELD_UNIFORM, FIELD_GAUSSIAN_LP, FIELD_ROTATING_E = 0, 1, 2, 3
ELECTRON, POSITRON, PHOTON, ION = 0, 1, 2, 3


def length(meters: float) -> float:
    return meters / LAMBDA_C_BAR


def duration(seconds: float) -> float:
    return seconds / TAU_C


def laser_omega(wavelength_m: float) -> float:
    """Laser angular frequency in units of m c^2/hbar."""
    return 2 * math.pi * LAMBDA_C_BAR / wavelength_m


def a0_to_field(a0: float, wavelength_m: float) -> float:
    """Peak field of normalised amplitude a0 = eE/(m c omega), in units of E_S."""
    return a0 * laser_omega(wavelength_m)


def a0_from_intensity(intensity_w_cm2: float, wavelength_m: float, circular: bool) -> float:
    """I lambda^2 = 1.37e18 a0^2 W cm^-2 um^2 (linear) or 2.74e18 a0^2 (circular)."""
    k = 2.74e18 if circular else 1.37e18
    return math.sqrt(intensity_w_cm2 * (wavelength_m * 1e6) ** 2 / k)


@dataclass
class Workload:
    name: str
    n: tuple
    d: tuple
    x0: tuple
    periodic: tuple
    field_mode: int
    fp: tuple
    dt: float
    nsteps: int
    particles: dict = field(default_factory=dict)   # species -> (x, p, w, id)
    capacity: tuple = (0, 0, 0, 0)
    seed: int = 1
    kappa: float = 0.1
    meta: dict = field(default_factory=dict)

    def n_initial(self) -> int:
        return sum(len(v[3]) for v in self.particles.values())


def test_particles_static_b(n_particles: int = 10_000, gamma: float = 1000.0, chi: float = 1.0,
                            nsteps: int = 200, seed: int = 1) -> Workload:
    """Electrons with gamma along +x in a uniform static B along z set for the
    given chi; dt = 0.01 gyro-period of the initial gamma (the paper's
    distribution-function test, Sec. VII.B, has gamma0 = 1000, H0 = 1e-3 E_S)."""
    p0 = math.sqrt(gamma ** 2 - 1)
    B = chi / p0
    t_gyro = 2 * math.pi * gamma / B
    dt = 0.01 * t_gyro
    reach = 1.05 * nsteps * dt + 2 * p0 / B        # photons fly at c, electrons gyrate
    cells = 512
    d = 2 * reach / cells
    x = np.zeros((n_particles, 3))
    p = np.zeros((n_particles, 3))
    p[:, 0] = p0
    return Workload(
        name=f"static_B_{n_particles}e_chi{chi:g}_gamma{gamma:g}",
        n=(cells, cells, 1), d=(d, d, d), x0=(-reach, -reach, -0.5 * d), periodic=(1, 1, 1),
        field_mode=FIELD_UNIFORM, fp=(0, 0, 0, 0, 0, B), dt=dt, nsteps=nsteps,
        particles={ELECTRON: (x, p, np.ones(n_particles), np.arange(n_particles, dtype=np.uint64))},
        seed=seed, meta={"B": B, "t_gyro": t_gyro, "gamma0": gamma, "chi0": chi})


def beam_laser_collision(n_particles: int = 1_000_000, seed: int = 1, nsteps: int = 600,
                         energy_gev: float = 1.0, spread: float = 0.01, sigma_r_m: float = 1e-6,
                         sigma_x_m: float = 3e-6, wavelength_m: float = 0.8e-6, a0: float = 200.0,
                         fwhm_s: float = 30e-15, waist_m: float = 2e-6, meet_step: int | None = None
                         ) -> Workload:
    """Head-on collision of a Gaussian electron beam with a counter-propagating
    linearly polarised Gaussian laser pulse (test particles, analytic field).
    The beam and the pulse centres meet at the focus at step nsteps/2."""
    rng = np.random.default_rng(seed)
    gamma0 = energy_gev * 1e9 / MC2_EV
    omega = laser_omega(wavelength_m)
    t_laser = 2 * math.pi / omega
    dt = t_laser / 100.0
    meet = nsteps // 2 if meet_step is None else meet_step
    t_focus = meet * dt
    sx, sr = length(sigma_x_m), length(sigma_r_m)
    eps = gamma0 * (1 + spread * rng.standard_normal(n_particles))
    eps = np.maximum(eps, 2.0)
    x = np.empty((n_particles, 3))
    x[:, 0] = -t_focus + np.clip(rng.standard_normal(n_particles), -5, 5) * sx
    x[:, 1:] = np.clip(rng.standard_normal((n_particles, 2)), -5, 5) * sr
    p = np.zeros((n_particles, 3))
    p[:, 0] = np.sqrt(eps ** 2 - 1)
    half_x = 5.5 * sx + (nsteps - meet) * dt + t_focus
    half_r = 6.0 * sr
    cell = length(0.1e-6)
    nx = int(math.ceil(2 * half_x / cell))
    nr = int(math.ceil(2 * half_r / cell))
    E0 = a0_to_field(a0, wavelength_m)
    fp = (E0, omega, length(waist_m), duration(fwhm_s), 0.0, 0.0, 0.0, t_focus, 0.0)
    return Workload(
        name=f"beam_laser_{n_particles}e_a0{a0:g}_{energy_gev:g}GeV",
        n=(nx, nr, nr), d=(cell, cell, cell), x0=(-half_x, -half_r, -half_r), periodic=(0, 0, 0),
        field_mode=FIELD_GAUSSIAN_LP, fp=fp, dt=dt, nsteps=nsteps,
        particles={ELECTRON: (x, p, np.ones(n_particles), np.arange(n_particles, dtype=np.uint64))},
        seed=seed, meta={"gamma0": gamma0, "E0": E0, "omega": omega, "t_focus": t_focus,
                         "chi_headon": 2 * gamma0 * E0})


def subset(w: Workload, species: int, index: np.ndarray) -> Workload:
    """The same workload restricted to the listed particles of one species."""
    x, p, wt, ids = w.particles[species]
    out = Workload(**{k: getattr(w, k) for k in w.__dataclass_fields__})
    out.particles = {species: (x[index].copy(), p[index].copy(), wt[index].copy(), ids[index].copy())}
    return out
