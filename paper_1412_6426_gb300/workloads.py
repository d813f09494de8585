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
ALPHA = 7.2973525693e-3                        # fine-structure constant

FIELD_GRID, FIELD_UNIFORM, FIELD_GAUSSIAN_LP, FIELD_ROTATING_E, FIELD_ENSEMBLE, FIELD_STANDING_WAVE = 0, 1, 2, 3, 4, 5
ENS_STRIDE = 10   # ensemble table row: E0, omega, phase, Eu[3], Bu[3], thin_scale
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
    ens: np.ndarray | None = None      # (n_ens, ENS_STRIDE) table for FIELD_ENSEMBLE
    ens_bits: int = 0                  # top id bits naming the ensemble

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
        seed=seed, meta={"gamma0": gamma0, "E0": E0, "omega": omega, "t_focus": t_focus, "a0": a0,
                         "chi_headon": 2 * gamma0 * E0})


def rotating_field_for_chi(chi: float, omega: float) -> float:
    """E0 (units of E_S) of a rotating E field in which an electron on the
    drift-free circular orbit, p = a0 = E0/omega perpendicular to E, has the
    given chi = gamma E0 with gamma = sqrt(1 + a0^2):
    E0^2 = (omega^2/2) (sqrt(1 + 4 chi^2/omega^2) - 1)."""
    r = 2.0 * chi / omega
    # sqrt(1 + r^2) - 1 written without cancellation
    u = 0.5 * omega * omega * (r * r / (math.sqrt(1.0 + r * r) + 1.0))
    return math.sqrt(u)


def batched_ensembles(n_ens: int = 512, count_range=(1e3, 1e6), chi_range=(0.1, 100.0), nsteps: int = 500,
                      seed: int = 1, wavelength_m: float = 0.8e-6, steps_per_period: int = 100,
                      thin_interval: int = 4, thin_limit=(1, 1, 2, 0)) -> Workload:
    """Independent test-particle instances in uniform rotating electric fields
    (the field at the antinode of a circularly polarised standing wave).

    Ensemble e has chi_e log-uniform in chi_range and N_e electrons with N_e
    log-uniform in count_range (seeded).  Its field rotates at the laser
    frequency with amplitude E0_e such that an electron on the drift-free
    circular orbit, p = a0 (-sin phi_e, cos phi_e, 0) with a0 = E0_e/omega,
    has chi = chi_e; the phase phi_e is random.  Positions are uniform in a
    periodic box (the field is uniform, so they only label cells).  Every
    ensemble keeps its own particle budget through thinning (Sec. VI): every
    thin_interval steps a species group above thin_limit[sp] x N_e particles
    is thinned with global even redistribution.  dt = T_laser /
    steps_per_period.  Ids carry the ensemble in their top ens_bits bits."""
    rng = np.random.default_rng(seed)
    omega = laser_omega(wavelength_m)
    t_laser = 2 * math.pi / omega
    bits = max(1, int(math.ceil(math.log2(n_ens))))
    lo, hi = (math.log10(v) for v in chi_range)
    chi = 10.0 ** rng.uniform(lo, hi, n_ens)
    clo, chi_ = (math.log10(v) for v in count_range)
    counts = np.maximum(1, np.rint(10.0 ** rng.uniform(clo, chi_, n_ens))).astype(np.int64)
    phase = rng.uniform(0.0, 2 * math.pi, n_ens)
    E0 = np.array([rotating_field_for_chi(c, omega) for c in chi])
    a0 = E0 / omega
    table = np.zeros((n_ens, ENS_STRIDE))
    table[:, 0] = E0
    table[:, 1] = omega
    table[:, 2] = phase
    table[:, 9] = counts
    cells = 16
    d = length(wavelength_m) / cells
    total = int(counts.sum())
    x = rng.uniform(0.0, cells * d, (total, 3))
    p = np.zeros((total, 3))
    ids = np.empty(total, dtype=np.uint64)
    o = 0
    for e in range(n_ens):
        n = int(counts[e])
        p[o:o + n, 0] = -a0[e] * math.sin(phase[e])
        p[o:o + n, 1] = a0[e] * math.cos(phase[e])
        ids[o:o + n] = (np.uint64(e) << np.uint64(64 - bits)) | np.arange(n, dtype=np.uint64)
        o += n
    cap_e = int(2.5 * total) + 4096
    cap_g = int(thin_limit[2] * total * 4) + 4096
    return Workload(
        name=f"batched_{n_ens}ens_{total}e_chi{chi_range[0]:g}-{chi_range[1]:g}",
        n=(cells, cells, cells), d=(d, d, d), x0=(0.0, 0.0, 0.0), periodic=(1, 1, 1),
        field_mode=FIELD_ENSEMBLE, fp=(), dt=t_laser / steps_per_period, nsteps=nsteps,
        particles={ELECTRON: (x, p, np.ones(total), ids)},
        capacity=(cap_e, cap_e, cap_g, 0), seed=seed, ens=table, ens_bits=bits,
        meta={"chi": chi, "counts": counts, "E0": E0, "a0": a0, "phase": phase, "omega": omega,
              "thin_interval": thin_interval, "thin_limit": tuple(thin_limit)})


def self_consistent_cascade(n: int = 256, seed: int = 1, nsteps: int = 2000, wavelength_m: float = 0.8e-6,
                            cells_per_lambda: int = 32, steps_per_period: int = 64,
                            intensity_w_cm2: float = 1e24, n_seed: int = 100_000, seed_cube_m: float = 1e-6,
                            precision: int = 32):
    """A self-consistent QED cascade on a periodic Yee mesh: two counter-
    propagating circularly polarised plane-wave pulses along +-x with a sin^2
    envelope of 2 lambda intensity FWHM (4 lambda full width), each at the
    given intensity, meeting at the box centre after 2 lambda of travel; a
    cold seed of n_seed electrons and n_seed positrons uniform in a cube at the
    centre.  Returns (workload, fields) with fields = [Ex, Ey, Ez, Bx, By, Bz]
    on the Yee staggering at t = 0 (numpy arrays, x fastest)."""
    rng = np.random.default_rng(seed)
    lam = length(wavelength_m)
    d = lam / cells_per_lambda
    omega = laser_omega(wavelength_m)
    t_laser = 2 * math.pi / omega
    dt = t_laser / steps_per_period
    a0 = a0_from_intensity(intensity_w_cm2, wavelength_m, circular=True)
    E0 = a0_to_field(a0, wavelength_m)
    L = n * d
    xc = 0.5 * L
    W = 4.0 * lam                              # full width of the sin^2 envelope (FWHM 2 lambda)
    ftype = np.float32 if precision == 32 else np.float64

    def envelope(u):
        # sin^2 envelope centred at u = 0, zero outside |u| < W/2
        e = np.sin(math.pi * (u / W + 0.5)) ** 2
        return np.where(np.abs(u) < 0.5 * W, e, 0.0)

    def wrap(u):
        return (u + 0.5 * L) % L - 0.5 * L

    def pulses(x, comp):
        # pulse A moves +x from xc - 2 lam, pulse B moves -x from xc + 2 lam (t = 0)
        ua = wrap(x - (xc - 2 * lam))
        ub = wrap(x - (xc + 2 * lam))
        pa = omega * ua
        pb = omega * ub
        fa, fb = E0 * envelope(ua), E0 * envelope(ub)
        if comp == "Ey":
            return fa * np.cos(pa) + fb * np.cos(pb)
        if comp == "Ez":
            return fa * np.sin(pa) + fb * np.sin(pb)
        if comp == "By":      # B = +x x E for A, -x x E for B
            return -fa * np.sin(pa) + fb * np.sin(pb)
        if comp == "Bz":
            return fa * np.cos(pa) - fb * np.cos(pb)
        raise ValueError(comp)

    xi = np.arange(n) * d                      # Ey, Ez at x = i d
    xh = (np.arange(n) + 0.5) * d              # By, Bz at x = (i + 1/2) d
    nc = n ** 3
    f = [np.zeros(nc, dtype=ftype) for _ in range(6)]
    for k, (comp, xs) in enumerate((("Ey", xi), ("Ez", xi))):
        f[1 + k][:] = np.broadcast_to(pulses(xs, comp)[None, None, :], (n, n, n)).ravel()
    for k, (comp, xs) in enumerate((("By", xh), ("Bz", xh))):
        f[4 + k][:] = np.broadcast_to(pulses(xs, comp)[None, None, :], (n, n, n)).ravel()
    side = length(seed_cube_m)
    parts = {}
    for sp in (ELECTRON, POSITRON):
        x = xc + (rng.uniform(-0.5, 0.5, (n_seed, 3)) * side)
        parts[sp] = (x, np.zeros((n_seed, 3)), np.ones(n_seed),
                     np.arange(n_seed, dtype=np.uint64) + np.uint64(sp * n_seed))
    w = Workload(name=f"cascade_{n}cubed_{intensity_w_cm2:g}Wcm2", n=(n, n, n), d=(d, d, d), x0=(0.0, 0.0, 0.0),
                 periodic=(1, 1, 1), field_mode=FIELD_GRID, fp=(), dt=dt, nsteps=nsteps, particles=parts, seed=seed,
                 meta={"a0": a0, "E0": E0, "omega": omega, "lambda": lam, "meet_step": 2 * steps_per_period})
    return w, f


def large_cascade(n: int = 512, seed: int = 1, nsteps: int = 3000, wavelength_m: float = 0.8e-6,
                  cells_per_lambda: int = 32, steps_per_period: int = 64, intensity_w_cm2: float = 2e24,
                  density_cm3: float = 1e22, thickness_m: float = 0.5e-6, ppc: int = 8):
    """The large self-consistent cascade: an n^3 periodic Yee mesh (dx =
    lambda/32, box 16 lambda at n = 512) with four circularly polarised
    plane-wave pulses at the given intensity each, two along +-x and two
    along +-y, meeting at the box centre, and a cold hydrogen slab target
    (electrons and protons at the same points, so rho = 0 at t = 0) of
    density n_e and the given thickness along x at the centre, spanning the
    transverse box, with ppc macro-particles per cell and species.

    Each pulse has a sin^2 envelope of full width half the box (8 lambda at
    n = 512; intensity FWHM 4 lambda), the longest that lets two
    counter-propagating pulses start side by side in the periodic box; at
    t = 0 their centres are a quarter box from the centre, so they meet there
    at step 4 steps_per_period (n = 512).  Every field component is the sum
    of an x-profile and a y-profile:
        F_c[k, j, i] = fx[c][i] + fy[c][j]
    on the Yee staggering.  Returns (workload, fx, fy) with fx, fy lists of
    six 1-D numpy arrays (Ex, Ey, Ez, Bx, By, Bz); expand with
    expand_profiles."""
    rng = np.random.default_rng(seed)
    lam = length(wavelength_m)
    d = lam / cells_per_lambda
    omega = laser_omega(wavelength_m)
    t_laser = 2 * math.pi / omega
    dt = t_laser / steps_per_period
    a0 = a0_from_intensity(intensity_w_cm2, wavelength_m, circular=True)
    E0 = a0_to_field(a0, wavelength_m)
    L = n * d
    c0 = 0.5 * L
    W = 0.5 * L                                 # full width of the sin^2 envelope
    off = 0.25 * L                              # pulse centres at c0 -+ off

    def envelope(u):
        e = np.sin(math.pi * (u / W + 0.5)) ** 2
        return np.where(np.abs(u) < 0.5 * W, e, 0.0)

    def wrap(u):
        return (u + 0.5 * L) % L - 0.5 * L

    def pair(s):
        # the +s pulse starts at c0 - off and the -s pulse at c0 + off:
        # (amplitude, phase) of each at coordinate s
        ua, ub = wrap(s - (c0 - off)), wrap(s - (c0 + off))
        return E0 * envelope(ua), omega * ua, E0 * envelope(ub), omega * ub

    node = np.arange(n) * d
    half = (np.arange(n) + 0.5) * d
    fx = [np.zeros(n) for _ in range(6)]
    fy = [np.zeros(n) for _ in range(6)]
    # along x: E in the y-z plane; B = +x x E for the +x pulse, -x x E for the other
    fa, pa, fb, pb = pair(node)                 # Ey, Ez sit at x = i d
    fx[1] = fa * np.cos(pa) + fb * np.cos(pb)
    fx[2] = fa * np.sin(pa) + fb * np.sin(pb)
    fa, pa, fb, pb = pair(half)                 # By, Bz sit at x = (i + 1/2) d
    fx[4] = -fa * np.sin(pa) + fb * np.sin(pb)
    fx[5] = fa * np.cos(pa) - fb * np.cos(pb)
    # along y: E in the z-x plane (E = f (cos p z + sin p x)); B = +y x E, -y x E
    fa, pa, fb, pb = pair(node)                 # Ex, Ez sit at y = j d
    fy[0] = fa * np.sin(pa) + fb * np.sin(pb)
    fy[2] = fa * np.cos(pa) + fb * np.cos(pb)
    fa, pa, fb, pb = pair(half)                 # Bx, Bz sit at y = (j + 1/2) d
    fy[3] = fa * np.cos(pa) - fb * np.cos(pb)
    fy[5] = -fa * np.sin(pa) + fb * np.sin(pb)
    # target: n_e per Compton volume, weight = real particles per macro-particle
    ne = density_cm3 * 1e6 * LAMBDA_C_BAR ** 3
    cells_x = int(round(length(thickness_m) / d))
    i0 = n // 2 - cells_x // 2
    count = cells_x * n * n * ppc
    x = np.empty((count, 3))
    x[:, 0] = (i0 + rng.uniform(0.0, cells_x, count)) * d
    x[:, 1] = rng.uniform(0.0, n, count) * d
    x[:, 2] = rng.uniform(0.0, n, count) * d
    wt = np.full(count, ne * d ** 3 / ppc)
    p = np.zeros((count, 3))
    ids = np.arange(count, dtype=np.uint64)
    parts = {ELECTRON: (x, p, wt, ids), ION: (x, p, wt, ids + np.uint64(count))}
    scale = count / (20 * 512 * 512 * 8)
    w = Workload(name=f"large_cascade_{n}cubed_{intensity_w_cm2:g}Wcm2_x4", n=(n, n, n), d=(d, d, d),
                 x0=(0.0, 0.0, 0.0), periodic=(1, 1, 1), field_mode=FIELD_GRID, fp=(), dt=dt, nsteps=nsteps,
                 particles=parts, seed=seed,
                 meta={"a0": a0, "E0": E0, "omega": omega, "lambda": lam, "n_e": ne, "weight": wt[0],
                       "target_cells": (i0, i0 + cells_x), "meet_step": int(round(off / dt)),
                       # the cascade would pass 1e9 particles within ~200 steps: thinning (Sec. VI)
                       # every 8 steps holds e-, e+ and photons to these counts (at n = 512;
                       # smaller boxes scale them with the target)
                       "thin_interval": 8,
                       "thin_limit": tuple(int(v * scale) for v in (2.0e8, 1.6e8, 6.0e8)) + (0,),
                       # FP32 stores: 80 B a slot (two buffers); FP64: 144 B, 1.05e9 slots in 164 GB
                       # plus 9.7 GB of FP64 mesh, within 180 GB
                       "capacity32": tuple(int(v * scale) for v in (2.5e8, 2.0e8, 7.5e8)) + (count,),
                       "capacity64": tuple(int(v * scale) for v in (2.0e8, 2.0e8, 6.0e8)) + (count,)})
    return w, fx, fy


def expand_profiles(fx, fy, n, xp=np, **kw):
    """F_c[k, j, i] = fx[c][i] + fy[c][j] as flat arrays (x fastest), with
    numpy or any array module of the same broadcasting rules (xp.asarray
    takes the keyword arguments, e.g. dtype and device)."""
    out = []
    for a, b in zip(fx, fy):
        ax = xp.asarray(a, **kw).reshape(1, 1, n)
        by = xp.asarray(b, **kw).reshape(1, n, 1)
        out.append((ax + by).expand(n, n, n).reshape(-1) if hasattr(ax, "expand")
                   else np.broadcast_to(ax + by, (n, n, n)).reshape(-1))
    return out


def shower_t_rad(gamma0: float, H0: float) -> float:
    """Radiation time of the shower benchmark (Sec. VII.A):
    t_rad = 3.85 gamma0^(1/3) (E_S/H0)^(2/3) hbar^2/(m c e^2), and
    hbar^2/(m c e^2) = (hbar/(m c^2)) / alpha in Compton units."""
    return 3.85 * gamma0 ** (1.0 / 3.0) * (1.0 / H0) ** (2.0 / 3.0) / ALPHA


def shower_cascade(n_seeds: int = 1000, gamma0: float = 2e5, H0: float = 0.2, dt_per_trad: float = 1e-3,
                   t_end_trad: float = 2.0, seed: int = 1) -> Workload:
    """Shower-type cascade of Sec. VII.A: n_seeds independent electrons with
    gamma0 along +x in a constant magnetic field H0 (units of E_S) along z,
    perpendicular to the motion.  The field is uniform and the particles are
    test particles, so one run of n_seeds electrons is n_seeds independent
    cascades (the benchmark averages 10^3 runs).  dt = dt_per_trad t_rad;
    nsteps reaches t_end_trad t_rad.  The periodic box is larger than the
    gyro-radius (uniform field: the wrap changes nothing)."""
    t_rad = shower_t_rad(gamma0, H0)
    dt = dt_per_trad * t_rad
    nsteps = int(round(t_end_trad / dt_per_trad))
    p0 = math.sqrt(gamma0 ** 2 - 1.0)
    cells = 16
    d = 4.0 * p0 / H0 / cells
    x = np.zeros((n_seeds, 3))
    x[:, 0] = 0.5 * cells * d
    x[:, 1] = 0.5 * cells * d - p0 / H0          # orbit centred in the box
    x[:, 2] = 0.5 * d
    p = np.zeros((n_seeds, 3))
    p[:, 0] = p0
    return Workload(
        name=f"shower_{n_seeds}e_gamma{gamma0:g}_H{H0:g}_dt{dt_per_trad:g}trad",
        n=(cells, cells, 1), d=(d, d, d), x0=(0.0, 0.0, 0.0), periodic=(1, 1, 1),
        field_mode=FIELD_UNIFORM, fp=(0.0, 0.0, 0.0, 0.0, 0.0, H0), dt=dt, nsteps=nsteps,
        particles={ELECTRON: (x, p, np.ones(n_seeds), np.arange(n_seeds, dtype=np.uint64))},
        seed=seed, meta={"t_rad": t_rad, "gamma0": gamma0, "H0": H0, "eps_cut": 1e-3 * gamma0})


def avalanche_t_rad(E0: float) -> float:
    """t_rad of the avalanche benchmark (Sec. VII.C): 14 (E_S/H0)^(2/3)
    lambda_C/c, lambda_C = 2 pi hbar/(m c) the Compton wavelength, so
    lambda_C/c is 2 pi Compton time units."""
    return 14.0 * (1.0 / E0) ** (2.0 / 3.0) * 2.0 * math.pi


def avalanche_cascade(n_seeds: int = 256, E0: float = 1e-2, wavelength_m: float = 1e-6,
                      dt_large_trad: float = 173.0, substeps: int = 1, periods: float = 1.0,
                      cells: int = 64, seed: int = 1) -> Workload:
    """Avalanche-type cascade of Sec. VII.C: seed electrons at x = lambda/8
    with p_y = 1000 (gamma0 ~ 1000) in the plane standing wave whose only
    field at t = 0 is E_y = E0 sin(2 pi x/lambda) (FIELD_STANDING_WAVE).
    The large step is dt_large_trad t_rad (173 t_rad: about 8 steps per
    cycle); substeps > 1 divides it (substeps = 1018 gives 0.17 t_rad), so
    both runs reach the same times.  The box is one wavelength, periodic (the
    wave's period); y and z are one periodic cell.  Test particles: one run
    holds n_seeds independent avalanches."""
    lam = length(wavelength_m)
    omega = laser_omega(wavelength_m)
    t_rad = avalanche_t_rad(E0)
    dt_large = dt_large_trad * t_rad
    dt = dt_large / substeps
    t_period = 2.0 * math.pi / omega
    n_large = int(math.ceil(periods * t_period / dt_large))
    d = lam / cells
    x = np.empty((n_seeds, 3))
    x[:, 0] = lam / 8.0
    x[:, 1] = 0.5 * lam
    x[:, 2] = 0.5 * lam
    p = np.zeros((n_seeds, 3))
    p[:, 1] = 1000.0
    return Workload(
        name=f"avalanche_{n_seeds}e_E{E0:g}_dt{dt / t_rad:.4g}trad",
        n=(cells, 1, 1), d=(d, lam, lam), x0=(0.0, 0.0, 0.0), periodic=(1, 1, 1),
        field_mode=FIELD_STANDING_WAVE, fp=(E0, omega), dt=dt, nsteps=n_large * substeps,
        particles={ELECTRON: (x, p, np.ones(n_seeds), np.arange(n_seeds, dtype=np.uint64))},
        seed=seed, meta={"t_rad": t_rad, "dt_large": dt_large, "substeps": substeps, "n_large": n_large,
                         "omega": omega, "lambda": lam, "t_period": t_period})


def subset(w: Workload, species: int, index: np.ndarray) -> Workload:
    """The same workload restricted to the listed particles of one species."""
    x, p, wt, ids = w.particles[species]
    out = Workload(**{k: getattr(w, k) for k in w.__dataclass_fields__})
    out.particles = {species: (x[index].copy(), p[index].copy(), wt[index].copy(), ids[index].copy())}
    return out
