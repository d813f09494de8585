"""The synthetic inputs (no GPU): unit conversions, the paper's benchmark
times, the slab target, and the initial fields of the mesh workloads checked
as vacuum plane waves by their Poynting flux (a pulse that should move along
+x carries its energy along +x at c: B = k x E)."""
import math

import numpy as np

from oracle import oracle as o
from paper_1412_6426_gb300 import workloads as wl


def test_units_and_field_scales():
    # 0.8 um laser: omega = 2 pi lambda_C / lambda in m c^2 / hbar
    w = wl.laser_omega(0.8e-6)
    assert abs(w - 2 * math.pi * 3.8615926796e-13 / 0.8e-6) < 1e-9 * w     # CODATA 2018 lambda_C / 2 pi
    # a0 = 200 -> E0 = a0 omega (E_S units), 6.07e-4
    assert abs(wl.a0_to_field(200.0, 0.8e-6) / 6.0658e-4 - 1) < 1e-3
    # I lambda^2 = 1.37e18 a0^2 (linear) / 2.74e18 (circular) W cm^-2 um^2
    assert abs(wl.a0_from_intensity(1.37e18, 1e-6, circular=False) - 1) < 1e-12
    assert abs(wl.a0_from_intensity(2.74e18, 1e-6, circular=True) - 1) < 1e-12


def test_benchmark_times():
    # Sec. VII.A: t_rad = 3.85 gamma0^(1/3) (E_S/H0)^(2/3) hbar^2/(m c e^2) = ... / alpha
    assert abs(wl.shower_t_rad(2e5, 0.2) / 90216.4 - 1) < 1e-5
    # Sec. VII.C: t_rad = 14 (E_S/H0)^(2/3) lambda_C/c; 173 t_rad is about an eighth of a 1 um cycle
    t = wl.avalanche_t_rad(1e-2)
    assert abs(t / (14 * 100 ** (2 / 3) * 2 * math.pi) - 1) < 1e-14
    a = wl.avalanche_cascade(n_seeds=4)
    assert 7.5 < a.meta["t_period"] / a.meta["dt_large"] < 8.5
    small = wl.avalanche_cascade(n_seeds=4, substeps=1018)
    assert abs(small.dt / t - 0.17) < 1e-3 and small.nsteps == 1018 * a.nsteps
    # the seed sits at lambda/8 with p_y = 1000, where E_y(t=0) = E0 sin(pi/4)
    x = a.particles[0][0][0]
    E, B = o.field(a.field_mode, a.fp, x, 0.0)
    assert abs(E[1] - 1e-2 * math.sqrt(0.5)) < 1e-15 and not np.any(B)
    assert np.all(a.particles[0][1][:, 1] == 1000.0)


def test_large_cascade_target():
    w, fx, fy = wl.large_cascade(n=64)
    xe, pe, we, ie = w.particles[wl.ELECTRON]
    xi, pi_, wi, ii = w.particles[wl.ION]
    # neutral: protons at the electrons' points with their weights; cold
    assert np.array_equal(xe, xi) and np.array_equal(we, wi) and not pe.any() and not pi_.any()
    assert len(np.intersect1d(ie, ii)) == 0
    # 20 cells thick at the centre, spanning the transverse box; 8 per cell
    i0, i1 = w.meta["target_cells"]
    assert i1 - i0 == 20 and len(ie) == 20 * 64 * 64 * 8
    assert xe[:, 0].min() >= i0 * w.d[0] and xe[:, 0].max() < i1 * w.d[0]
    # density: the weights add up to n_e x the slab volume (1e22 cm^-3 in Compton units)
    vol = (i1 - i0) * w.d[0] * (64 * w.d[1]) * (64 * w.d[2])
    ne = 1e22 * 1e6 * wl.LAMBDA_C_BAR ** 3
    assert abs(we.sum() / vol / ne - 1) < 1e-12


def _poynting_ratio(f, n, axis):
    """(integral of the Poynting flux along the axis) / (integral of the
    energy density) over each half of the box along that axis: +1 for a
    vacuum plane wave moving up the axis, -1 moving down (c = 1)."""
    Ex, Ey, Ez, Bx, By, Bz = (np.asarray(a, dtype=np.float64).reshape(n, n, n) for a in f)
    S = Ey * Bz - Ez * By if axis == 0 else Ez * Bx - Ex * Bz
    u = 0.5 * (Ex ** 2 + Ey ** 2 + Ez ** 2 + Bx ** 2 + By ** 2 + Bz ** 2)
    red = (0, 1) if axis == 0 else (0, 2)
    S, u = S.sum(axis=red), u.sum(axis=red)
    return [float(S[h].sum() / u[h].sum()) for h in (slice(0, n // 2), slice(n // 2, n))]


def test_large_cascade_pulses_are_vacuum_plane_waves():
    # the pulse below the centre moves up the axis (B = k x E), the other
    # down, along x and along y; both fill their half of the box
    n = 64
    w, fx, fy = wl.large_cascade(n=n)
    zero = [np.zeros(n) for _ in range(6)]
    for axis, prof in ((0, (fx, zero)), (1, (zero, fy))):
        f = wl.expand_profiles(prof[0], prof[1], n)
        lo, hi = _poynting_ratio(f, n, axis)
        assert abs(lo - 1) < 0.02 and abs(hi + 1) < 0.02, (axis, lo, hi)
    # the peak field of each pulse is E0
    assert abs(max(np.abs(a).max() for a in fx[1:3]) / w.meta["E0"] - 1) < 0.01


def test_self_consistent_cascade_pulses_are_vacuum_plane_waves():
    # the same recipe on a 128^3 mesh of the same 8 lambda box
    n = 128
    w, f = wl.self_consistent_cascade(n=n, n_seed=10, precision=64, cells_per_lambda=16, steps_per_period=32)
    lo, hi = _poynting_ratio(f, n, 0)
    assert abs(lo - 1) < 0.03 and abs(hi + 1) < 0.03, (lo, hi)


def test_profile_expansion_same_with_torch_and_numpy():
    # the bench and the full-size tests expand the mesh profiles with torch on
    # the device; the layout (x fastest) must be numpy's
    import torch
    n = 16
    w, fx, fy = wl.large_cascade(n=n)
    a = wl.expand_profiles(fx, fy, n)
    b = wl.expand_profiles(fx, fy, n, xp=torch, dtype=torch.float64)
    for u, v in zip(a, b):
        assert np.array_equal(np.asarray(u), v.numpy())
    # F[k, j, i] = fx[i] + fy[j]
    f = np.asarray(a[2]).reshape(n, n, n)
    assert f[3, 5, 7] == fx[2][7] + fy[2][5]
