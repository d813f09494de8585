"""Pins of the oracle's grid kernels (Appendix C: FDTD, CIC, Esirkepov).

Yee: a vacuum plane wave obeys the discrete dispersion relation
(sin(w dt/2)/dt)^2 = sum_i (sin(k_i d_i/2)/d_i)^2; the FDTD keeps div B at
rounding level.  CIC reproduces linear fields exactly.  Esirkepov: the
deposited current satisfies the discrete continuity equation
(rho^{n+1} - rho^n)/dt + div J = 0 cell by cell, and sum J dV = q w dx/dt.
Together (Gauss's law in Compton units, div E = 4 pi alpha rho): one FDTD step
with that current changes the discrete div E by exactly 4 pi alpha times the
change of the charge density at every node, whatever the fields.
"""
import math

import numpy as np

from oracle import oracle as o


def idx(n, i, j, k):
    return ((k % n[2]) * n[1] + (j % n[1])) * n[0] + (i % n[0])


def test_plane_wave_dispersion():
    n = (16, 12, 4)
    d = (1.0, 1.3, 0.9)
    dt = 0.4
    m1, m2 = 3, 2
    kx, ky = 2 * math.pi * m1 / (n[0] * d[0]), 2 * math.pi * m2 / (n[1] * d[1])
    nc = int(np.prod(n))
    f = [np.zeros(nc) for _ in range(6)]
    J = [np.zeros(nc) for _ in range(3)]
    I, Jj, K = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    flat = ((K * n[1] + Jj) * n[0] + I).ravel()
    # E_z at (i, j, k+1/2), transverse to k in the x-y plane: div E = 0 exactly
    f[2][flat] = np.cos(kx * I * d[0] + ky * Jj * d[1]).ravel()
    basis = np.zeros(nc)
    basis[flat] = np.cos(kx * I * d[0] + ky * Jj * d[1]).ravel()
    a = []
    for _ in range(6):
        a.append(f[2] @ basis)
        o.yee_step(n, d, dt, f, J)
    a = np.array(a)
    cos_wdt = (a[2:] + a[:-2]) / (2 * a[1:-1])
    s = (math.sin(kx * d[0] / 2) / d[0]) ** 2 + (math.sin(ky * d[1] / 2) / d[1]) ** 2
    expect = 1 - 2 * dt * dt * s          # cos(w dt) = 1 - 2 sin^2(w dt/2)
    assert np.allclose(cos_wdt, expect, rtol=0, atol=1e-12)


def test_divB_preserved():
    rng = np.random.default_rng(0)
    n = (8, 6, 5)
    d = (1.0, 1.0, 1.0)
    nc = int(np.prod(n))
    f = [rng.standard_normal(nc) for _ in range(3)] + [np.zeros(nc) for _ in range(3)]
    J = [rng.standard_normal(nc) * 0.1 for _ in range(3)]
    for _ in range(5):
        o.yee_step(n, d, 0.3, f, J)
    Bx, By, Bz = f[3], f[4], f[5]
    worst = 0.0
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                # div B at the cell centre (i+1/2, j+1/2, k+1/2)
                dv = (Bx[idx(n, i + 1, j, k)] - Bx[idx(n, i, j, k)]) \
                   + (By[idx(n, i, j + 1, k)] - By[idx(n, i, j, k)]) \
                   + (Bz[idx(n, i, j, k + 1)] - Bz[idx(n, i, j, k)])
                worst = max(worst, abs(dv))
    assert worst < 1e-13
    assert np.abs(Bx).max() > 0.1


def test_cic_linear_exact():
    n = (6, 5, 7)
    d = (0.5, 2.0, 1.0)
    x0 = (-1.0, 3.0, 0.25)
    nc = int(np.prod(n))
    stag = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    coef = [(1.0, 2.0, -1.0, 0.5), (0.3, -0.2, 0.1, 1.0), (2.0, 0.0, 0.0, -1.0),
            (0.0, 1.0, 1.0, 0.0), (-1.0, 0.5, 2.0, 3.0), (0.7, 0.7, 0.7, 0.7)]
    f = []
    for c in range(6):
        a = np.zeros(nc)
        for k in range(n[2]):
            for j in range(n[1]):
                for i in range(n[0]):
                    X = [x0[0] + (i + stag[c][0]) * d[0], x0[1] + (j + stag[c][1]) * d[1],
                         x0[2] + (k + stag[c][2]) * d[2]]
                    a[idx(n, i, j, k)] = coef[c][0] * X[0] + coef[c][1] * X[1] + coef[c][2] * X[2] + coef[c][3]
        f.append(a)
    # interior points (away from the periodic seam, where the linear field jumps)
    for X in [(0.2, 5.1, 2.0), (-0.1, 7.9, 3.3), (0.77, 4.2, 5.5)]:
        E, B = o.gather(n, d, x0, f, X)
        got = list(E) + list(B)
        for c in range(6):
            want = coef[c][0] * X[0] + coef[c][1] * X[1] + coef[c][2] * X[2] + coef[c][3]
            assert abs(got[c] - want) < 1e-12


def test_esirkepov_continuity():
    rng = np.random.default_rng(3)
    n = (6, 7, 5)
    d = (1.0, 0.8, 1.2)
    x0 = (0.0, 0.0, 0.0)
    nc = int(np.prod(n))
    dt = 0.37
    npart = 60
    L = np.array(n) * np.array(d)
    xa = rng.uniform(0, 1, (npart, 3)) * L
    dx = rng.uniform(-0.9, 0.9, (npart, 3)) * np.array(d)
    xb = xa + dx
    qw = rng.uniform(-2, 2, npart)
    J = [np.zeros(nc) for _ in range(3)]
    for p in range(npart):
        o.deposit(n, d, x0, J, xa[p], xb[p], qw[p], dt)
    rho0 = o.charge_density(n, d, x0, xa[:, 0], xa[:, 1], xa[:, 2], qw)
    rho1 = o.charge_density(n, d, x0, xb[:, 0], xb[:, 1], xb[:, 2], qw)
    worst = 0.0
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                c = idx(n, i, j, k)
                div = (J[0][c] - J[0][idx(n, i - 1, j, k)]) / d[0] \
                    + (J[1][c] - J[1][idx(n, i, j - 1, k)]) / d[1] \
                    + (J[2][c] - J[2][idx(n, i, j, k - 1)]) / d[2]
                worst = max(worst, abs((rho1[c] - rho0[c]) / dt + div))
    assert worst < 1e-12
    dV = np.prod(d)
    for c in range(3):
        assert abs(J[c].sum() * dV - (qw * dx[:, c]).sum() / dt) < 1e-11


def div_nodes(n, d, F):
    """Discrete divergence at the nodes (i, j, k) of a field staggered like E
    and J (x component at (i+1/2, j, k), ...): backward differences."""
    a = [np.asarray(F[c]).reshape(n[2], n[1], n[0]) for c in range(3)]
    return ((a[0] - np.roll(a[0], 1, axis=2)) / d[0] + (a[1] - np.roll(a[1], 1, axis=1)) / d[1]
            + (a[2] - np.roll(a[2], 1, axis=0)) / d[2]).ravel()


def test_gauss_law_kept_by_the_field_update():
    # random E, B (the curl B part of the update has no discrete divergence)
    # and random charges moving less than a cell: the E update's current term
    # -4 pi alpha J must change div E by 4 pi alpha (rho1 - rho0) node by node
    rng = np.random.default_rng(8)
    n, d, x0, dt = (6, 7, 5), (1.0, 0.8, 1.2), (0.0, 0.0, 0.0), 0.37
    nc = int(np.prod(n))
    f = [rng.standard_normal(nc) for _ in range(6)]
    npart = 80
    L = np.array(n) * np.array(d)
    xa = rng.uniform(0, 1, (npart, 3)) * L
    xb = xa + rng.uniform(-0.9, 0.9, (npart, 3)) * np.array(d)
    qw = rng.uniform(-2, 2, npart) * 50.0
    J = [np.zeros(nc) for _ in range(3)]
    for p in range(npart):
        o.deposit(n, d, x0, J, xa[p], xb[p], qw[p], dt)
    rho0 = o.charge_density(n, d, x0, xa[:, 0], xa[:, 1], xa[:, 2], qw)
    rho1 = o.charge_density(n, d, x0, xb[:, 0], xb[:, 1], xb[:, 2], qw)
    div0 = div_nodes(n, d, f[:3])
    o.yee_step(n, d, dt, f, J)
    div1 = div_nodes(n, d, f[:3])
    want = 4 * math.pi * 7.2973525693e-3 * (rho1 - rho0)
    assert np.abs(want).max() > 1e-2                  # the charges do move
    scale = max(np.abs(div0).max(), np.abs(want).max())
    assert np.abs((div1 - div0) - want).max() < 1e-12 * scale


def test_step_current_is_continuous():
    # a whole step of the particle path on a mesh, deposit on: electrons
    # (charge -1), positrons (+1) and ions (+1) of unequal weights, and the
    # photons of an earlier step, some of which convert (pairs are born
    # co-located, so they add no net charge at birth).  The current the step
    # leaves in J obeys (rho_end - rho_start) / dt + div J = 0 at every node,
    # with rho from the positions before the step and after it
    from oracle import drive
    rng = np.random.default_rng(21)
    n, cell = (8, 8, 8), 2e4
    d, x0 = (cell,) * 3, (0.0, 0.0, 0.0)
    nc = int(np.prod(n))
    dt = 0.45 * cell / math.sqrt(3)
    f = [rng.standard_normal(nc) * 3e-2 for _ in range(6)]          # chi ~ 50
    parts = {}
    for sp, count in ((0, 400), (1, 400), (3, 150)):
        x = rng.uniform(0, 1, (count, 3)) * np.array(n) * cell
        u = rng.standard_normal((count, 3))
        pm = 50.0 if sp == 3 else 1000.0
        parts[sp] = (x, u / np.linalg.norm(u, axis=1)[:, None] * pm, rng.uniform(0.5, 2.0, count),
                     np.arange(count, dtype=np.uint64) + 10_000 * sp)
    common = dict(kappa=0.1, seed=2, caps=(20_000, 20_000, 40_000, 400))
    first, _, _, _ = drive.run(n, d, x0, (1, 1, 1), o.FIELD_GRID, (), dt, 1, parts,
                               fields=[a.copy() for a in f], **common)
    J = [np.zeros(nc) for _ in range(3)]
    out, D, _, _ = drive.run(n, d, x0, (1, 1, 1), o.FIELD_GRID, (), dt, 1, first, step0=1, t0=dt,
                             fields=[a.copy() for a in f], J=J, deposit_on=1, **common)
    assert D["emissions"] > 100 and D["pairs"] > 5, (D["emissions"], D["pairs"])
    charge = {0: -1.0, 1: 1.0, 3: 1.0}

    def rho(ps):
        acc = np.zeros(nc)
        for sp, q in charge.items():
            x, _, w, _ = ps[sp]
            if len(x):
                acc += o.charge_density(n, d, x0, x[:, 0], x[:, 1], x[:, 2], q * np.asarray(w))
        return acc
    drho = rho(out) - rho(first)
    res = drho / dt + div_nodes(n, d, J)
    scale = np.abs(drho).max() / dt
    assert scale > 0 and np.abs(res).max() < 1e-10 * scale, np.abs(res).max() / scale
