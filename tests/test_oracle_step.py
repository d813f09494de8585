"""Pins of the oracle's particle step (Sec. IV.F-H, V.A).

* Per-event conservation: emission and pair creation conserve 3-momentum, so in
  a uniform E field the weighted total momentum of all species grows exactly by
  sum q w E t of the particles present from the start (products of a pair
  carry opposite charges and cancel).  In a uniform B field the push conserves
  energy, so the total energy changes only by the closed-form defects of the
  events (emission: gamma - delta|p| - sqrt(1+(1-delta)^2 p^2); pairs:
  eps - sqrt(1+r^2 eps^2) - sqrt(1+(1-r)^2 eps^2)).
* Adaptive sub-stepping (Sec. IV.H): a few large steps agree statistically with
  many small steps that never subdivide (brute force), the paper's own
  small-vs-large time step check (Sec. VII).
* Pairs in the step (Sec. V.A): photons convert at the rate of Eq. (30) over
  the sub-intervals of Eq. (33), and split their momentum by its density.
* Products of a step evolve for exactly the rest of it (N - 1 - s sub-intervals).
* Boundaries: open boxes remove particles, periodic boxes wrap them, on all six faces.
* Analytic fields: the Gaussian pulse peaks at E0 at the focus, halves its
  intensity at +-tau/2, falls to 1/e at r = w0 and travels along -x at c.
"""
import math

import numpy as np
from scipy.stats import ks_2samp, kstest

from oracle import oracle as o

GAMMA0 = 1000.0
B_CHI1 = 1e-3     # chi = 1 for gamma = 1000 perpendicular to B


def electrons(n, gamma=GAMMA0, direction=(1.0, 0.0, 0.0), x=(0.0, 0.0, 0.0)):
    p = math.sqrt(gamma ** 2 - 1)
    return (np.tile(x, (n, 1)), np.tile(np.array(direction) * p, (n, 1)), np.ones(n),
            np.arange(n, dtype=np.uint64))


def big_periodic_box():
    return dict(n=(4, 4, 4), d=(1e9, 1e9, 1e9), x0=(-2e9, -2e9, -2e9), periodic=(1, 1, 1))


def total(run, key):
    out = 0.0
    for sp in run.sp:
        x, p, w, _ = sp.get()
        if key == "p":
            out = out + (w[:, None] * p).sum(axis=0)
    return out


def test_momentum_conservation_uniform_E():
    E = 2e-3
    P = o.make_params(field_mode=o.FIELD_UNIFORM, fp=(0, E, 0, 0, 0, 0), kappa=0.1, **big_periodic_box())
    run = o.Run(P, caps=(20000, 20000, 20000, 1))
    x, p, w, ids = electrons(200, gamma=3000.0)
    run.sp[0].set(x, p, w, ids)
    p0 = total(run, "p")
    dt = 2e5
    for s in range(4):
        run.step(s, s * dt, dt)
    D = run.diag()
    assert D["emissions"] > 50 and D["pairs"] > 0
    p1 = total(run, "p")
    expect = p0 + np.array([0.0, -1.0 * E * 4 * dt * 200, 0.0])
    assert np.allclose(p1, expect, rtol=1e-11, atol=1e-9 * np.abs(expect).max())


def test_energy_conservation_uniform_B():
    P = o.make_params(field_mode=o.FIELD_UNIFORM, fp=(0, 0, 0, 0, 0, 2e-2), kappa=0.1, **big_periodic_box())
    run = o.Run(P, caps=(20000, 20000, 20000, 1))
    x, p, w, ids = electrons(100, gamma=500.0)
    run.sp[0].set(x, p, w, ids)

    def energy():
        e = 0.0
        for k, sp in enumerate(run.sp[:3]):
            _, pp, ww, _ = sp.get()
            m2 = 0.0 if k == 2 else 1.0
            e += (ww * np.sqrt(m2 + (pp ** 2).sum(1))).sum()
        return e
    e0 = energy()
    for s in range(3):
        run.step(s, 0.0, 3e4)
    D = run.diag()
    assert D["emissions"] > 30 and D["pairs"] > 0
    assert abs(energy() + D["energy_defect"] - e0) < 1e-10 * e0
    # defects are tiny: at most ~ 1/gamma per event relative to the event energy
    assert abs(D["energy_defect"]) < 1e-3 * e0


def test_free_streaming_velocity():
    # no field: each step moves a particle by p / sqrt(m^2 + p^2) dt (c = 1),
    # for an electron (m = 1) and a proton (m = 1836.15)
    P = o.make_params(field_mode=o.FIELD_UNIFORM, fp=(0,) * 6, kappa=0.1, **big_periodic_box())
    run = o.Run(P, caps=(4, 1, 4, 4))
    pv = np.array([[500.0, -300.0, 100.0]])
    for sp in (0, 3):
        run.sp[sp].set(np.zeros((1, 3)), pv, [1.0], [sp])
    dt, n = 1e3, 5
    for s in range(n):
        run.step(s, s * dt, dt)
    for sp, m in ((0, 1.0), (3, 1836.15267343)):
        x, p, _, _ = run.sp[sp].get()
        assert np.allclose(p, pv, rtol=0, atol=0)
        assert np.allclose(x[0], n * dt * pv[0] / math.sqrt(m * m + pv[0] @ pv[0]), rtol=1e-13, atol=0), sp


def test_ions_never_emit():
    # ions are pushed with their charge and mass and take no part in the
    # event generators: a proton at p = 1e6 m_e c across a strong B (chi would
    # be ~1e3 for an electron of that momentum) keeps |p| and makes nothing
    P = o.make_params(field_mode=o.FIELD_UNIFORM, fp=(0, 0, 0, 0, 0, 1e-3), kappa=0.1, emission_on=1, pairs_on=1,
                      **big_periodic_box())
    run = o.Run(P, caps=(16, 16, 16, 64))
    n = 64
    run.sp[3].set(np.zeros((n, 3)), np.tile([1e6, 0.0, 0.0], (n, 1)), np.ones(n), np.arange(n, dtype=np.uint64))
    for s in range(3):
        run.step(s, s * 1e5, 1e5)
    D = run.diag()
    assert D["emissions"] == D["photons_created"] == D["substeps_lepton"] == 0
    assert run.sp[0].n == run.sp[1].n == run.sp[2].n == 0 and run.sp[3].n == n
    _, p, _, _ = run.sp[3].get()
    assert np.allclose(np.linalg.norm(p, axis=1), 1e6, rtol=1e-13, atol=0)
    assert np.all(p[:, 1] < -100.0)                   # it did turn in the field (q v x B along -y)


def test_radiated_power_at_small_chi():
    # the modified generator emits the whole spectrum, so the radiation
    # reaction of the low-energy limit needs no classical term (Sec. IV.G):
    # electrons at chi = 0.01 in a uniform B lose energy at the quantum-
    # corrected synchrotron power alpha (2/3) chi^2 (1 - 5.95 chi + 48 chi^2)
    # per Compton time, 5.5% below the classical (2/3) alpha chi^2, which the
    # sample resolves (its statistical error is 0.5%)
    g0, chi0, n, dt, nsteps = 1000.0, 0.01, 80000, 1e6, 20
    p0 = math.sqrt(g0 ** 2 - 1)
    P = o.make_params(field_mode=o.FIELD_UNIFORM, fp=(0, 0, 0, 0, 0, chi0 / p0), kappa=1e9, pairs_on=0,
                      same_step_children=0, **big_periodic_box())
    run = o.Run(P, caps=(n, 1, 20 * n, 1))
    run.sp[0].set(np.zeros((n, 3)), np.tile([p0, 0.0, 0.0], (n, 1)), np.ones(n), np.arange(n, dtype=np.uint64))
    for s in range(nsteps):
        run.step(s, s * dt, dt)
    D = run.diag()
    assert D["pm_gt1"] == 0 and D["emissions"] > 100000
    _, pe, _, _ = run.sp[0].get()
    _, k, _, _ = run.sp[2].get()
    loss = g0 - np.sqrt(1 + (pe ** 2).sum(1))
    assert np.isclose(loss.sum(), np.linalg.norm(k, axis=1).sum(), rtol=1e-6)   # carried off by photons
    alpha = 7.2973525693e-3
    chi_mid = chi0 * (1 - 0.5 * loss.mean() / g0)      # chi ~ gamma falls ~1% over the run
    power = alpha * (2 / 3) * chi_mid ** 2 * (1 - 5.95 * chi_mid + 48 * chi_mid ** 2)
    err = loss.std() / math.sqrt(n)
    assert abs(loss.mean() - power * nsteps * dt) < 4 * err, (loss.mean(), power * nsteps * dt, err)
    assert abs(loss.mean() - alpha * (2 / 3) * chi_mid ** 2 * nsteps * dt) > 8 * err


def test_full_store_counts_what_it_drops():
    # a photon store of capacity 5: emissions beyond it are lost and counted,
    # and the store never holds more than its capacity
    P = o.make_params(field_mode=o.FIELD_UNIFORM, fp=(0, 0, 0, 0, 0, B_CHI1), kappa=0.1, pairs_on=0,
                      same_step_children=0, **big_periodic_box())
    run = o.Run(P, caps=(200, 1, 5, 1))
    run.sp[0].set(*electrons(200))
    run.step(0, 0.0, 2e5)
    D = run.diag()
    assert D["emissions"] > 20
    assert run.sp[2].n == 5 and D["overflow"] == D["photons_created"] - 5


def test_boundaries_open_and_periodic():
    # one photon leaves through each of the six faces of a 10^3 box in one
    # step: an open box removes all six, a periodic one wraps each to the
    # opposite face, half a cell inside
    x0 = [[9.5, 5, 5], [0.5, 5, 5], [5, 9.5, 5], [5, 0.5, 5], [5, 5, 9.5], [5, 5, 0.5]]
    k = [[2, 0, 0], [-2, 0, 0], [0, 2, 0], [0, -2, 0], [0, 0, 2], [0, 0, -2]]
    wrapped = {7: [0.5, 5, 5], 8: [9.5, 5, 5], 9: [5, 0.5, 5], 10: [5, 9.5, 5], 11: [5, 5, 0.5], 12: [5, 5, 9.5]}
    for periodic in (0, 1):
        P = o.make_params(n=(10, 10, 10), d=(1.0, 1.0, 1.0), x0=(0.0, 0.0, 0.0), periodic=(periodic,) * 3,
                          field_mode=o.FIELD_UNIFORM, fp=(0,) * 6, pairs_on=1)
        run = o.Run(P, caps=(1, 1, 8, 1))
        run.sp[2].set(np.array(x0, float), np.array(k, float), np.ones(6), np.arange(7, 13))
        run.step(0, 0.0, 1.0)
        if periodic:
            x, _, _, ids = run.sp[2].get()
            assert sorted(ids.tolist()) == list(range(7, 13))
            for xi, i in zip(x, ids):
                assert np.abs(xi - wrapped[int(i)]).max() < 1e-14, (i, xi)
        else:
            assert run.sp[2].n == 0
            assert run.diag()["absorbed"] == 6


def run_stats(dt, nsteps, kappa, n=800, seed=11):
    T_chi = dict(field_mode=o.FIELD_UNIFORM, fp=(0, 0, 0, 0, 0, B_CHI1))
    P = o.make_params(kappa=kappa, pairs_on=0, seed=seed, **T_chi, **big_periodic_box())
    run = o.Run(P, caps=(n, 1, 40 * n, 1))
    x, p, w, ids = electrons(n)
    run.sp[0].set(x, p, w, ids)
    for s in range(nsteps):
        run.step(s, s * dt, dt)
    _, pe, _, _ = run.sp[0].get()
    _, pg, _, _ = run.sp[2].get()
    ge = np.sqrt(1 + (pe ** 2).sum(1))
    eg = np.sqrt((pg ** 2).sum(1))
    return run.diag(), ge, eg


def test_adaptive_substeps_match_brute_force():
    T = 0.02 * 2 * math.pi * GAMMA0 / B_CHI1      # 0.02 gyro periods, ~1 photon per electron
    Da, ga, ea = run_stats(T / 2, 2, 0.1)          # AEG: N ~ 7 sub-steps per step
    Db, gb, eb = run_stats(T / 300, 300, 1e9, seed=12)   # never subdivides, P_m ~ 1e-3
    assert Da["substeps_lepton"] > 5 * 2 * 800
    assert Db["substeps_lepton"] == 300 * 800
    na, nb = Da["emissions"], Db["emissions"]
    assert abs(na - nb) < 4 * math.sqrt(na + nb)
    assert abs(ga.mean() - gb.mean()) < 4 * math.hypot(ga.std() / math.sqrt(len(ga)), gb.std() / math.sqrt(len(gb)))
    assert ks_2samp(ea, eb).pvalue > 1e-3
    # non-emitting electrons form an atom at gamma0; round away last-ulp differences of the push
    assert ks_2samp(np.round(ga, 6), np.round(gb, 6)).pvalue > 1e-3


def test_children_modes():
    # with products evolving in the same step, photons born in step 0 already
    # move in step 0: a photon born in sub-interval s of N flies at c for the
    # rest of the step, (N - 1 - s) h, along its momentum
    common = dict(field_mode=o.FIELD_UNIFORM, fp=(0, 0, 0, 0, 0, B_CHI1), kappa=0.1, pairs_on=0,
                  **big_periodic_box())
    dt, n_e = 2e5, 300
    res = {}
    for mode in (0, 1):
        P = o.make_params(same_step_children=mode, **common)
        run = o.Run(P, caps=(n_e, 1, 3000, 1))
        run.sp[0].set(*electrons(n_e))
        run.step(0, 0.0, dt)
        x, p, _, ids = run.sp[2].get()
        order = np.argsort(ids)
        res[mode] = (x[order], p[order], ids[order], run.diag())
    # identical events (same streams), only the photon positions differ
    assert len(res[0][0]) == len(res[1][0]) > 20
    assert np.array_equal(res[0][2], res[1][2])
    assert np.array_equal(res[0][1], res[1][1])
    # identical electrons take the same number N of sub-intervals
    n_sub = res[1][3]["substeps_lepton"] / n_e
    assert n_sub == int(n_sub) > 4
    n_sub = int(n_sub)
    flown = res[1][0] - res[0][0]
    k_hat = res[1][1] / np.linalg.norm(res[1][1], axis=1)[:, None]
    assert np.allclose(np.cross(flown, k_hat), 0.0, atol=1e-9 * dt)     # along k
    rest = np.einsum("ij,ij->i", flown, k_hat) / (dt / n_sub)          # in sub-intervals
    assert np.abs(rest - np.round(rest)).max() < 1e-9
    assert rest.min() > -0.5 and rest.max() < n_sub - 0.5               # 0 .. N - 1
    # births in the first and in the last sub-interval both occur
    assert np.isclose(rest.max(), n_sub - 1) and np.isclose(rest.min(), 0.0)


def test_pair_products_evolve_for_the_rest_of_the_step():
    # photons along x in a uniform E along y convert; with emission off a
    # lepton takes one push over its remaining time, which in a pure E field
    # is exact: p gains q E t_rem.  A pair born in sub-interval s of the
    # photon's N has t_rem = (N - 1 - s) h, so t_rem / h is an integer in
    # 0 .. N - 1, and with products starting at the next step it is 0
    E, eps, dt, n_g = 2e-3, 1e4, 4e5, 300
    common = dict(field_mode=o.FIELD_UNIFORM, fp=(0, E, 0, 0, 0, 0), kappa=0.1, pairs_on=1, emission_on=0,
                  **big_periodic_box())
    out = {}
    for mode in (0, 1):
        P = o.make_params(same_step_children=mode, **common)
        run = o.Run(P, caps=(2000, 2000, n_g, 1))
        run.sp[2].set(np.zeros((n_g, 3)), np.tile([eps, 0.0, 0.0], (n_g, 1)), np.ones(n_g),
                      np.arange(n_g, dtype=np.uint64))
        run.step(0, 0.0, dt)
        D = run.diag()
        got = {}
        for sp in (0, 1):
            _, p, _, ids = run.sp[sp].get()
            order = np.argsort(ids)
            got[sp] = (p[order], ids[order])
        out[mode] = (got, D)
    D = out[1][1]
    # k perpendicular to E, no B: H_eff of Eq. (32) is |E|, and Eq. (33)
    # with lambda_C / c = 2 pi Compton times bounds the sub-interval
    n_sub = math.ceil(dt / (0.1 * 130.0 * 2.0 * math.pi / E))
    assert D["pairs"] > 50 and n_sub > 4
    h = dt / n_sub
    for sp, q in ((0, -1.0), (1, 1.0)):
        (p0, i0), (p1, i1) = out[0][0][sp], out[1][0][sp]
        assert np.array_equal(i0, i1)
        # born with a share of the photon's momentum along x; E changes only p_y
        assert np.array_equal(p0[:, [0, 2]], p1[:, [0, 2]]) and np.all(p0[:, 1] == 0.0)
        rest = p1[:, 1] / (q * E * h)
        assert np.abs(rest - np.round(rest)).max() < 1e-6
        assert rest.min() > -0.5 and rest.max() < n_sub - 0.5
        assert np.isclose(rest.max(), n_sub - 1) and np.isclose(rest.min(), 0.0)


def test_pair_step_converts_at_the_rate_and_splits_by_its_density():
    # photons of energy eps along x in a uniform E along y (chi_g = eps |E|,
    # Eq. (31)): in each of the N sub-intervals of Eq. (33) a photon converts
    # with probability w = int_0^1 P_p(d) dd (Eq. (30); P_p < 1 here, and the
    # generator accepts r2 < P_p(r1)), so a fraction 1 - (1 - w)^N converts in
    # the step, and the electron's share of the photon momentum is
    # distributed as P_p
    E, eps, dt, n_g = 2e-3, 1e4, 4e5, 4000
    P = o.make_params(field_mode=o.FIELD_UNIFORM, fp=(0, E, 0, 0, 0, 0), kappa=0.1, pairs_on=1,
                      emission_on=0, same_step_children=0, **big_periodic_box())
    run = o.Run(P, caps=(n_g, n_g, n_g, 1))
    run.sp[2].set(np.zeros((n_g, 3)), np.tile([eps, 0.0, 0.0], (n_g, 1)), np.ones(n_g),
                  np.arange(n_g, dtype=np.uint64))
    run.step(0, 0.0, dt)
    D = run.diag()
    n_sub = math.ceil(dt / (0.1 * 130.0 * 2.0 * math.pi / E))
    h, chig = dt / n_sub, eps * E
    grid = np.linspace(0.0, 1.0, 4001)
    dens = np.array([o.Pp(d, chig, eps, h) for d in grid])
    assert dens.max() < 1.0
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(grid))])
    w = cdf[-1]
    expect = n_g * (1.0 - (1.0 - w) ** n_sub)
    assert abs(D["pairs"] - expect) < 4.0 * math.sqrt(expect * (1.0 - expect / n_g)), (D["pairs"], expect)
    _, pe, _, _ = run.sp[0].get()
    _, pp, _, _ = run.sp[1].get()
    assert len(pe) == len(pp) == D["pairs"] > 1000
    assert np.allclose(pe[:, 0] + pp[:, 0], eps, rtol=1e-15, atol=0)
    assert kstest(pe[:, 0] / eps, lambda x: np.interp(x, grid, cdf / w)).pvalue > 1e-3


def test_energy_spectrum_is_the_photons_energies():
    # with pairs off every emitted photon stays in the store and keeps its
    # momentum, so the diagnostic spectrum over log10(photon energy) is the
    # weighted histogram of log10|k| of the stored photons, bin by bin
    from oracle import drive
    n_e, nbins, lo, hi = 400, 64, -12.0, 4.0
    x, p, _, ids = electrons(n_e)
    w = 1.0 + np.arange(n_e) % 3                       # unequal weights
    out, D, spec, spec_e = drive.run(
        (4, 4, 4), (1e9,) * 3, (-2e9,) * 3, (1, 1, 1), o.FIELD_UNIFORM, (0, 0, 0, 0, 0, B_CHI1),
        2e5, 3, {0: (x, p, w, ids)}, kappa=0.1, seed=5, pairs_on=0, same_step_children=0,
        caps=(n_e, 1, 40 * n_e, 1), nbins=nbins, lg_lo=lo, lg_hi=hi)
    _, k, wk, _ = out[2]
    assert D["emissions"] == len(k) > 200
    hist, _ = np.histogram(np.log10(np.linalg.norm(k, axis=1)), bins=nbins, range=(lo, hi), weights=wk)
    assert np.allclose(spec_e, hist, rtol=1e-12, atol=0)
    assert spec_e.sum() == wk.sum()


def test_gaussian_pulse_properties():
    E0, w, w0, tau = 6e-4, 3e-6, 5e6, 2e7
    fp = (E0, w, w0, tau, 0.0, 0.0, 0.0, 0.0, 0.0)
    E, B = o.field(o.FIELD_GAUSSIAN_LP, fp, (0, 0, 0), 0.0)
    assert abs(E[1] - E0) < 1e-18 and B[2] == -E[1] and E[0] == E[2] == 0
    # intensity half maximum at t = +-tau/2 on the envelope (carrier phase removed)
    for t in (tau / 2, -tau / 2):
        Et, _ = o.field(o.FIELD_GAUSSIAN_LP, fp[:8] + (-w * t,), (0, 0, 0), t)
        assert abs((Et[1] / E0) ** 2 - 0.5) < 1e-12
    # 1/e at r = w0 in the focal plane
    Er, _ = o.field(o.FIELD_GAUSSIAN_LP, fp, (0, w0, 0), 0.0)
    assert abs(Er[1] / E0 - math.exp(-1)) < 1e-12
    # travels along -x at c: the same field value at (x - c dt, t + dt) up to diffraction
    Ea, _ = o.field(o.FIELD_GAUSSIAN_LP, fp, (0, 0, 0), 0.0)
    Eb, _ = o.field(o.FIELD_GAUSSIAN_LP, fp, (-1e3, 0, 0), 1e3)
    assert abs(Eb[1] / Ea[1] - 1) < 1e-6
    # rotating E
    Er, Br = o.field(o.FIELD_ROTATING_E, (2.0, 0.5), (1, 2, 3), 1.3)
    assert abs(math.hypot(Er[0], Er[1]) - 2.0) < 1e-15 and abs(math.atan2(Er[1], Er[0]) - 0.65) < 1e-15
    assert not Br.any()


def test_gaussian_pulse_solves_the_wave_equation():
    # the pulse is a paraxial solution of the vacuum wave equation: at random
    # points of the focal region (two Rayleigh lengths each side, out to 1.2
    # w0, within the envelope) the residual of (laplacian - d^2/dt^2) E_y,
    # by central differences, stays within the paraxial error, of order
    # theta^4 k^2 E0 with theta = 2 / (k w0).  A wrong Rayleigh length, beam
    # width, amplitude factor w0/w(x) or Gouy phase sign leaves a residual of
    # order theta^2 (measured 20 to 140 times this one)
    rng = np.random.default_rng(3)
    E0, w, w0, tau = 1.0, 1.0, 15.7, 70.7            # units of 1/k: the collision's w0 and duration
    fp = (E0, w, w0, tau, 0.0, 0.0, 0.0, 0.0, 0.3)
    zr, theta, s = 0.5 * w * w0 * w0, 2.0 / (w * w0), 0.02

    def Ey(x, t):
        return o.field(o.FIELD_GAUSSIAN_LP, fp, x, t)[0][1]
    worst = 0.0
    for _ in range(200):
        zeta = rng.uniform(-2, 2) * zr
        r, ph = rng.uniform(0, 1.2) * w0, rng.uniform(0, 2 * math.pi)
        x = np.array([-zeta, r * math.cos(ph), r * math.sin(ph)])
        t = rng.uniform(-0.5, 0.5) * tau + zeta
        c = Ey(x, t)
        lap = sum((Ey(x + e, t) - 2 * c + Ey(x - e, t)) / s ** 2 for e in np.eye(3) * s)
        dtt = (Ey(x, t + s) - 2 * c + Ey(x, t - s)) / s ** 2
        worst = max(worst, abs(lap - dtt))
    assert worst < 4 * theta ** 4 * w * w * E0, worst


def test_standing_wave_field():
    """The standing wave of the avalanche benchmark (Sec. VII.C): at t = 0
    only E_y = E0 sin(2 pi x/lambda); at all times a vacuum solution of
    Maxwell's equations (checked by central differences, c = 1):
    dBz/dt = -dEy/dx and dEy/dt = -dBz/dx; |E| + |B| <= E0."""
    lam = 2.5896e6
    w = 2 * math.pi / lam
    E0 = 1e-2
    fp = (E0, w)
    E, B = o.field(o.FIELD_STANDING_WAVE, fp, (lam / 8, 7.0, -3.0), 0.0)
    assert abs(E[1] - E0 * math.sqrt(0.5)) < 1e-17 and E[0] == E[2] == 0 and not np.any(B)
    E, B = o.field(o.FIELD_STANDING_WAVE, fp, (lam / 4, 0, 0), 0.0)
    assert abs(E[1] - E0) < 1e-17
    rng = np.random.default_rng(3)
    h = lam * 1e-5
    for x, t in rng.uniform(0, 3 * lam, (20, 2)):
        Ey = lambda xx, tt: o.field(o.FIELD_STANDING_WAVE, fp, (xx, 0, 0), tt)[0][1]
        Bz = lambda xx, tt: o.field(o.FIELD_STANDING_WAVE, fp, (xx, 0, 0), tt)[1][2]
        dEdx = (Ey(x + h, t) - Ey(x - h, t)) / (2 * h)
        dEdt = (Ey(x, t + h) - Ey(x, t - h)) / (2 * h)
        dBdx = (Bz(x + h, t) - Bz(x - h, t)) / (2 * h)
        dBdt = (Bz(x, t + h) - Bz(x, t - h)) / (2 * h)
        scale = E0 * w
        assert abs(dBdt + dEdx) < 1e-6 * scale and abs(dEdt + dBdx) < 1e-6 * scale
        E, B = o.field(o.FIELD_STANDING_WAVE, fp, (x, 0, 0), t)
        assert abs(E[1]) + abs(B[2]) <= E0 * (1 + 1e-15)
        assert E[0] == E[2] == B[0] == B[1] == 0


def test_pulse_reproducible_under_origin_shift():
    """The FP64 oracle in the focused pulse (the collision workload, 40 seed
    electrons and their products over 600 steps) against itself with the
    coordinate origin shifted by 3e7 Compton lengths: the same physics, but
    the pulse's phase at an absolute FP64 position carries |x| 2^-53 of
    rounding.  Every particle (ids identical) agrees to 1e-12 of
    max(|p|, a0), a0 the field's momentum scale -- the scale to which the
    GPU's FP64 path is held in this field -- while particles born slow
    (soft photons, pairs) differ by far more than 1e-12 of their own
    momentum."""
    import copy
    from paper_1412_6426_gb300 import workloads
    from tests.util import run_oracle
    w = workloads.beam_laser_collision(n_particles=1_000_000, seed=1, nsteps=600)
    idx = np.sort(np.random.default_rng(12).choice(len(w.particles[0][3]), 40, replace=False))
    ws = workloads.subset(w, 0, idx)
    shift = 3.0e7
    wb = copy.deepcopy(ws)
    wb.x0 = (ws.x0[0] + shift, ws.x0[1], ws.x0[2])
    fp = list(ws.fp)
    fp[4] += shift                        # the focus moves with the origin
    wb.fp = tuple(fp)
    x, p, wt, ids = ws.particles[0]
    wb.particles = {0: (x + np.array([shift, 0.0, 0.0]), p, wt, ids)}
    caps = (50_000, 50_000, 400_000, 1)
    a, _, _, _ = run_oracle(ws, caps=caps)
    b, _, _, _ = run_oracle(wb, caps=caps)
    a0 = w.meta["a0"]
    worst_rel = worst_scaled = 0.0
    for sp in range(3):
        assert np.array_equal(np.sort(a[sp][3]), np.sort(b[sp][3]))
        _, i, j = np.intersect1d(a[sp][3], b[sp][3], return_indices=True)
        d = np.linalg.norm(a[sp][1][i] - b[sp][1][j], axis=1)
        m = np.linalg.norm(a[sp][1][i], axis=1)
        worst_rel = max(worst_rel, float((d / m).max()))
        worst_scaled = max(worst_scaled, float((d / np.maximum(m, a0)).max()))
    assert worst_scaled <= 1e-12
    assert worst_rel > 1e-12
