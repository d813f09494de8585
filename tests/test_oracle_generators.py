"""Pins of the oracle's standard and alternative event generators (Sec. IV.F)
and of the three-generator comparison (Sec. IV.G, the paper's Fig.
"generators": gamma = 100, chi = 1).

* Standard generator (inverse transform with delta_min -> 0): the oracle's
  normalised W(x) = int_0^x G(delta, chi) d delta against scipy's Bessel-K
  quadrature (independent of the oracle), its total W(1) against the same,
  and the photon energy it returns for r2 against the root of scipy's CDF.
  The 8-point Gauss-Legendre rule W is integrated with (its nodes found by
  Newton's method on P_8) against mpmath's roots of P_8 and their weights.
* Frozen spectra: for each generator the expected count per log-delta bin
  is known in closed form from the emission density P of Eq. (24):
    modified:    ndraw int_bin P,
    alternative: ndraw int_bin min(P, 1)   (it under-samples where P > 1,
                 the low-energy region the paper points out),
    standard:    ndraw W(1) (CDF(bin_hi) - CDF(bin_lo)).
  The sampled histograms agree with these within 4 sigma.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as o
from tests.test_oracle_generator import ALPHA, scipy_P


def scipy_G(delta, chi):
    # the density without the prefactor alpha h / gamma
    return scipy_P(delta, chi, 1.0, 1.0 / ALPHA)


def scipy_W(x, chi):
    # int_0^x G d delta in s = delta^(1/3) (finite integrand at s = 0)
    return quad(lambda s: 3 * s * s * scipy_G(s ** 3, chi), 0.0, x ** (1 / 3), limit=400, epsabs=0,
                epsrel=1e-12)[0]


def test_standard_total_and_cdf_against_scipy():
    for chi in (0.1, 1.0, 10.0):
        w1 = scipy_W(1.0 - 1e-15, chi)
        assert math.isclose(o.Wnorm(1.0, chi), w1, rel_tol=1e-9), chi
        for x in (1e-9, 1e-4, 0.05, 0.3, 0.7, 0.95):
            assert math.isclose(o.Wnorm(x, chi) / o.Wnorm(1.0, chi), scipy_W(x, chi) / w1, rel_tol=1e-8,
                                abs_tol=1e-13), (chi, x)
    # at chi = 1 the total is the number rate 1.033914 (the smooth s-integral)
    assert abs(o.Wnorm(1.0, 1.0) - 1.033914) < 2e-6


def test_standard_energy_is_the_inverse_cdf():
    chi = 1.0
    w1 = scipy_W(1.0 - 1e-15, chi)
    for r2 in (1e-8, 0.01, 0.25, 0.5, 0.9, 0.999):
        d = o.delta_std(chi, r2)
        assert 0.0 < d < 1.0
        assert abs(scipy_W(d, chi) / w1 - r2) < 1e-9 * max(r2, 1e-3), (r2, d)


def _expected(generator, chi, gamma, h, ndraw, edges):
    out = []
    if generator == o.GEN_STANDARD:
        w1 = scipy_W(1.0 - 1e-15, chi)
        pstd = ALPHA * h / gamma * w1
        cdf = [scipy_W(10 ** e, chi) / w1 for e in edges]
        return ndraw * pstd * np.diff(cdf)
    for i in range(len(edges) - 1):
        f = (lambda u: scipy_P(10 ** u, chi, gamma, h) * 10 ** u * math.log(10)) if generator == o.GEN_MODIFIED \
            else (lambda u: min(scipy_P(10 ** u, chi, gamma, h), 1.0) * 10 ** u * math.log(10))
        out.append(ndraw * quad(f, edges[i], edges[i + 1], limit=200)[0])
    return np.array(out)


def test_three_generators_frozen_spectra():
    gamma, chi = 100.0, 1.0
    lo, hi, nb = -10.0, 0.0, 20
    edges = np.linspace(lo, hi, nb + 1)
    for gen, h, ndraw in ((o.GEN_MODIFIED, 0.1 * gamma / (ALPHA * 1.6), 200_000),
                          (o.GEN_ALTERNATIVE, 0.1 * gamma / (ALPHA * 1.6), 200_000),
                          (o.GEN_STANDARD, 0.5 * gamma / (ALPHA * 1.04), 3000)):
        acc, hist, viol = o.sample_frozen_gen(gen, chi, gamma, h, ndraw, 11, lo, hi, nb)
        exp = _expected(gen, chi, gamma, h, ndraw, edges)
        sig = np.sqrt(np.maximum(exp, 1.0))
        z = (hist - exp) / sig
        assert np.all(np.abs(z) < 4.0), (gen, z)
        if gen == o.GEN_ALTERNATIVE:
            # P(delta) > 1 at low delta: the alternative generator misses photons there
            assert viol > 0
            full = _expected(o.GEN_MODIFIED, chi, gamma, h, ndraw, edges)
            assert hist[0] < 0.5 * full[0]
        if gen == o.GEN_MODIFIED:
            assert viol == 0 and hist[0] > 0


def test_generators_in_the_particle_step_conserve_what_they_should():
    # uniform E: 3-momentum of all species grows exactly by sum q w E t (the
    # events split momentum exactly, whatever the generator); uniform B: the
    # energy changes only by the closed-form defects the diagnostics add up
    box = dict(n=(4, 4, 4), d=(1e9, 1e9, 1e9), x0=(-2e9, -2e9, -2e9), periodic=(1, 1, 1))
    for gen in (o.GEN_ALTERNATIVE, o.GEN_STANDARD):
        E = 2e-3
        P = o.make_params(field_mode=o.FIELD_UNIFORM, fp=(0, E, 0, 0, 0, 0), kappa=0.1, generator=gen, **box)
        run = o.Run(P, caps=(4000, 4000, 8000, 1))
        n = 12
        p0 = math.sqrt(3000.0 ** 2 - 1)
        run.sp[0].set(np.zeros((n, 3)), np.tile([p0, 0, 0], (n, 1)), np.ones(n), np.arange(n, dtype=np.uint64))
        dt = 2e5
        for s in range(2):
            run.step(s, s * dt, dt)
        D = run.diag()
        assert D["emissions"] > 5, gen
        tot = np.zeros(3)
        for sp in run.sp:
            x, pp, w, _ = sp.get()
            tot += (w[:, None] * pp).sum(0)
        expect = np.array([n * p0, -E * 2 * dt * n, 0.0])
        assert np.allclose(tot, expect, rtol=1e-11, atol=1e-9 * np.abs(expect).max()), gen
        assert D["photons_created"] == D["emissions"]


def test_step_emits_the_generator_densities():
    # the same spectra through the particle step itself (the code path of a
    # run, not the frozen sampler): electrons with gamma = 100, perpendicular
    # to a static B with chi = 1, one step of one sub-interval.  The push in B
    # keeps |p|, so chi and gamma hold at the event and delta = |k| / |p0|.
    # The standard generator integrates W(1) for every particle (about 5 ms
    # each), so it runs fewer electrons at a larger P = W(1); an unbounded
    # margin kappa keeps its step one sub-interval long
    gamma, chi = 100.0, 1.0
    p0 = math.sqrt(gamma ** 2 - 1)
    lo, hi, nb = -10.0, 0.0, 20
    edges = np.linspace(lo, hi, nb + 1)
    for gen, h, n, kappa in ((o.GEN_MODIFIED, 0.1 * gamma / (ALPHA * 1.6), 200_000, 0.1),
                             (o.GEN_ALTERNATIVE, 0.1 * gamma / (ALPHA * 1.6), 200_000, 0.1),
                             (o.GEN_STANDARD, 0.5 * gamma / (ALPHA * 1.04), 2_000, 1e9)):
        P = o.make_params(n=(4, 4, 4), d=(1e9,) * 3, x0=(-2e9,) * 3, periodic=(1, 1, 1),
                          field_mode=o.FIELD_UNIFORM, fp=(0, 0, 0, 0, 0, chi / p0), kappa=kappa, pairs_on=0,
                          generator=gen, seed=5)
        run = o.Run(P, caps=(n, 1, n, 1))
        x = np.zeros((n, 3))
        p = np.zeros((n, 3))
        p[:, 0] = p0
        run.sp[0].set(x, p, np.ones(n), np.arange(n, dtype=np.uint64))
        run.step(0, 0.0, h)
        assert run.diag()["substeps_lepton"] == n              # one sub-interval each
        _, k, _, _ = run.sp[2].get()
        delta = np.linalg.norm(k, axis=1) / p0
        hist, _ = np.histogram(np.log10(delta), bins=edges)
        exp = _expected(gen, chi, gamma, h, n, edges)
        sig = np.sqrt(np.maximum(exp, 1.0))
        assert np.all(np.abs(hist - exp) <= 4 * sig + 1e-9), (gen, hist, exp)


def test_gauss_legendre_rule_of_the_standard_generator():
    # the oracle's rule (nodes found by Newton's method on P_8) against
    # mpmath's roots of P_8 and the weights 2 / ((1 - x^2) P_8'(x)^2)
    mpmath = pytest.importorskip("mpmath")
    xs, ws = o.gauss_legendre8()
    mpmath.mp.dps = 30
    P8 = lambda t: mpmath.legendre(8, t)
    roots = sorted(float(mpmath.findroot(P8, math.cos(math.pi * (i + 0.75) / 8.5))) for i in range(4))
    roots = [-r for r in roots[::-1]] + roots
    for x, w, r in zip(xs, ws, roots):
        wt = float(2 / ((1 - mpmath.mpf(r) ** 2) * mpmath.diff(P8, mpmath.mpf(r)) ** 2))
        assert abs(x - r) <= math.ulp(r) and abs(w - wt) <= 8 * math.ulp(wt), (x, r, w, wt)
    assert abs(ws.sum() - 2.0) < 1e-15
