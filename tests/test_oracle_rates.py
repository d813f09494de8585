"""Pins of the oracle's emission and pair rates.

Eq. (24) P(delta), Eq. (25) P_m, Eq. (30) P_p, Eq. (27)-(29) and (33) time-step
bounds.  Pinned against: the classical radiated power of Sec. IV.C
(I_cl = (2/3) alpha chi^2 in Compton units) including the known quantum
correction 1 - (55 sqrt3/16) chi + 48 chi^2; the large-chi power I_q ~ 0.37 chi^(2/3)
(Sec. IV.D); the small-delta asymptote 0.52 chi^(2/3) delta^(-2/3) printed in
Sec. IV.F together with its closed form; the Erber small-chi_gamma asymptote of
the Breit-Wheeler rate; the delta_e <-> 1-delta_e symmetry of Eq. (30); and the
paper's bounds on max P_m (Sec. IV.H).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import gamma as Gamma
from scipy.special import kv

from oracle import oracle as o

ALPHA = 7.2973525693e-3


def log_quad(f, lo, hi):
    """int_lo^hi f(d) dd, integrated in u = ln d."""
    return quad(lambda u: f(math.exp(u)) * math.exp(u), math.log(lo), math.log(hi),
                limit=400, epsabs=0, epsrel=1e-11)[0]


def scipy_F1(x):
    # int_x^inf K_{5/3} = 2 K_{2/3}(x) - int_x^inf K_{1/3}  (K_{nu-1} + K_{nu+1} = -2 K'_nu)
    if x > 1.0:
        i13 = quad(lambda t: kv(1 / 3, t), x, np.inf, limit=500, epsabs=0, epsrel=1e-13)[0]
    else:
        i13 = math.pi / math.sqrt(3) - quad(lambda t: kv(1 / 3, t), 0, x, limit=500,
                                            epsabs=0, epsrel=1e-13)[0]
    return x * (2 * kv(2 / 3, x) - i13)


def scipy_G(delta, chi):
    """Eq. (24) bracket evaluated with scipy's K (independent of the oracle)."""
    z = 2 / 3 * delta / (chi * (1 - delta))
    f2 = z * kv(2 / 3, z)
    f1 = scipy_F1(z)
    return math.sqrt(3) / (2 * math.pi) * chi * (1 - delta) / delta * (f1 + 1.5 * delta * chi * z * f2)


@pytest.mark.parametrize("delta,chi", [(1e-3, 1.0), (0.3, 1.0), (0.9, 10.0), (0.01, 0.1)])
def test_G_against_scipy(delta, chi):
    assert abs(o.G(delta, chi) / scipy_G(delta, chi) - 1) < 1e-9


@pytest.mark.parametrize("chi", [1e-4, 1e-3])
def test_classical_power_limit(chi):
    # energy radiated per unit time / (alpha) = int delta G d delta -> (2/3) chi^2 (1 - 5.95 chi)
    e = log_quad(lambda d: d * o.G(d, chi), 1e-16 * chi, 0.5) + quad(lambda d: d * o.G(d, chi), 0.5, 1)[0]
    ratio = e / (2 / 3 * chi ** 2)
    # known expansion of the quantum correction: 1 - (55 sqrt3/16) chi + 48 chi^2 + O(chi^3)
    corr = 1 - 55 * math.sqrt(3) / 16 * chi + 48 * chi ** 2
    assert abs(ratio - corr) < 600 * chi ** 3 + 1e-9


def test_quantum_power_limit():
    chi = 1e4
    f = lambda d: d * o.G(d, chi)
    e = log_quad(f, 1e-20, 0.5) + quad(f, 0.5, 1 - 1e-12, limit=400, points=[0.9, 0.99, 0.999, 0.9999])[0]
    assert abs(e / (0.37 * chi ** (2 / 3)) - 1) < 0.01


def test_small_delta_asymptote():
    c = math.sqrt(3) / (2 * math.pi) * 2 ** (2 / 3) * Gamma(2 / 3) * (2 / 3) ** (1 / 3)
    assert abs(c - 0.52) < 0.003                       # the paper's 0.52
    for chi in (0.1, 1.0, 30.0):
        d = 1e-24
        val = o.P(d, chi, 100.0, 2.0) * 100.0 / (ALPHA * 2.0)
        assert abs(val / (c * chi ** (2 / 3) * d ** (-2 / 3)) - 1) < 1e-6


def test_Pm_finite_at_zero_and_consistent():
    chi, gam, h = 1.0, 1000.0, 50.0
    c = math.sqrt(3) / (2 * math.pi) * 2 ** (2 / 3) * Gamma(2 / 3) * (2 / 3) ** (1 / 3)
    lim = 3 * c * chi ** (2 / 3) * ALPHA * h / gam
    assert abs(o.Pm(1e-15, chi, gam, h) / lim - 1) < 1e-6
    for r in (0.1, 0.5, 0.9):
        assert o.Pm(r, chi, gam, h) == pytest.approx(3 * r * r * o.P(r ** 3, chi, gam, h), rel=1e-15)
    assert o.Pm(1.0, chi, gam, h) == 0.0


def test_number_rate_chi1():
    # int_0^1 G(delta, 1) d delta = int_0^1 3 r^2 G(r^3, 1) dr (the modified generator's
    # substitution makes the integrand smooth); compared with the same integral of
    # the scipy-K density
    n = quad(lambda r: 3 * r * r * o.G(r ** 3, 1.0), 0, 1, limit=400, epsrel=1e-12)[0]
    ref = quad(lambda r: 3 * r * r * scipy_G(r ** 3, 1.0), 1e-12, 0.999999, limit=200, epsrel=1e-10)[0]
    assert abs(n - ref) < 1e-6
    assert abs(n - 1.0339139) < 1e-6


@pytest.mark.parametrize("chi,bound", [(0.1, 1.5 * 0.1 ** (2 / 3)), (1.0, 1.5), (100.0, 50.0)])
def test_max_Pm_matches_paper_bounds(chi, bound):
    r = np.linspace(1e-4, 0.9999, 2000)
    m = max(o.G(x ** 3, chi) * 3 * x * x for x in r)
    assert abs(m / bound - 1) < 0.05


def test_pair_symmetry_and_positivity():
    for chig in (0.3, 1.0, 10.0):
        for de in (0.05, 0.2, 0.4):
            a, b = o.Pp(de, chig, 50.0, 3.0), o.Pp(1 - de, chig, 50.0, 3.0)
            assert a > 0 and abs(a / b - 1) < 1e-12


@pytest.mark.parametrize("chig,eps", [(0.05, 1.0), (0.02, 1.0), (0.05, 37.0)])
def test_pair_rate_erber_limit(chig, eps):
    # total Breit-Wheeler rate * eps / alpha -> (3/16) sqrt(3/2) chi exp(-8/(3 chi)):
    # at fixed chi_gamma the rate falls as 1/eps (Eq. (30)'s chi_g / eps_g)
    tot = quad(lambda d: o.Pp(d, chig, eps, 1.0) * eps / ALPHA, 0, 1, points=[0.5], limit=200, epsrel=1e-10)[0]
    er = 3 / 16 * math.sqrt(1.5) * chig * math.exp(-8 / (3 * chig))
    assert abs(tot / er - 1) < 0.2 * chig


def test_pair_rate_known_values():
    # int eps_g P_p / (alpha dt) at chi_g = 1 and 10, evaluated with scipy's K
    def sp(de, cg):
        z = 2 / 3 / (cg * de * (1 - de))
        f1 = scipy_F1(z)
        f2 = z * kv(2 / 3, z)
        return math.sqrt(3) / (2 * math.pi) * cg * (de - 1) * de * (f1 - 1.5 * cg * z * f2)
    for cg in (1.0, 10.0):
        for de in (0.1, 0.5):
            assert o.Pp(de, cg, 1.0, 1.0) / ALPHA == pytest.approx(sp(de, cg), rel=1e-9)


def test_time_step_bounds():
    # Eq. (28): dt_q = kappa*137*min(0.67 gamma^(1/3) H^(-2/3), 2/H); Eq. (33): kappa*130*2pi/H
    assert o.dtq_lepton(1000.0, 1e-3, 1.0) == pytest.approx(137 * min(0.67 * 10 * 100, 2000), rel=1e-14)
    assert o.dtq_lepton(1.0, 10.0, 0.1) == pytest.approx(0.1 * 137 * min(0.67 * 10 ** (-2 / 3), 0.2), rel=1e-14)
    assert o.dtq_photon(0.5, 0.1) == pytest.approx(0.1 * 130 * 2 * math.pi / 0.5, rel=1e-14)
    assert math.isinf(o.dtq_lepton(10.0, 0.0, 0.1))
    # the bound keeps alpha dt_q * max_r P_m-density below ~kappa (the paper's P_m << 1)
    for gam, H in ((1000.0, 1e-3), (1e4, 1e-2), (100.0, 0.5)):
        chi = gam * H
        dtq = o.dtq_lepton(gam, H, 1.0)
        worst = max(1.5 * chi ** (2 / 3), 0.5 * chi) * ALPHA * dtq / gam
        assert 0.5 < worst < 1.1
    assert o.nsub(10.0, 3.0, 100) == (4, False)
    assert o.nsub(10.0, 20.0, 100) == (1, False)
    assert o.nsub(1e6, 1.0, 100) == (100, True)
    assert o.nsub(5.0, math.inf, 100) == (1, False)


def test_chi_definitions():
    # electron along x, B along z: chi = gamma*|v x B| ... exact: sqrt((p x B)^2) = |p| B
    p, E, B = (999.9995, 0, 0), (0, 0, 0), (0, 0, 1e-3)
    assert o.chi(p, E, B) == pytest.approx(999.9995e-3, rel=1e-14)
    g = math.sqrt(1 + 999.9995 ** 2)
    assert o.heff(p, E, B) == pytest.approx(999.9995 / g * 1e-3, rel=1e-14)
    # crossed field co-propagating with the particle: chi = gamma (1 - beta) E
    p, E, B = (0, 0, 1e3), (1e-3, 0, 0), (0, 1e-3, 0)
    g = math.sqrt(1 + 1e6)
    assert o.chi(p, E, B) == pytest.approx((g - 1e3) * 1e-3, rel=1e-9)
    # head-on: chi = (gamma + p) E
    p = (0, 0, -1e3)
    assert o.chi(p, E, B) == pytest.approx((g + 1e3) * 1e-3, rel=1e-12)
    # photon: chi_gamma = eps * H_eff(k_hat); along E x B direction it vanishes
    assert o.chi_photon((0, 0, 5.0), E, B) == pytest.approx(0.0, abs=1e-18)
    assert o.chi_photon((0, 0, -5.0), E, B) == pytest.approx(5.0 * 2e-3, rel=1e-14)
    # invariance: chi is a Lorentz scalar; pure E field, p perpendicular: chi = gamma E
    assert o.chi((3.0, 0, 0), (0, 0.01, 0), (0, 0, 0)) == pytest.approx(math.sqrt(10) * 0.01, rel=1e-14)


def test_longitudinal_field_terms():
    # the (p_hat . E)^2 term of Eq. (3) and the (k_hat . E)^2 term of Eq. (32),
    # with a field component along the motion.  Lepton: chi = gamma H_eff
    # (Sec. IV.C) holds up to relative terms of order 1/gamma^2 against the
    # invariant form of Eq. (4); without the term H_eff is ~40% too large here
    p, E, B = (1000.0, 0.0, 0.0), (1e-3, 2e-3, 0.0), (0.0, 0.0, 1e-3)
    g = math.sqrt(1 + 1e6)
    assert abs(o.chi(p, E, B) / (g * o.heff(p, E, B)) - 1) < 1e-5
    # photon: chi_gamma is the massless limit of Eq. (4) with p = k
    for k in ((1e6, 0.0, 0.0), (3e5, -4e5, 1e5)):
        E, B = (2e-3, -1e-3, 5e-4), (1e-3, 3e-3, -2e-3)
        assert abs(o.chi_photon(k, E, B) / o.chi(k, E, B) - 1) < 1e-9
