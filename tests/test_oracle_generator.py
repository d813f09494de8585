"""Pin of the oracle's modified event generator (Sec. IV.G, Eq. (25)).

The paper's own check (Sec. IV.G, figure "generators"): for fixed gamma = 100
and chi = 1, running the generator many times reproduces the quantum
synchrotron spectrum Eq. (21) over the whole range, with no low-energy cutoff.
Here the expected count in each log-delta bin is ndraw * int_bin P(delta) d delta
with P computed from scipy's Bessel K (independent of the oracle), and the
sampled histogram must agree bin by bin within 4 sigma, down to delta = 1e-10.
"""
import math

import numpy as np
from scipy.integrate import quad
from scipy.special import kv

from oracle import oracle as o

ALPHA = 7.2973525693e-3


def scipy_P(delta, chi, gamma, h):
    z = 2 / 3 * delta / (chi * (1 - delta))
    if z > 700:
        return 0.0
    f2 = z * kv(2 / 3, z)
    if z > 1.0:
        i13 = quad(lambda t: kv(1 / 3, t), z, np.inf, limit=300)[0]
    else:
        i13 = math.pi / math.sqrt(3) - quad(lambda t: kv(1 / 3, t), 0, z, limit=300)[0]
    f1 = z * (2 * kv(2 / 3, z) - i13)
    G = math.sqrt(3) / (2 * math.pi) * chi * (1 - delta) / delta * (f1 + 1.5 * delta * chi * z * f2)
    return ALPHA * h * G / gamma


def test_frozen_spectrum_gamma100_chi1():
    gamma, chi = 100.0, 1.0
    h = 0.1 * gamma / (ALPHA * 1.6)        # max_r P_m ~ 0.1 (P_m << 1 regime, Sec. IV.H)
    ndraw = 400_000
    lo, hi, nb = -10.0, 0.0, 20
    acc, hist, viol = o.sample_frozen(chi, gamma, h, ndraw, 7, lo, hi, nb)
    assert viol == 0
    edges = np.linspace(lo, hi, nb + 1)
    expected = np.array([
        ndraw * quad(lambda u: scipy_P(10 ** u, chi, gamma, h) * 10 ** u * math.log(10),
                     edges[i], edges[i + 1], limit=200)[0]
        for i in range(nb)])
    sigma = np.sqrt(np.maximum(expected, 1.0))
    z = (hist - expected) / sigma
    assert np.all(np.abs(z) < 4.0), (z, hist, expected)
    # lowest bins are populated: no cutoff
    assert hist[0] > 10 and hist[1] > 10
    # the total number of events matches ndraw * int P
    tot = ndraw * quad(lambda r: 3 * r * r * scipy_P(r ** 3, chi, gamma, h), 1e-9, 1 - 1e-9, limit=200)[0]
    assert abs(acc - tot) < 4 * math.sqrt(tot)


def test_uniform_draws_are_uniform():
    # the (0,1) uniforms derived from Philox are uniform: chi-square over 64 bins, 2e5 draws
    raw = o.philox_block(12345, 3, 0, o.PURPOSE_EMIT, 1, 100_000)
    r = np.array([o.u52(int(a), int(b)) for a, b in raw[:, :2]] +
                 [o.u52(int(a), int(b)) for a, b in raw[:, 2:]])
    assert r.min() > 0 and r.max() < 1
    c, _ = np.histogram(r, bins=64, range=(0, 1))
    e = len(r) / 64
    chi2 = ((c - e) ** 2 / e).sum()
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)
    # successive draws uncorrelated
    assert abs(np.corrcoef(r[:-1], r[1:])[0, 1]) < 0.01


def test_u52_range_edges():
    assert o.u52(0, 0) == 0.5 / 2 ** 52
    assert o.u52(0xFFFFFFFF, 0xFFFFFFFF) == 1 - 0.5 / 2 ** 52


def test_philox_counter_and_key_sensitivity():
    a = o.philox([0, 0, 0, 0], [0, 0])
    b = o.philox([1, 0, 0, 0], [0, 0])
    c = o.philox([0, 0, 0, 0], [1, 0])
    assert a != b and a != c and b != c
    # distinct ids give distinct child ids; same inputs give the same id
    ids = {o.child_id(p, 5, s, k, 1) for p in range(50) for s in range(4) for k in range(3)}
    assert len(ids) == 600
    assert o.child_id(9, 1, 2, 2, 1) == o.child_id(9, 1, 2, 2, 1)
