"""Pins of the oracle's synchrotron functions F1, F2 (Sec. IV.E, Eq. (20)-(21)).

They are pinned against independent library routines (scipy.special.kv with
adaptive quadrature), closed forms (small-argument limits from the series of
K_nu, the Mellin integral of F1) and the constants the paper prints in
Sec. IV.H (F1(x<<1) ~ 2.15 x^(1/3), max F2 ~ 0.6).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import gamma as Gamma
from scipy.special import kv

from oracle import oracle as o


def scipy_F1(x):
    # int_x^inf K_{5/3} = 2 K_{2/3}(x) - int_x^inf K_{1/3}, from K_{nu-1} + K_{nu+1} = -2 K'_nu
    if x > 1.0:
        i13 = quad(lambda t: kv(1 / 3, t), x, np.inf, limit=500, epsabs=0, epsrel=1e-13)[0]
    else:
        i13 = math.pi / math.sqrt(3) - quad(lambda t: kv(1 / 3, t), 0, x, limit=500,
                                            epsabs=0, epsrel=1e-13)[0]
    return x * (2 * kv(2 / 3, x) - i13)


@pytest.mark.parametrize("x", [1e-9, 1e-4, 0.01, 0.1, 0.29, 1.0, 3.0, 10.0, 40.0, 150.0])
def test_F_against_scipy(x):
    assert abs(o.F2(x) / (x * kv(2 / 3, x)) - 1) < 2e-13
    assert abs(o.F1(x) / scipy_F1(x) - 1) < 1e-11


def test_F1_known_value():
    # F1(1) from two independent scipy evaluations (kv + quad) agree to 1e-13
    assert abs(o.F1(1.0) - 0.6514228153553) < 2e-13


def test_small_argument_limits():
    # K_nu(x) ~ Gamma(nu)/2 (2/x)^nu  =>  F1 ~ 2^{2/3} Gamma(2/3) x^{1/3}, F2 ~ 2^{-1/3} Gamma(2/3) x^{1/3}
    c1 = 2 ** (2 / 3) * Gamma(2 / 3)
    c2 = 2 ** (-1 / 3) * Gamma(2 / 3)
    x = 1e-24
    assert abs(o.F1(x) / x ** (1 / 3) - c1) < 1e-7
    assert abs(o.F2(x) / x ** (1 / 3) - c2) < 1e-7
    # the paper's printed constant (Sec. IV.H): F1(x << 1) ~ 2.15 x^{1/3}
    assert abs(o.F1(1e-12) / 1e-4 - 2.15) < 0.01


def test_max_F2():
    xs = np.linspace(0.05, 1.5, 600)
    vals = np.array([o.F2(x) for x in xs])
    i = int(vals.argmax())
    assert abs(vals[i] - 0.6070472) < 2e-6          # scipy: 0.607047226
    assert abs(vals[i] - 0.6) < 0.01                  # the paper's "max F2 ~ 0.6"


def test_integral_of_F1():
    # Mellin transform: int_0^inf F1(x) dx = 8 pi / (9 sqrt 3)
    val = quad(o.F1, 0, 1, limit=200)[0] + quad(o.F1, 1, 50, limit=200)[0]
    assert abs(val - 8 * math.pi / (9 * math.sqrt(3))) < 1e-9


def test_large_argument_decay():
    # F2(x) = x K_{2/3}(x) ~ sqrt(pi x / 2) e^{-x} (1 + 7/(72 x) + ...)
    x = 300.0
    asym = math.sqrt(math.pi * x / 2) * math.exp(-x) * (1 + (4 * (2 / 3) ** 2 - 1) / (8 * x))
    assert abs(o.F2(x) / asym - 1) < 1e-5
    assert o.F1(800.0) == 0.0 and o.F2(800.0) == 0.0
