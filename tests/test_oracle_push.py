"""Pins of the oracle's Boris pusher (Appendix A) against closed forms.

Uniform B: |p| is conserved to rounding and every step rotates p by exactly
2 atan(q B h / (2 m gamma)).  Crossed fields E < B: the mean velocity is the
E x B drift E/B.  Uniform E: p grows by q E t exactly.
"""
import math

import numpy as np

from oracle import oracle as o


def test_uniform_B_rotation_exact():
    # the Boris rotation in a uniform B turns p by exactly 2 atan(q B h / (2 m gamma))
    # per step, gamma = sqrt(1 + p^2/m^2), and keeps |p|: an electron at gamma = 1000,
    # a proton and a doubly charged ion of four proton masses at gamma = 3
    B, n = 1e-3, 37
    m_p = 1836.15267343
    for q, m, gam0 in ((-1.0, 1.0, 1000.0), (1.0, m_p, 3.0), (2.0, 4.0 * m_p, 3.0)):
        p0 = m * math.sqrt(gam0 ** 2 - 1)
        p = np.array([p0, 0.0, 0.0])
        h = 2 * math.pi * m * gam0 / (abs(q) * B) / 100.0
        for _ in range(n):
            p = o.boris(p, (0, 0, 0), (0, 0, B), q, m, h)
        assert abs(np.linalg.norm(p) / p0 - 1) < 1e-14
        theta = 2 * math.atan(abs(q) * B * h / (2 * m * gam0))
        ang = math.atan2(p[1], p[0])
        # a negative charge in a +z field turns counter-clockwise, a positive one clockwise
        expect = math.remainder(-math.copysign(1.0, q) * n * theta, 2 * math.pi)
        assert abs(math.remainder(ang - expect, 2 * math.pi)) < 1e-11, (q, m)


def test_uniform_E_acceleration_exact():
    p = np.array([0.0, 2.0, 0.0])
    for _ in range(10):
        p = o.boris(p, (0.01, 0, 0), (0, 0, 0), 1.0, 1.0, 3.0)
    assert np.allclose(p, [0.3, 2.0, 0.0], rtol=0, atol=1e-15)


def test_ExB_drift():
    # E = 0.5 B (x,z), B along z: drift along E x B = -y... here E along x, B along z: E x B = -y
    E, B = 0.5e-2, 1e-2
    p = np.array([0.0, 0.0, 0.0])
    x = np.zeros(3)
    h = 0.5
    nsteps = 40000
    ys = np.empty(nsteps)
    xs = np.empty(nsteps)
    for i in range(nsteps):
        p = o.boris(p, (E, 0, 0), (0, 0, B), 1.0, 1.0, h)
        g = math.sqrt(1 + p @ p)
        x += p / g * h
        xs[i], ys[i] = x[0], x[1]
    t = h * np.arange(1, nsteps + 1)
    vy = np.polyfit(t, ys, 1)[0]     # least-squares slope averages out the gyration
    vx = np.polyfit(t, xs, 1)[0]
    assert abs(vy + E / B) < 2e-4
    assert abs(vx) < 2e-4
