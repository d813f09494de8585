"""Pins of the oracle's Boris pusher (Appendix A) against closed forms.

Uniform B: |p| is conserved to rounding and every step rotates p by exactly
2 atan(q B h / (2 m gamma)).  Crossed fields E < B: the mean velocity is the
E x B drift E/B.  Uniform E: p grows by q E t exactly.
"""
import math

import numpy as np

from oracle import oracle as o


def test_uniform_B_rotation_exact():
    B, gam0 = 1e-3, 1000.0
    p = np.array([math.sqrt(gam0 ** 2 - 1), 0.0, 0.0])
    h = 2 * math.pi * gam0 / B / 100.0
    n = 37
    for _ in range(n):
        p = o.boris(p, (0, 0, 0), (0, 0, B), -1.0, 1.0, h)
    assert abs(np.linalg.norm(p) / math.sqrt(gam0 ** 2 - 1) - 1) < 1e-14
    theta = 2 * math.atan(B * h / (2 * gam0))
    ang = math.atan2(p[1], p[0])
    # electron (q=-1) in +z field rotates counter-clockwise
    expect = math.remainder(n * theta, 2 * math.pi)
    assert abs(math.remainder(ang - expect, 2 * math.pi)) < 1e-11


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
