"""The bounds behind the step kernels' early exits, checked against the
oracle's probabilities (no GPU).

After drawing (r1, r2) the kernels skip the probability evaluation when r2
is at least an upper bound of P over every r1, which leaves every decision
unchanged only if the bound really holds:
  emission (Eq. (25)): P_m(r1) <= alpha h sqrt3/(2 pi gamma) (5.6336
      chi^(2/3) + 1.8212 chi), before the kernels' 2% rounding margin;
  pairs (Eq. (30)):    P_p(de) <= alpha h sqrt3/(2 pi) (chi/eps) F2(z_min),
      z_min = 8/(3 chi), F2 at most 0.60705 (at 0.4169) and decreasing
      beyond, where F2(z) <= sqrt(pi z/2) e^(-z) (1 + 7/(72 z)) (the kernels
      evaluate this form, with a 2% rounding margin).
"""
import math

import numpy as np

from oracle import oracle as o

ALPHA = 7.2973525693e-3
K = math.sqrt(3) / (2 * math.pi)


def test_g1_decreases_from_its_limit():
    zs = np.logspace(-12, 2, 1500)
    g1 = np.array([o.F1(z) / z ** (1 / 3) for z in zs])
    assert np.all(np.diff(g1) <= 1e-15 * g1[:-1])
    assert abs(g1[0] - 2.14953) < 1e-5 and g1[0] * 3 * (2 / 3) ** (1 / 3) <= 5.6336


def test_emission_bound():
    r1s = np.concatenate([np.linspace(1e-6, 1 - 1e-9, 2001), 1 - np.logspace(-12, -1, 100),
                          np.logspace(-8, -1, 100)])
    worst = 0.0
    for chi in np.logspace(-5, 5, 41):
        for gamma, h in ((1.0, 1.0), (1e3, 30.0), (2e5, 1e3)):
            b = ALPHA * h * K / gamma * (5.6336 * chi ** (2 / 3) + 1.8212 * chi)
            worst = max(worst, max(o.Pm(r1, chi, gamma, h) for r1 in r1s) / b)
    assert worst <= 1.0 and worst > 0.98       # tight: the F1 term near r1 -> 0, the F2 term at large chi


def test_pair_bound():
    zs = np.linspace(0.0, 40.0, 4001)[1:]
    f2 = np.array([o.F2(z) for z in zs])
    assert f2.max() <= 0.60706 and abs(zs[f2.argmax()] - 0.4169) < 0.01
    beyond = zs > 0.4169
    assert np.all(np.diff(f2[beyond]) <= 0.0)
    bound_f2 = lambda z: math.sqrt(math.pi * z / 2) * math.exp(-z) * (1 + 7 / (72 * z))
    zz = np.concatenate([np.linspace(0.42, 5, 3000), np.logspace(math.log10(5), 2.5, 1000)])
    ratio = np.array([o.F2(z) / bound_f2(z) for z in zz])
    assert ratio.max() <= 1.0 and ratio.max() > 0.999       # tight at large z
    des = np.concatenate([np.linspace(1e-6, 1 - 1e-6, 1001), np.logspace(-9, -2, 50)])
    for chig in np.logspace(-2, 4, 31):
        eps, h = 100.0, 10.0
        zmin = 8.0 / (3.0 * chig)
        f = bound_f2(zmin) if zmin > 0.42 else 0.6071
        b = ALPHA * h * K * (chig / eps) * f
        assert max(o.Pp(de, chig, eps, h) for de in des) <= b * (1 + 1e-12)


def test_kernels_evaluate_the_verified_bounds():
    # the constants above are the ones the step kernels' early exits use:
    # read them from the kernel source, so that an edit there cannot leave
    # these checks verifying a different bound
    import re
    from pathlib import Path
    src = (Path(__file__).resolve().parent.parent / "paper_1412_6426_gb300" / "csrc" / "step_kernels.cuh").read_text()

    def body(name):
        m = re.search(r"__device__ __forceinline__ R " + name + r"\(.*?\n}\n", src, re.S)
        assert m, name
        return m.group(0)
    emit, pair = body("emit_bound"), body("pair_bound")
    assert "5.6336f * c23 + 1.8212f * c" in emit and "1.02 * kAlpha * kSqrt3Over2Pi" in emit
    assert "0.6666667f * __log2f(c)" in emit                       # chi^(2/3)
    assert "zmin = (8.0f / 3.0f) / c" in pair and "float f2 = 0.6071f;" in pair
    assert "if (zmin > 0.42f)" in pair and "(1.0f + float(7.0 / 72.0) / zmin)" in pair
    assert "sqrtf(float(kPi / 2) * zmin) * __expf(-zmin)" in pair
    assert "1.02 * kAlpha * kSqrt3Over2Pi" in pair and "(c / (float)eps) * f2" in pair
