"""Pins of the oracle's pairs from the vacuum (Sec. V.B).

* Unit conversion: the pair count of a uniform-field box matches
  N_cells * P_S within binomial errors, with P_S = R_S V_cell c dt evaluated
  in SI units from the paper's formula (lambda_C, c and E_S in SI), so the
  oracle's Compton-unit form is checked against an independent evaluation.
* Only |E| matters: a rotating E field of amplitude E0 makes exactly the
  pairs a uniform E0 does (the draws are keyed by cell and step).
* Pairs are at rest, co-located, with equal numbers of electrons and
  positrons; their positions are uniform inside the cells (KS test).
* Weak fields make none; P_S > 1 is counted per cell.
* On a mesh the cell's field is the CIC value at its centre (the paper takes
  the field constant over a cell): with E_y alternating E0, 0 along x every
  centre sees E0/2, so every cell draws at P_S(E0/2).
"""
import math

import numpy as np
from scipy.stats import kstest

from oracle import drive
from oracle import oracle as o

HBAR, M_E, C, Q_E = 1.054571817e-34, 9.1093837015e-31, 299792458.0, 1.602176634e-19
LAMBDA_C = HBAR / (M_E * C)
TAU_C = HBAR / (M_E * C * C)


def p_schwinger_si(E_over_ES, cell_m3, dt_s):
    r_s = (1.0 / (4 * math.pi ** 3 * LAMBDA_C ** 4)) * E_over_ES ** 2 * math.exp(-math.pi / E_over_ES)
    return r_s * cell_m3 * C * dt_s


def run_box(fp_mode, fp, n=24, d=60.0, dt=40.0, nsteps=1, t0=0.0):
    return drive.run((n, n, n), (d, d, d), (0.0, 0.0, 0.0), (1, 1, 1), fp_mode, fp, dt, nsteps, {},
                     kappa=0.1, seed=9, caps=(4 * n ** 3 * nsteps, 4 * n ** 3 * nsteps, 1, 1),
                     schwinger_on=1, t0=t0)


def test_pair_count_matches_the_si_rate():
    E0, n, d, dt = 0.25, 24, 60.0, 40.0
    out, D, _, _ = run_box(o.FIELD_UNIFORM, (0, E0, 0, 0, 0, 0), n=n, d=d, dt=dt)
    p = p_schwinger_si(E0, (d * LAMBDA_C) ** 3, dt * TAU_C)
    assert 0.005 < p < 0.5
    N = n ** 3
    k = D["schwinger_pairs"]
    assert abs(k - N * p) < 5 * math.sqrt(N * p * (1 - p)), (k, N * p)
    assert len(out[0][3]) == len(out[1][3]) == k
    assert D["schwinger_gt1"] == 0


def test_pairs_at_rest_colocated_uniform_in_cells():
    E0, n, d = 0.25, 24, 60.0
    out, D, _, _ = run_box(o.FIELD_UNIFORM, (0, E0, 0, 0, 0, 0), n=n, d=d)
    xe, pe, we, ie = out[0]
    xp, pp, wp, ip = out[1]
    assert np.all(pe == 0) and np.all(pp == 0) and np.all(we == 1.0)
    assert np.array_equal(xe, xp)
    assert len(np.unique(np.concatenate([ie, ip]))) == 2 * len(ie)
    frac = (xe / d) % 1.0
    for c in range(3):
        assert kstest(frac[:, c], "uniform").pvalue > 1e-3
    # the three offsets are independent draws
    cc = np.corrcoef(frac.T)
    assert np.all(np.abs(cc[np.triu_indices(3, 1)]) < 4 / math.sqrt(len(frac)))


def test_only_the_field_strength_matters():
    E0, w = 0.25, 3e-5
    a, Da, _, _ = run_box(o.FIELD_UNIFORM, (0, E0, 0, 0, 0, 0), nsteps=2)
    b, Db, _, _ = run_box(o.FIELD_ROTATING_E, (E0, w), nsteps=2)
    assert Da["schwinger_pairs"] == Db["schwinger_pairs"] > 100
    for sp in (0, 1):
        ia, ib = np.sort(a[sp][3]), np.sort(b[sp][3])
        assert np.array_equal(ia, ib)


def test_weak_field_none_strong_field_counted():
    _, D, _, _ = run_box(o.FIELD_UNIFORM, (0, 0.01, 0, 0, 0, 0))
    assert D["schwinger_pairs"] == 0
    _, D, _, _ = run_box(o.FIELD_UNIFORM, (0, 2.0, 0, 0, 0, 0), n=6)
    assert D["schwinger_gt1"] == 6 ** 3 and D["schwinger_pairs"] == 6 ** 3


def test_mesh_field_taken_at_the_cell_centre():
    # E_y nodes (i, j + 1/2, k) hold E0 for even i and 0 for odd i; the CIC
    # value at any cell centre is E0/2.  P_S(E0) > 1, so a field read at the
    # cell's corner would make exactly one pair in every even cell and none
    # in the odd ones
    E0, n, d, dt = 0.5, 16, 60.0, 40.0
    N = n ** 3
    ey = np.zeros((n, n, n))
    ey[:, :, 0::2] = E0                              # [k][j][i], x fastest
    fields = [np.zeros(N), ey.ravel().copy(), np.zeros(N), np.zeros(N), np.zeros(N), np.zeros(N)]
    J = [np.zeros(N) for _ in range(3)]
    out, D, _, _ = drive.run((n, n, n), (d, d, d), (0.0, 0.0, 0.0), (1, 1, 1), o.FIELD_GRID, (), dt, 1, {},
                             kappa=0.1, seed=9, caps=(N, N, 1, 1), schwinger_on=1, fields=fields, J=J)
    p = p_schwinger_si(E0 / 2, (d * LAMBDA_C) ** 3, dt * TAU_C)
    assert 0.005 < p < 0.5 and p_schwinger_si(E0, (d * LAMBDA_C) ** 3, dt * TAU_C) > 1.0
    k = D["schwinger_pairs"]
    assert abs(k - N * p) < 5 * math.sqrt(N * p * (1 - p)), (k, N * p)
    assert D["schwinger_gt1"] == 0
    # the pairs' cells, even and odd in x alike
    ix = np.floor(out[0][0][:, 0] / d).astype(int)
    even = int((ix % 2 == 0).sum())
    assert abs(even - (k - even)) < 5 * math.sqrt(k)
