"""Pins of the oracle's ensembles, generator factors and thinning (Sec. VI).

* Ensembles: with one ensemble the table field reproduces the uniform and
  rotating single-field modes bit for bit; ensembles run together give
  exactly what each gives when run alone (no cross-talk, products stay in
  their parent's ensemble); with the emission off, an electron in a rotating
  E field frozen over each step follows the closed-form geometric sum
  p_N = p_0 - q E0 dt sum_n exp(i (omega t_n + phase)).
* Generator factors f_g and N_g (Sec. VI): the parents' histories do not
  depend on them (bit for bit); products carry w f_g / N_g; the weighted
  photon yield and emitted energy agree with f_g = N_g = 1 within the
  statistical error; kept products follow Binomial(events, 1/f_g).
* Thinning with global even redistribution (Sec. VI): each group keeps its
  total weight; groups at or below the limit are untouched; the survivors
  of a group of N are Binomial(N, L/N); a shower thinned on the way has the
  same weighted yields as the unthinned one (the paper's own check,
  Sec. VII.C).
"""
import math

import numpy as np

from oracle import drive
from oracle import oracle as o

GAMMA0 = 1000.0


def box():
    return dict(n=(4, 4, 4), d=(1e9, 1e9, 1e9), x0=(-2e9, -2e9, -2e9), periodic=(1, 1, 1))


def beam(n, gamma=GAMMA0, direction=(1.0, 0.0, 0.0), ens=0, bits=0, first_id=0):
    p = math.sqrt(gamma ** 2 - 1)
    ids = np.arange(first_id, first_id + n, dtype=np.uint64)
    if bits:
        ids |= np.uint64(ens) << np.uint64(64 - bits)
    return (np.zeros((n, 3)), np.tile(np.array(direction) * p, (n, 1)), np.ones(n), ids)


def run(parts, fp_mode, fp, dt, nsteps, caps=(40000, 40000, 200000, 1), **kw):
    b = box()
    return drive.run(b["n"], b["d"], b["x0"], b["periodic"], fp_mode, fp, dt, nsteps, parts,
                     kappa=0.1, seed=3, caps=caps, **kw)


def same(out_a, out_b, species=range(4)):
    for sp in species:
        xa, pa, wa, ia = out_a[sp]
        xb, pb, wb, ib = out_b[sp]
        oa, ob = np.argsort(ia), np.argsort(ib)
        assert np.array_equal(ia[oa], ib[ob]), sp
        assert np.array_equal(pa[oa], pb[ob]) and np.array_equal(xa[oa], xb[ob])
        assert np.array_equal(wa[oa], wb[ob])


def ens_row(E0=0.0, omega=0.0, phase=0.0, Eu=(0.0, 0.0, 0.0), Bu=(0.0, 0.0, 0.0), thin_scale=0.0):
    return [E0, omega, phase, *Eu, *Bu, thin_scale]


# ---- ensembles -----------------------------------------------------------

def test_one_ensemble_is_the_uniform_mode():
    # a B along z alone, and a general field with six different components
    parts = {0: beam(200)}
    for Eu, Bu in (((0, 0, 0), (0, 0, 1e-3)), ((2e-4, -1e-4, 3e-4), (4e-4, -6e-4, 1e-3))):
        a = run(parts, o.FIELD_UNIFORM, (*Eu, *Bu), 2e4, 4)[0]
        b = run(parts, o.FIELD_ENSEMBLE, (), 2e4, 4, ens=np.array([ens_row(Eu=Eu, Bu=Bu)]))[0]
        assert sum(len(a[s][3]) for s in range(4)) > 200
        same(a, b)


def test_one_ensemble_is_the_rotating_mode():
    parts = {0: beam(200, gamma=300.0, direction=(0, 1, 0))}
    E0, w = 2e-3, 3e-5
    a = run(parts, o.FIELD_ROTATING_E, (E0, w), 3e3, 5)[0]
    b = run(parts, o.FIELD_ENSEMBLE, (), 3e3, 5, ens=np.array([ens_row(E0=E0, omega=w)]))[0]
    same(a, b)


def test_an_ensemble_without_a_row_sees_no_field():
    # a table of one row handed over in a buffer whose next, uncounted row
    # holds a strong field: ensemble 0 sees its row, ensemble 1 has no row
    # and sees nothing (its field is never read from beyond the table)
    rows = np.array([ens_row(Eu=(1e-3, 0, 0), Bu=(0, 2e-3, 0)), ens_row(Eu=(5.0, 5.0, 5.0), Bu=(5.0, 5.0, 5.0))])
    P = o.make_params(field_mode=o.FIELD_ENSEMBLE, ens_bits=1, ens=rows, **box())
    P.n_ens = 1
    E, B = o.field_ensemble(P, 7, 0.0)
    assert np.array_equal(E, [1e-3, 0, 0]) and np.array_equal(B, [0, 2e-3, 0])
    E, B = o.field_ensemble(P, (1 << 63) | 7, 0.0)
    assert np.all(E == 0.0) and np.all(B == 0.0)


def test_ensembles_together_equal_ensembles_alone():
    bits = 8
    table = np.array([ens_row(Bu=(0, 0, 1e-3)),
                      ens_row(E0=3e-3, omega=2e-5, phase=0.7),
                      ens_row(E0=1e-3, omega=5e-5, Eu=(0, 0, 5e-4), Bu=(2e-4, 0, 0))])
    seeds = [beam(60 + 40 * e, gamma=800.0 + 300 * e, direction=(0, 1, 0), ens=e, bits=bits) for e in range(3)]
    together = {0: tuple(np.concatenate([s[k] for s in seeds]) for k in range(4))}
    kw = dict(ens_bits=bits, ens=table, thin_interval=2, thin_limit=(120, 120, 150, 0))
    a, da, _, _ = run(together, o.FIELD_ENSEMBLE, (), 1e4, 6, **kw)
    assert da["emissions"] > 100 and da["thinned"] > 0
    hi = np.uint64(64 - bits)
    for e in range(3):
        b, _, _, _ = run({0: seeds[e]}, o.FIELD_ENSEMBLE, (), 1e4, 6, **kw)
        sub = {sp: tuple(v[(a[sp][3] >> hi) == e] for v in a[sp]) for sp in range(4)}
        same(sub, b)
    # every product stayed in one of the seeded ensembles
    for sp in range(4):
        assert np.all((a[sp][3] >> hi) < 3)


def test_rotating_field_closed_form_orbit():
    # emission off: p_{n+1} = p_n - E(t_n) dt for charge -1 with B = 0 and the
    # field frozen at the step start, so p_N = p_0 - E0 dt sum_n e^{i(w t_n + phase)}
    E0, w, phase, dt, N = 4e-3, 2e-5, 0.3, 1.5e4, 40
    a0 = E0 / w
    parts = {0: (np.zeros((3, 3)), np.tile([0.0, a0, 0.0], (3, 1)), np.ones(3), np.arange(3, dtype=np.uint64))}
    out = run(parts, o.FIELD_ENSEMBLE, (), dt, N, emission_on=0, pairs_on=0,
              ens=np.array([ens_row(E0=E0, omega=w, phase=phase)]))[0]
    z = np.exp(1j * (w * dt * np.arange(N) + phase)).sum()
    expect = np.array([0.0 - E0 * dt * z.real, a0 - E0 * dt * z.imag, 0.0])
    assert np.allclose(out[0][1], expect, rtol=0, atol=1e-12 * a0)


# ---- generator factors ---------------------------------------------------

def shower(**kw):
    # chi = 1 electrons in a uniform B, pairs on; a few steps
    parts = {0: beam(400)}
    return run(parts, o.FIELD_UNIFORM, (0, 0, 0, 0, 0, 1e-3), 3e4, 4, nbins=0, **kw)


def test_parents_do_not_depend_on_factors():
    base, d0, _, _ = shower()
    seeds = np.arange(400, dtype=np.uint64)
    for kw in (dict(emit_fg=4.0), dict(emit_ng=3), dict(emit_fg=2.5, emit_ng=2, pair_fg=3.0, pair_ng=2)):
        out, d, _, _ = shower(**kw)
        assert d["emissions"] == d0["emissions"] and d["pairs"] == d0["pairs"]
        ia, ib = base[0][3], out[0][3]
        ka, kb = np.isin(ia, seeds), np.isin(ib, seeds)
        oa, ob = np.argsort(ia[ka]), np.argsort(ib[kb])
        assert np.array_equal(base[0][1][ka][oa], out[0][1][kb][ob])


def test_trivial_factors_are_the_plain_generator():
    a = shower()[0]
    b = shower(emit_fg=1.0, emit_ng=1, pair_fg=0.0, pair_ng=0)[0]
    same(a, b)


def _photon_yield(out):
    x, p, w, _ = out[2]
    return w.sum(), (w * np.linalg.norm(p, axis=1)).sum()


def test_emission_factor_fg_keeps_yields():
    ref, d0, _, _ = shower(pairs_on=0)
    n0, e0 = _photon_yield(ref)
    fg = 4.0
    out, d, _, _ = shower(pairs_on=0, emit_fg=fg)
    n1, e1 = _photon_yield(out)
    x, p, w, _ = out[2]
    assert np.all(w == fg)
    # kept products: Binomial(created without the factor, 1/fg)
    m = d0["photons_created"]
    k = d["photons_created"]
    assert abs(k - m / fg) < 5 * math.sqrt(m * (1 / fg) * (1 - 1 / fg))
    # weighted yield and emitted energy: same expectation (errors of the thinned sample)
    assert abs(n1 - n0) < 5 * fg * math.sqrt(k)
    assert abs(e1 - e0) < 5 * math.sqrt(fg * (w * np.linalg.norm(p, axis=1) ** 2).sum())


def test_emission_factor_ng_keeps_yields():
    ref, d0, _, _ = shower(pairs_on=0)
    n0, e0 = _photon_yield(ref)
    ng = 4
    out, d, _, _ = shower(pairs_on=0, emit_ng=ng)
    n1, e1 = _photon_yield(out)
    x, p, w, _ = out[2]
    assert np.all(w == 1.0 / ng)
    assert d["photons_created"] > 3 * d0["photons_created"]
    assert abs(n1 - n0) < 5 * math.sqrt(d0["photons_created"])
    eps0 = np.linalg.norm(ref[2][1], axis=1)
    assert abs(e1 - e0) < 5 * math.sqrt((eps0 ** 2).sum())


def test_pair_factor_keeps_lepton_yield():
    # high chi: many pairs; compare weighted positron numbers
    parts = {0: beam(300, gamma=4000.0)}
    kw = dict(emission_on=1)
    ref, d0, _, _ = run(parts, o.FIELD_UNIFORM, (0, 0, 0, 0, 0, 5e-3), 1e5, 6, **kw)
    out, d, _, _ = run(parts, o.FIELD_UNIFORM, (0, 0, 0, 0, 0, 5e-3), 1e5, 6, pair_fg=3.0, **kw)
    assert d0["pairs"] > 100
    w0, w1 = ref[1][2].sum(), out[1][2].sum()
    assert np.all(np.isin(out[1][2], [3.0, 9.0, 27.0]))
    assert abs(w1 - w0) < 5 * 3.0 * math.sqrt(max(d["pairs_created"], 1)) + 5 * math.sqrt(w0)
    # N_g = 3 samples per photon sub-interval, each pair of weight w / 3
    out, d, _, _ = run(parts, o.FIELD_UNIFORM, (0, 0, 0, 0, 0, 5e-3), 1e5, 6, pair_ng=3, **kw)
    w3 = out[1][2]
    assert d["pairs_created"] > 2 * d0["pairs"]
    assert np.allclose(w3 * 3 ** np.round(-np.log(w3) / np.log(3)), 1.0, rtol=1e-12)   # powers of 1/3
    assert abs(w3.sum() - w0) < 5 * math.sqrt(max(d["pairs_created"], 1)) / 3 + 5 * math.sqrt(w0)


# ---- thinning -------------------------------------------------------------

def _thin_once(parts, limit, bits=0, table=None, step=7):
    P = o.make_params(field_mode=o.FIELD_ENSEMBLE if table is not None else o.FIELD_UNIFORM,
                      ens_bits=bits, ens=table, thin_limit=limit, seed=5, **box())
    r = o.Run(P, caps=(5000, 5000, 5000, 5000))
    for sp, v in parts.items():
        r.sp[sp].set(*v)
    before = {sp: r.sp[sp].get() for sp in range(4)}
    r.thin(step)
    after = {sp: r.sp[sp].get() for sp in range(4)}
    return before, after, r.diag()


def test_thinning_conserves_group_weight_and_is_binomial():
    rng = np.random.default_rng(0)
    bits = 4
    sizes = [50, 400, 1200, 3000]
    ids = np.concatenate([np.arange(n, dtype=np.uint64) | (np.uint64(e) << np.uint64(64 - bits))
                          for e, n in enumerate(sizes)])
    n = len(ids)
    w = rng.uniform(0.5, 2.0, n)
    x = rng.normal(size=(n, 3))
    p = rng.normal(size=(n, 3)) * 100
    table = np.zeros((4, o.ENS_STRIDE))
    L = 300
    table[3, 9] = 2.5          # the largest ensemble keeps floor(2.5 L)
    before, after, d = _thin_once({2: (x, p, w, ids)}, (0, 0, L, 0), bits, table)
    xb, pb, wb, ib = before[2]
    xa, pa, wa, ia = after[2]
    assert d["thinned"] == len(ib) - len(ia)
    for e, N in enumerate(sizes):
        gb = (ib >> np.uint64(64 - bits)) == e
        ga = (ia >> np.uint64(64 - bits)) == e
        assert math.isclose(wb[gb].sum(), wa[ga].sum(), rel_tol=1e-12)
        Lg = int(2.5 * L) if e == 3 else L
        if N <= Lg:
            assert np.array_equal(ib[gb], ia[ga]) and np.array_equal(wb[gb], wa[ga])
        else:
            q = Lg / N
            assert abs(ga.sum() - Lg) < 5 * math.sqrt(N * q * (1 - q))
            # survivors: a subsequence of the group, positions and momenta untouched
            keep = np.isin(ib, ia[ga])
            assert np.array_equal(ib[keep & gb], ia[ga])
            assert np.array_equal(pb[keep & gb], pa[ga]) and np.array_equal(xb[keep & gb], xa[ga])
            # even redistribution: one common factor
            ratio = wa[ga] / wb[keep & gb]
            assert np.allclose(ratio, ratio[0], rtol=1e-14)


def test_thinning_without_ensembles_is_one_group_per_species():
    rng = np.random.default_rng(1)
    n = 2000
    parts = {sp: (rng.normal(size=(n, 3)), rng.normal(size=(n, 3)), rng.uniform(1, 2, n),
                  np.arange(n, dtype=np.uint64) + 10000 * sp) for sp in range(4)}
    before, after, d = _thin_once(parts, (500, 0, 100, 2000))
    for sp, L in enumerate((500, 0, 100, 2000)):
        nb, na = len(before[sp][3]), len(after[sp][3])
        assert math.isclose(before[sp][2].sum(), after[sp][2].sum(), rel_tol=1e-12)
        if L == 0 or L >= n:
            assert na == nb
        else:
            assert abs(na - L) < 5 * math.sqrt(L)


def test_lineage_bits_outside_ensembles_keep_one_group():
    """Outside the ensemble field mode the top id bits only record a seed's
    lineage: thinning still treats each species as one group, so the result
    equals the run without the bits (same survivors, same weight factor)."""
    rng = np.random.default_rng(2)
    n = 2000
    seeds = rng.integers(0, 16, n).astype(np.uint64)
    ids = (seeds << np.uint64(60)) | np.arange(n, dtype=np.uint64)
    parts = {0: (rng.normal(size=(n, 3)), rng.normal(size=(n, 3)), rng.uniform(1, 2, n), ids)}
    _, plain, _ = _thin_once(parts, (500, 0, 0, 0))
    _, tagged, d = _thin_once(parts, (500, 0, 0, 0), bits=4)
    assert d["thinned"] > 0
    assert np.array_equal(plain[0][3], tagged[0][3]) and np.array_equal(plain[0][2], tagged[0][2])
    assert abs(len(tagged[0][3]) - 500) < 5 * math.sqrt(500)


def test_thinned_shower_keeps_weighted_yields():
    # a chi = 1 shower, photons thinned to 300 every 2 steps vs not thinned:
    # the weighted photon number and energy agree within the thinning noise
    parts = {0: beam(300)}
    kw = dict(pairs_on=0)
    ref, d0, _, _ = run(parts, o.FIELD_UNIFORM, (0, 0, 0, 0, 0, 1e-3), 3e4, 6, **kw)
    out, d, _, _ = run(parts, o.FIELD_UNIFORM, (0, 0, 0, 0, 0, 1e-3), 3e4, 6,
                       thin_interval=2, thin_limit=(0, 0, 300, 0), **kw)
    assert d["thinned"] > 0 and len(out[2][3]) < len(ref[2][3])
    n0, e0 = _photon_yield(ref)
    n1, e1 = _photon_yield(out)
    # electrons are never thinned here, and their histories are the same
    same({0: ref[0]}, {0: out[0]}, species=(0,))
    assert abs(n1 - n0) < 0.05 * n0
    x, p, w, _ = out[2]
    assert abs(e1 - e0) < 5 * math.sqrt((w * w * np.linalg.norm(p, axis=1) ** 2).sum()) + 5 * math.sqrt(
        (np.linalg.norm(ref[2][1], axis=1) ** 2).sum())


def test_spectra_are_weighted():
    # the spectra sum the photons' weights (Sec. VI's weighted products):
    # electrons of weights 0.5 .. 3, and a log range that holds every photon
    rng = np.random.default_rng(4)
    x, p, _, ids = beam(300)
    w = rng.uniform(0.5, 3.0, 300)
    out, d, spec, spec_e = run({0: (x, p, w, ids)}, o.FIELD_UNIFORM, (0, 0, 0, 0, 0, 1e-3), 2e4, 3,
                               pairs_on=0, nbins=16, lg_lo=-60.0, lg_hi=4.0)
    wph = out[2][2]
    assert len(wph) > 100 and not np.all(wph == wph[0])
    assert math.isclose(spec.sum(), wph.sum(), rel_tol=1e-12)
    assert math.isclose(spec_e.sum(), wph.sum(), rel_tol=1e-12)
