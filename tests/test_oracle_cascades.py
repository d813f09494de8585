"""The shower benchmark of Sec. VII.A on the oracle (no GPU): the adaptive
event generator at a step that needs no subdivision and at one it divides
into hundreds of sub-intervals develops the same cascade.

256 electrons with gamma0 = 2e5 in H0 = 0.2 E_S perpendicular to the motion
(one run of 256 independent cascades: the field is uniform and the particles
are test particles; each seed's products inherit its index in the top id
bits).  After t_rad/2 the mean number of particles above 1e-3 gamma0 per seed
must agree between dt = 5e-3 t_rad (100 steps) and dt = t_rad/2 (one step)
within 4 standard errors of the per-seed counts.
"""
import numpy as np

from paper_1412_6426_gb300 import workloads as wl
from tests.util import run_oracle

S, BITS = 256, 8


def per_seed_counts(out, cut):
    c = np.zeros(S)
    for sp in (wl.ELECTRON, wl.POSITRON, wl.PHOTON):
        x, p, w, ids = out[sp]
        if len(ids) == 0:
            continue
        eps = np.sqrt((0.0 if sp == wl.PHOTON else 1.0) + (p ** 2).sum(1))
        seed = (ids >> np.uint64(64 - BITS)).astype(np.int64)
        sel = eps > cut
        c += np.bincount(seed[sel], weights=w[sel], minlength=S)[:S]
    return c


def shower(dt_per_trad, nsteps, seed):
    w = wl.shower_cascade(n_seeds=S, dt_per_trad=dt_per_trad, seed=seed)
    x, p, wt, _ = w.particles[wl.ELECTRON]
    w.particles = {wl.ELECTRON: (x, p, wt, np.arange(S, dtype=np.uint64) << np.uint64(64 - BITS))}
    w.ens_bits = BITS
    out, d, _, _ = run_oracle(w, nsteps, caps=(100_000, 100_000, 2_000_000, 1), nsub_max=100_000)
    assert d["overflow"] == 0 and d["capped"] == 0
    return per_seed_counts(out, w.meta["eps_cut"]), d


def test_shower_small_and_large_step_agree():
    small, ds = shower(5e-3, 100, 21)
    large, dl = shower(0.5, 1, 22)
    # the one large step: hundreds of sub-intervals for each seed (more for its products)
    assert dl["substeps_lepton"] > 100 * S
    ms, ml = small.mean(), large.mean()
    err = np.hypot(small.std(ddof=1), large.std(ddof=1)) / np.sqrt(S)
    assert ms > 3.0 and ml > 3.0
    assert abs(ms - ml) < 4 * err, (ms, ml, err)
