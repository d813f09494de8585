"""The photon spectrum of the first workload against its exact expectation
along the realised trajectories (no GPU).

For every lepton sub-interval the oracle adds, per spectrum bin, the
probability int_bin P(delta) d delta of emitting a photon with delta in that
bin (Eq. (24); with P_m <= 1 the modified generator of Sec. IV.G emits with
exactly this probability), and p (1 - p) to its variance.  Whatever the
trajectories, the sampled histogram minus this sum is a martingale: in every
bin it must lie within 4 standard deviations.  The check reaches down to
delta = 1e-9: no low-energy cutoff.
"""
import numpy as np

from oracle import drive
from paper_1412_6426_gb300 import workloads


def test_sampled_spectrum_matches_its_expectation_along_the_trajectories():
    w = workloads.test_particles_static_b(n_particles=60, nsteps=80, seed=7)
    nbins = 9
    out, d, spec, _ = drive.run(w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt, w.nsteps, w.particles,
                                kappa=w.kappa, seed=w.seed, caps=(1000, 1000, 20000, 1), nbins=nbins,
                                lg_lo=-9.0, lg_hi=0.0, pairs_on=0, expect=True)
    exp, var = d["expected"], d["expected_var"]
    assert d["pm_gt1"] == 0 and d["emissions"] > 2000
    assert d["emissions"] - 20 < spec.sum() <= d["emissions"]   # all but the few below 1e-9
    z = (spec - exp) / np.sqrt(var)
    assert np.all(np.abs(z) < 4.0), (spec, exp, z)
    assert abs(spec.sum() - exp.sum()) < 4.0 * np.sqrt(var.sum())
    # the soft bins are populated: no cutoff
    assert exp[0] > 1.0 and spec[:3].sum() > 0
