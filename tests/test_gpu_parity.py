"""Parity of the CUDA particle step with the FP64 oracle (GPU tests).

FP64 path: the same Philox streams drive both sides, so every particle must
exist on both sides (same ids: identical event histories, including every
product's birth step and sub-step) with momenta within 1e-12 relative and
positions within 1e-12 of the box size (the tolerance the FP64 form is held
to).  FP32 path: statistical agreement (event counts and spectrum bins within
3 sigma, pair yields within 3 sigma, momentum relative error <= 1e-5 between
events for every particle, and within 1e-5 plus the quantisation of the FP32
event draws in its ancestry for every particle with the same event history,
energy conservation 1e-4).
"""
import math

import numpy as np
import pytest

from paper_1412_6426_gb300 import workloads
from tests.util import box_scale, compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1412_6426_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()


def assert_parity(w, nsteps=None, rtol=1e-12, **opts):
    ora, od, _, _ = run_oracle(w, nsteps, **dict(opts))
    assert od["overflow"] == 0
    gpu, gd = run_gpu(w, nsteps, precision=64, **dict(opts))
    assert gd["status"] == 0, gd
    rep = compare(gpu, ora, rtol_p=rtol, xtol=1e-12 * box_scale(w))
    assert rep["ok"], rep
    for k in ("emissions", "pairs", "substeps_lepton", "substeps_photon", "capped", "pm_gt1"):
        assert gd[k] == od[k], (k, gd[k], od[k])
    return rep, gd, od


def test_fp64_static_b_parity():
    # chi = 1, gamma = 1000, dt = 0.01 gyro periods (first workload, 1000 of its electrons)
    w = workloads.test_particles_static_b(n_particles=1000, nsteps=20)
    rep, gd, od = assert_parity(w)
    assert gd["emissions"] > 5000 and rep["matched"] > 6000


def test_fp64_pairs_uniform_E():
    # chi ~ 6: photons convert to pairs within the run
    w = workloads.test_particles_static_b(n_particles=200, nsteps=4)
    w.field_mode, w.fp, w.dt = workloads.FIELD_UNIFORM, (0, 2e-3, 0, 0, 0, 0), 2e5
    x, p, wt, ids = w.particles[0]
    p = p / np.linalg.norm(p[0]) * math.sqrt(3000.0 ** 2 - 1)
    w.particles = {0: (x, p, wt, ids)}
    rep, gd, od = assert_parity(w)
    assert gd["pairs"] > 0 and gd["emissions"] > 100


@pytest.mark.parametrize("same_step", [0, 1])
def test_fp64_children_modes(same_step):
    w = workloads.test_particles_static_b(n_particles=100, nsteps=6)
    w.fp = (0, 0, 0, 0, 0, 3e-2)      # chi ~ 30: deep in-step cascades
    w.dt = 2e4
    # Leptons cooled to gamma ~ 3 gyrate ~1000 rad in these 6 steps at ~1.4 rad
    # per sub-interval: the FP64 push rounds like the oracle's, operation by
    # operation, so no rotation-angle difference accumulates.
    rep, gd, od = assert_parity(w, same_step_children=same_step, caps=(60000, 60000, 60000, 1))
    assert gd["pairs"] > 0


def test_fp64_gaussian_pulse_parity():
    # beam-laser collision (a0 = 200, 1 GeV), the pulse peak meets the beam centre at step 10
    w = workloads.beam_laser_collision(n_particles=400, nsteps=20, seed=3)
    rep, gd, od = assert_parity(w)
    assert gd["emissions"] > 100


def test_fp64_nsub_cap_and_absorbing_box():
    w = workloads.test_particles_static_b(n_particles=200, nsteps=5)
    w.periodic = (0, 0, 0)
    w.n = (8, 8, 1)                    # small open box around the origin: photons leave it
    w.x0 = (-4 * w.d[0], -4 * w.d[1], -0.5 * w.d[2])
    rep, gd, od = assert_parity(w, nsub_max=3, kappa=0.01)
    assert gd["capped"] > 0 and gd["absorbed"] == od["absorbed"] > 0


def fp32_momentum_bounds(gpu, ora, p_max, n_ev):
    """The FP32 path against the FP64 oracle, particle by particle, for every
    particle whose event history the FP32 run shares (same id).

    Between events the push keeps within 1e-5 relative (the FP32 path's
    bound; tested alone by test_fp32_push_between_events).  An event moves a
    momentum by a drawn fraction of its parent's: the parent keeps 1 - delta,
    the photon takes delta = r1^3, a pair splits r1 : 1 - r1.  The FP32 path
    takes r1 from the top 23 bits of the Philox word whose top 52 bits the
    FP64 oracle reads, so |r1_32 - r1_64| <= 2^-24 and every fraction differs
    by at most (r1 + 2^-24)^3 - r1^3 <= 7 2^-24 (r1 <= 1): an absolute error
    of at most 7 2^-24 p_max per event, which later fractions (all <= 1) do
    not enlarge.  A particle with at most n_ev events in its ancestry is
    therefore within 1e-5 |p| + n_ev 7 2^-24 p_max.  Returns (matched, the
    largest error over this bound)."""
    matched, worst = 0, 0.0
    for sp in (0, 1, 2):
        xg, pg, _, ig = gpu[sp]
        xo, po, _, io = ora[sp]
        _, a, b = np.intersect1d(ig, io, return_indices=True)
        matched += len(a)
        if len(a) == 0:
            continue
        err = np.linalg.norm(pg[a] - po[b], axis=1)
        bound = 1e-5 * np.linalg.norm(po[b], axis=1) + n_ev * 7.0 * 2.0 ** -24 * p_max
        worst = max(worst, float((err / bound).max()))
    return matched, worst


def test_fp32_push_between_events():
    # The FP32 path's bound, momentum relative error <= 1e-5 between events,
    # on its own: emission and pairs off, so that every step
    # is the push between events, over far more steps than an event takes
    # (at chi = 1 an electron emits about every 2 steps): every particle
    # within 1e-5 of the FP64 oracle's momentum.  Measured on a GB300: 2.2e-6
    # after 200 steps in the static B, 3e-7 after 20 in the pulse.
    cases = [workloads.test_particles_static_b(n_particles=4000, nsteps=200),
             workloads.beam_laser_collision(n_particles=3000, nsteps=20, seed=4)]
    for w in cases:
        ora, od, _, _ = run_oracle(w, emission_on=0, pairs_on=0)
        gpu, gd = run_gpu(w, precision=32, emission_on=0, pairs_on=0)
        assert gd["status"] == 0
        xg, pg, _, ig = gpu[0]
        xo, po, _, io = ora[0]
        common, a, b = np.intersect1d(ig, io, return_indices=True)
        assert len(common) == len(io) == len(ig)
        rel = np.linalg.norm(pg[a] - po[b], axis=1) / np.linalg.norm(po[b], axis=1)
        assert rel.max() <= 1e-5, (w.name, rel.max())


def test_fp32_statistics():
    w = workloads.test_particles_static_b(n_particles=4000, nsteps=20)
    ora, od, spo, _ = run_oracle(w, nbins=24)
    gpu, gd = run_gpu(w, precision=32, nbins=24)
    assert gd["status"] == 0
    n_o, n_g = od["emissions"], gd["emissions"]
    assert abs(n_g - n_o) <= 3 * math.sqrt(n_o)
    # spectra bin by bin within 3 sigma (Poisson, both sides)
    sg = np.array(gd["spectrum"])
    sig = np.sqrt(np.maximum(spo + sg, 1.0))
    assert np.all(np.abs(sg - spo) <= 3 * sig + 1e-9), (sg, spo)
    # same random words: most particles share their event history with the oracle
    rep = compare(gpu, ora, rtol_p=1.0, xtol=np.inf, species=(0,))
    assert rep["matched"] >= 0.99 * len(ora[0][3])
    # every particle with a shared history within the FP32 bound (at most 40
    # events in any ancestry: about 9 emissions per electron in 20 steps)
    matched, worst = fp32_momentum_bounds(gpu, ora, 1000.0, n_ev=40)
    assert matched >= 0.99 * sum(len(ora[sp][3]) for sp in range(3))
    assert worst <= 1.0, worst
    # energy: the push in a static B conserves it; emission defects are ~1e-6 relative
    e0 = 4000 * 1000.0
    e1 = sum(np.sqrt((1.0 if sp < 2 else 0.0) + (gpu[sp][1] ** 2).sum(1)).sum() for sp in range(3))
    assert abs(e1 / e0 - 1) < 1e-4


def test_fp32_pair_statistics():
    # chi ~ 10 in a static B: photons convert within the run
    w = workloads.test_particles_static_b(n_particles=3000, nsteps=4)
    w.fp = (0, 0, 0, 0, 0, 1e-2)
    w.dt = 3e4
    caps = (60_000, 60_000, 200_000, 1)
    ora, od, _, _ = run_oracle(w, caps=caps)
    gpu, gd = run_gpu(w, precision=32, caps=caps)
    assert gd["status"] == 0 and od["overflow"] == 0
    assert od["pairs"] > 200
    for k in ("emissions", "pairs"):
        assert abs(gd[k] - od[k]) <= 3 * math.sqrt(gd[k] + od[k]), (k, gd[k], od[k])
    # yields per species within 3 sigma
    for sp in range(3):
        n_o, n_g = len(ora[sp][3]), len(gpu[sp][3])
        assert abs(n_g - n_o) <= 3 * math.sqrt(n_g + n_o), (sp, n_g, n_o)
    matched, worst = fp32_momentum_bounds(gpu, ora, 1000.0, n_ev=40)
    assert matched >= 0.9 * sum(len(ora[sp][3]) for sp in range(3))
    assert worst <= 1.0, worst


def test_fp32_gaussian_pulse_statistics():
    # FP32 field evaluation (fixed-point carrier phase) against the FP64 oracle
    w = workloads.beam_laser_collision(n_particles=3000, nsteps=20, seed=4)
    ora, od, _, _ = run_oracle(w)
    gpu, gd = run_gpu(w, precision=32)
    assert gd["status"] == 0
    assert abs(gd["emissions"] - od["emissions"]) <= 3 * math.sqrt(od["emissions"]) and od["emissions"] > 1000
    xg, pg, _, ig = gpu[0]
    xo, po, _, io = ora[0]
    common, a, b = np.intersect1d(ig, io, return_indices=True)
    assert len(common) >= 0.99 * len(io)
    # every particle with a shared history within the FP32 bound; parents
    # never exceed 1.05 of the beam's largest |p|
    p_max = 1.05 * float(np.linalg.norm(w.particles[0][1], axis=1).max())
    matched, worst = fp32_momentum_bounds(gpu, ora, p_max, n_ev=40)
    assert worst <= 1.0, worst
    # photon yield per energy decade within 3 sigma
    eo = np.log10(np.linalg.norm(ora[2][1], axis=1))
    eg = np.log10(np.linalg.norm(gpu[2][1], axis=1))
    ho, edges = np.histogram(eo, bins=8, range=(-6, 2))
    hg, _ = np.histogram(eg, bins=edges)
    assert np.all(np.abs(hg - ho) <= 3 * np.sqrt(np.maximum(ho + hg, 1)))
