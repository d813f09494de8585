"""Parity at the workloads' full sizes (GPU tests).

The GPU runs the whole workload in the configuration the bench times
(capacities, compaction every 8 steps); the oracle advances sampled seed
electrons and every product they make, one family at a time.  Particles are
independent in these analytic fields, so each sampled family must appear in
the GPU output with the same ids (same event history) and, in FP64, momenta
within 1e-12 (of max(|p|, a0) in the pulse); the FP32 run on lineage-tagged
families: yields within 3 sigma, every particle with a shared history within
the FP32 bound.
"""
import numpy as np
import pytest

from paper_1412_6426_gb300 import workloads
from tests.util import box_scale, compare, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1412_6426_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()


def gpu_full(w, precision, caps, compact_interval=8):
    from paper_1412_6426_gb300.sim import Simulation
    with Simulation(w, precision=precision, capacity=caps, compact_interval=compact_interval) as s:
        s.set_all()
        s.step(w.nsteps)
        d = s.diag(check=False)
        out = {sp: s.get(sp) for sp in range(4)}
    return out, d


def sampled_families(w, n_sample, seed):
    idx = np.sort(np.random.default_rng(seed).choice(len(w.particles[0][3]), n_sample, replace=False))
    ws = workloads.subset(w, 0, idx)
    ora, od, _, _ = run_oracle(ws, caps=(50_000, 50_000, 400_000, 1))
    assert od["overflow"] == 0
    ids = np.concatenate([ora[sp][3] for sp in range(4)])
    return ora, od, ids


# Electrons cooled to gamma ~ 10 gyrate ~1000 rad over these runs; the FP64
# push rounds like the oracle's, operation by operation, so the rotation
# angle accumulates no difference and the FP64 bound holds: 1e-12.
RTOL_LONG_GYRATION = 1e-12


def test_fp64_static_b_full_size():
    # 1e4 electrons, chi = 1, 200 steps of 0.01 gyro periods
    w = workloads.test_particles_static_b(n_particles=10_000, nsteps=200)
    gpu, gd = gpu_full(w, 64, caps=(12_000, 1_000, 2_000_000, 0))
    assert gd["status"] == 0
    ora, od, ids = sampled_families(w, 60, seed=11)
    rep = compare(gpu, ora, rtol_p=RTOL_LONG_GYRATION, xtol=1e-12 * box_scale(w), subset_ids=ids)
    assert rep["ok"], rep
    assert rep["matched"] > 60 * 80
    for sp in (0, 1):
        common, a, b = np.intersect1d(gpu[sp][3], ora[sp][3], return_indices=True)
        mg, mo = np.linalg.norm(gpu[sp][1][a], axis=1), np.linalg.norm(ora[sp][1][b], axis=1)
        assert np.all(np.abs(mg - mo) <= 1e-13 * mo)


def test_fp64_beam_laser_full_size():
    # 1e6 electrons, a0 = 200, 600 steps: the collision workload.  The pulse's
    # phase at an absolute FP64 position carries |x| 2^-53 of rounding, so
    # the oracle reproduces itself only to 1e-12 of max(|p|, a0) when its
    # origin is shifted (tests/test_oracle_step.py): particles born slow in
    # the pulse (soft photons, pairs) are held to that scale, the others to
    # 1e-12 of their own momentum.
    w = workloads.beam_laser_collision(n_particles=1_000_000, seed=1, nsteps=600)
    gpu, gd = gpu_full(w, 64, caps=(1_300_000, 200_000, 60_000_000, 0))
    assert gd["status"] == 0
    ora, od, ids = sampled_families(w, 40, seed=12)
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w), subset_ids=ids, p_floor=w.meta["a0"])
    assert rep["ok"], rep
    assert rep["matched"] > 40 * 20


def test_fp32_beam_laser_full_size_statistics():
    # The sampled seeds carry lineage bits (the top 7 id bits, which products
    # inherit: 1 + their index among the samples, 0 for every other seed), so
    # the GPU's products of exactly those seeds are known whatever their event
    # histories: yields per species within 3 sigma of the oracle's, and every
    # particle that shares its event history within the FP32 bound (1e-5
    # plus the quantisation of the FP32 event draws in its ancestry,
    # tests/test_gpu_parity.py)
    from tests.test_gpu_parity import fp32_momentum_bounds
    w = workloads.beam_laser_collision(n_particles=1_000_000, seed=1, nsteps=600)
    bits = 7
    idx = np.sort(np.random.default_rng(13).choice(len(w.particles[0][3]), 60, replace=False))
    x, p, wt, ids = w.particles[0]
    lineage = np.zeros(len(ids), dtype=np.uint64)
    lineage[idx] = np.arange(1, 61, dtype=np.uint64)
    w.particles = {0: (x, p, wt, ids | (lineage << np.uint64(64 - bits)))}
    w.ens_bits = bits
    gpu, gd = gpu_full(w, 32, caps=(1_300_000, 200_000, 60_000_000, 0))
    assert gd["status"] == 0
    ws = workloads.subset(w, 0, idx)
    ora, od, _, _ = run_oracle(ws, caps=(50_000, 50_000, 400_000, 1))
    assert od["overflow"] == 0
    sub = {}
    for sp in range(3):
        xg, pg, wg, ig = gpu[sp]
        keep = (ig >> np.uint64(64 - bits)) != 0
        sub[sp] = (xg[keep], pg[keep], wg[keep], ig[keep])
        n_g, n_o = int(keep.sum()), len(ora[sp][3])
        assert abs(n_g - n_o) <= 3 * np.sqrt(max(n_g + n_o, 1)), (sp, n_g, n_o)
    assert len(ora[2][3]) > 1000
    # about 44 emissions per electron over the run: at most 200 events in any ancestry
    p_max = 1.05 * float(np.linalg.norm(p, axis=1).max())
    matched, worst = fp32_momentum_bounds(sub, ora, p_max, n_ev=200)
    assert matched >= 0.9 * sum(len(ora[sp][3]) for sp in range(3))
    assert worst <= 1.0, worst
