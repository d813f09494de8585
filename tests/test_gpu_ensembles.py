"""Independent ensembles, generator factors and thinning on the GPU (Sec. VI).

* FP64 parity with the oracle, particle by particle: a small batch of
  rotating-field ensembles with per-ensemble thinning; a static-B shower with
  the generator factors f_g and N_g on both generators; thinning without
  ensembles (one group per species).  Ids must match exactly (identical
  event, keep and thinning decisions); momenta within 1e-12; weights within
  1e-12 (thinning multiplies them by ratios of sums whose rounding depends
  on the summation order).
* The tuning (launch shapes, work stealing, compaction interval, sorting by
  ensemble) and the autotuner change no result: FP32 runs with different
  tunings give the same particles bit for bit (weights to rounding).
* A batched run captured in a CUDA graph and replayed equals the eager run.
"""
import numpy as np
import pytest

from paper_1412_6426_gb300 import qed, workloads
from tests.util import box_scale, compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1412_6426_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()


def small_batch(nsteps=12, n_ens=6, seed=3, count_range=(30, 300)):
    return workloads.batched_ensembles(n_ens=n_ens, count_range=count_range, nsteps=nsteps, seed=seed)


def thin_opts(w):
    return dict(thin_interval=w.meta["thin_interval"], thin_limit=w.meta["thin_limit"])


def caps_for(w, k=60):
    n = w.n_initial()
    return (k * n + 1024, k * n + 1024, 4 * k * n + 1024, 1)


def test_batched_ensembles_fp64_parity():
    w = small_batch()
    caps = caps_for(w)
    ora, od, _, _ = run_oracle(w, caps=caps, **thin_opts(w))
    assert od["overflow"] == 0 and od["emissions"] > 500 and od["pairs"] > 10 and od["thinned"] > 100
    gpu, gd = run_gpu(w, precision=64, caps=caps, compact_interval=4, **thin_opts(w))
    assert gd["status"] == 0
    assert gd["emissions"] == od["emissions"] and gd["pairs"] == od["pairs"]
    assert gd["thinned"] == od["thinned"]
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w), rtol_w=1e-12)
    assert rep["ok"], rep
    # every particle stayed in its seed's ensemble
    hi = np.uint64(64 - w.ens_bits)
    for sp in range(3):
        assert np.all((gpu[sp][3] >> hi) < 6)


def test_generator_factors_fp64_parity():
    w = workloads.test_particles_static_b(n_particles=300, nsteps=6)
    w.fp = (0, 0, 0, 0, 0, 1e-2)          # chi ~ 10: emissions and pairs
    w.dt = 3e4
    opts = dict(emit_fg=3.0, emit_ng=2, pair_fg=2.0, pair_ng=3)
    caps = (60_000, 60_000, 400_000, 1)
    ora, od, _, _ = run_oracle(w, caps=caps, **opts)
    assert od["overflow"] == 0 and od["pairs_created"] > 10
    gpu, gd = run_gpu(w, precision=64, caps=caps, **opts)
    assert gd["status"] == 0
    for k in ("emissions", "pairs", "photons_created", "pairs_created"):
        assert gd[k] == od[k], k
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w))
    assert rep["ok"], rep


def test_thinning_without_ensembles_fp64_parity():
    w = workloads.test_particles_static_b(n_particles=400, nsteps=8)
    opts = dict(thin_interval=2, thin_limit=(0, 0, 300, 0))
    caps = (20_000, 20_000, 100_000, 1)
    ora, od, _, _ = run_oracle(w, caps=caps, **opts)
    assert od["thinned"] > 100
    gpu, gd = run_gpu(w, precision=64, caps=caps, **opts)
    assert gd["status"] == 0 and gd["thinned"] == od["thinned"]
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w), rtol_w=1e-12)
    assert rep["ok"], rep


def test_lineage_bits_and_thinning_fp64_parity():
    # seeds tagged in the top 4 id bits, products inheriting them, thinning
    # of whole species (no ensemble field mode)
    w = workloads.test_particles_static_b(n_particles=400, nsteps=8)
    x, p, wt, ids = w.particles[0]
    w.particles = {0: (x, p, wt, ids | (np.uint64(7) << np.uint64(60)))}
    w.ens_bits = 4
    opts = dict(thin_interval=2, thin_limit=(0, 0, 300, 0))
    caps = (20_000, 20_000, 100_000, 1)
    ora, od, _, _ = run_oracle(w, caps=caps, **opts)
    assert od["thinned"] > 100
    gpu, gd = run_gpu(w, precision=64, caps=caps, **opts)
    assert gd["status"] == 0 and gd["thinned"] == od["thinned"]
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w), rtol_w=1e-12)
    assert rep["ok"], rep
    assert all(((i >> np.uint64(60)) == 7).all() for sp in range(3) for i in [gpu[sp][3]] if len(i))


def _run32(w, nsteps, tuning=None, autotune=None):
    from paper_1412_6426_gb300.sim import Simulation
    with Simulation(w, precision=32, capacity=caps_for(w), compact_interval=4, **thin_opts(w)) as s:
        s.set_all()
        done = 0
        if tuning:
            s.set_tuning(**tuning)
        if autotune:
            t, done = s.autotune(autotune, nsteps)
            assert done <= nsteps
        s.step(nsteps - done)
        d = s.diag()
        return {sp: s.get(sp) for sp in range(4)}, d


def test_tuning_changes_no_result():
    w = small_batch(nsteps=16, n_ens=8, count_range=(100, 2000))
    ref, dr = _run32(w, 16)
    assert dr["emissions"] > 1000 and dr["thinned"] > 0
    for tuning in (dict(work_chunk=256, massive_blocks_per_sm=1, photon_blocks_per_sm=1),
                   dict(work_chunk=4096, compact_interval=2, sort_massive=0),
                   dict(work_chunk=0, compact_interval=1, sort_massive=1),
                   dict(concurrent=1, photon_blocks_per_sm=2, massive_blocks_per_sm=1, work_chunk=1024)):
        out, d = _run32(w, 16, tuning=tuning)
        assert d["emissions"] == dr["emissions"] and d["pairs"] == dr["pairs"] and d["thinned"] == dr["thinned"]
        rep = compare(out, ref, rtol_p=0.0, xtol=0.0, rtol_w=1e-6)
        assert rep["ok"], (tuning, rep)


def test_autotune_changes_no_result():
    w = small_batch(nsteps=96, n_ens=8, count_range=(100, 2000))
    ref, dr = _run32(w, 96)
    out, d = _run32(w, 96, autotune=1)
    assert d["step"] == 96
    rep = compare(out, ref, rtol_p=0.0, xtol=0.0, rtol_w=1e-6)
    assert rep["ok"], rep


def test_batched_graph_replay_matches_eager():
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    w = small_batch(nsteps=16, n_ens=8, count_range=(100, 2000))
    ref, dr = _run32(w, 16)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with Simulation(w, precision=32, capacity=caps_for(w), compact_interval=4, stream=stream,
                        **thin_opts(w)) as b:
            b.set_all()
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            # 8 steps: two compactions, so the replay ends in the buffers it started from
            with torch.cuda.graph(g, stream=stream):
                qed.qed_step(b.ctx, None, w.dt, 8, torch.cuda.current_stream().cuda_stream)
            g.replay()
            g.replay()
            torch.cuda.synchronize()
            db = b.diag()
            out = {sp: b.get(sp) for sp in range(4)}
    assert db["step"] == 16 and db["emissions"] == dr["emissions"] and db["thinned"] == dr["thinned"]
    rep = compare(out, ref, rtol_p=0.0, xtol=0.0, rtol_w=1e-6)
    assert rep["ok"], rep
