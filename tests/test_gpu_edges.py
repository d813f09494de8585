"""Edge cases and failure reporting of the CUDA library (GPU tests).

Failures are provoked on the host side only (too-small buffers, non-finite
inputs, strict probability checks); the device reports them through its
status word and the context refuses further steps.  Also: empty stores,
table export/import, restart through qed_set_clock, host (pageable and
pinned) input/output, ions, and the rotating-field mode.
"""
import ctypes
import math

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


def sim_for(w, **kw):
    from paper_1412_6426_gb300.sim import Simulation
    return Simulation(w, **kw)


def test_capacity_overflow_reported_and_latched():
    w = workloads.test_particles_static_b(n_particles=500, nsteps=10)
    with sim_for(w, precision=64, capacity=(600, 10, 50, 0)) as s:
        s.set_all()
        s.step(10)
        d = s.diag(check=False)
        assert d["status"] == qed.QED_ERR_CAPACITY and d["overflow"] > 0
        with pytest.raises(qed.QedError) as e:
            s.step(1)
        assert e.value.status == qed.QED_ERR_STATE


def test_pending_overflow_reported():
    w = workloads.test_particles_static_b(n_particles=500, nsteps=3)
    w.fp = (0, 0, 0, 0, 0, 3e-2)
    w.dt = 2e4
    with sim_for(w, precision=32, capacity=(10**5,) * 3 + (0,), pending_capacity=16) as s:
        s.set_all()
        s.step(3)
        assert s.diag(check=False)["status"] == qed.QED_ERR_CAPACITY


def test_nonfinite_input_reported():
    w = workloads.test_particles_static_b(n_particles=64, nsteps=1)
    x, p, wt, ids = w.particles[0]
    p = p.copy()
    p[5, 1] = np.nan
    w.particles = {0: (x, p, wt, ids)}
    with sim_for(w, precision=64, capacity=(1000, 10, 1000, 0)) as s:
        s.set_all()
        s.step(1)
        assert s.diag(check=False)["status"] == qed.QED_ERR_NONFINITE


def test_pm_strict():
    # kappa = 50 and a step 4x the usual: one sub-interval, P_m up to ~2.8
    w = workloads.test_particles_static_b(n_particles=64, nsteps=2)
    w.dt *= 4
    with sim_for(w, precision=64, capacity=(1000, 10, 5000, 0), kappa=50.0, pm_strict=1) as s:
        s.set_all()
        s.step(2)
        d = s.diag(check=False)
        assert d["pm_gt1"] > 0 and d["status"] == qed.QED_ERR_PMGT1
    ora, od, _, _ = run_oracle(w, kappa=50.0)
    assert od["pm_gt1"] == d["pm_gt1"]


@pytest.mark.parametrize("precision", [32, 64])
def test_empty_stores(precision):
    w = workloads.test_particles_static_b(n_particles=0, nsteps=3)
    with sim_for(w, precision=precision, capacity=(0, 0, 0, 0)) as s:
        s.set_all()
        s.step(3)
        d = s.diag()
        assert d["count"] == [0, 0, 0, 0] and d["particle_steps"] == 0 and d["step"] == 3
        assert len(s.get(0)[3]) == 0


def test_invalid_step_arguments():
    w = workloads.test_particles_static_b(n_particles=8, nsteps=1)
    with sim_for(w, precision=32, capacity=(16, 16, 16, 0)) as s:
        with pytest.raises(qed.QedError) as e:
            s.step(1, dt=-1.0)
        assert e.value.status == qed.QED_ERR_ARG
        with pytest.raises(qed.QedError):
            qed.qed_particles_set(s.ctx, 0, 0, 0, 0, 0, 17)   # above capacity


@pytest.mark.parametrize("precision", [32, 64])
def test_tables_roundtrip(precision):
    w = workloads.test_particles_static_b(n_particles=300, nsteps=4)
    caps = (400, 10, 4000, 0)
    with sim_for(w, precision=precision, capacity=caps) as a:
        tab = qed.qed_tables_export(a.ctx)
        a.set_all()
        a.step(4)
        ra = {sp: a.get(sp) for sp in range(3)}
    with sim_for(w, precision=precision, capacity=caps, tables=tab) as b:
        assert qed.qed_tables_export(b.ctx) == tab
        b.set_all()
        b.step(4)
        rb = {sp: b.get(sp) for sp in range(3)}
    for sp in range(3):
        assert np.array_equal(np.sort(ra[sp][3]), np.sort(rb[sp][3]))


def test_restart_with_clock():
    w = workloads.test_particles_static_b(n_particles=300, nsteps=10)
    caps = (400, 10, 6000, 0)
    ref, _ = run_gpu(w, 10, precision=64, caps=caps)
    with sim_for(w, precision=64, capacity=caps) as a:
        a.set_all()
        a.step(5)
        mid = {sp: a.get(sp) for sp in range(3)}
    with sim_for(w, precision=64, capacity=caps) as b:
        for sp in range(3):
            b.set(sp, *mid[sp])
        b.set_clock(5, 5 * w.dt)
        b.step(5)
        out = {sp: b.get(sp) for sp in range(4)}
    rep = compare(out, ref, rtol_p=1e-12, xtol=1e-12 * box_scale(w))
    assert rep["ok"], rep


def test_host_io_pageable_and_pinned():
    import torch
    w = workloads.test_particles_static_b(n_particles=1000, nsteps=3)
    caps = (1200, 10, 6000, 0)
    ref, _ = run_gpu(w, precision=64, caps=caps)
    x, p, wt, ids = w.particles[0]
    for pinned in (False, True):
        with sim_for(w, precision=64, capacity=caps) as s:
            if pinned:
                bufs = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (x, p, wt)]
                bi = torch.from_numpy(ids.view(np.int64)).pin_memory()
                ptrs = [b.data_ptr() for b in bufs] + [bi.data_ptr()]
            else:
                arrs = [np.ascontiguousarray(a) for a in (x, p, wt)] + [np.ascontiguousarray(ids)]
                ptrs = [a.ctypes.data for a in arrs]
            qed.qed_particles_set(s.ctx, 0, *ptrs, len(ids), s.stream.cuda_stream)
            s.step(3)
            out = {}
            for sp in range(4):
                cap = max(caps[sp], 1)
                hx, hp, hw = np.zeros((cap, 3)), np.zeros((cap, 3)), np.zeros(cap)
                hi = np.zeros(cap, dtype=np.uint64)
                n = qed.qed_particles_get(s.ctx, sp, hx.ctypes.data, hp.ctypes.data, hw.ctypes.data,
                                          hi.ctypes.data, cap, s.stream.cuda_stream)
                out[sp] = (hx[:n], hp[:n], hw[:n], hi[:n])
        rep = compare(out, ref, rtol_p=0.0, xtol=0.0)
        assert rep["ok"], (pinned, rep)


def test_ions_pushed_without_emission():
    w = workloads.test_particles_static_b(n_particles=50, nsteps=5)
    x, p, wt, ids = w.particles[0]
    w.particles = {0: (x, p, wt, ids), 3: (x.copy(), p.copy() * 1836.0, wt, ids + 1000)}
    w.field_mode, w.fp = workloads.FIELD_UNIFORM, (1e-4, 2e-4, 0, 0, 0, 1e-3)
    caps = (100, 10, 2000, 60)
    ora, od, _, _ = run_oracle(w, caps=caps)
    gpu, gd = run_gpu(w, precision=64, caps=caps)
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w))
    assert rep["ok"], rep
    assert len(gpu[3][3]) == 50


def test_fp64_rotating_field_parity():
    # rotating E (the batched-ensemble field form): chi ~ 3
    w = workloads.test_particles_static_b(n_particles=300, nsteps=10)
    w.field_mode = workloads.FIELD_ROTATING_E
    omega = workloads.laser_omega(0.8e-6)
    w.fp = (3e-3, omega)
    w.dt = 2 * math.pi / omega / 100
    x, p, wt, ids = w.particles[0]
    p = np.zeros_like(p)
    p[:, 2] = math.sqrt(1000.0 ** 2 - 1)       # perpendicular to the rotation plane
    w.particles = {0: (x, p, wt, ids)}
    ora, od, _, _ = run_oracle(w)
    gpu, gd = run_gpu(w, precision=64)
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w))
    assert rep["ok"], rep
    assert gd["emissions"] == od["emissions"] > 100


def test_bounded_barrier_gives_up():
    # The grid barrier between the passes of the in-step products, with one
    # block that never arrives: the other blocks give up after the poll limit
    # (2^14 polls of ~64 ns) with QED_ERR_TIMEOUT instead of waiting forever,
    # and the context stays usable.  With every block present the barrier
    # lets them all through.
    import time
    from paper_1412_6426_gb300.sim import Simulation
    w = workloads.test_particles_static_b(n_particles=100, nsteps=2)
    with Simulation(w, precision=32, capacity=(2000, 100, 5000, 0)) as sim:
        sim.set_all()
        assert qed.qed_selftest_barrier(sim.ctx, -1, 1 << 20, sim.stream.cuda_stream) == qed.QED_OK
        t0 = time.perf_counter()
        assert qed.qed_selftest_barrier(sim.ctx, 3, 1 << 14, sim.stream.cuda_stream) == qed.QED_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 5.0
        sim.step(2)
        d = sim.diag()
        assert d["status"] == 0 and d["emissions"] > 0


def test_stage_events_per_step_of_a_call():
    # One block of stage events per step of a qed_step call: the first two
    # steps of a three-step call record theirs, in order on the stream, the
    # third records none; a count that is not a multiple of the stages (above
    # one block) is refused.  On the mesh the later steps of the call take
    # the field maxima from the field update before them.
    import torch
    from tests.test_gpu_grid import grid_case
    from paper_1412_6426_gb300.sim import Simulation
    w, f = grid_case(seed=21, npart=300)
    n = qed.QED_NSTAGES
    with Simulation(w, precision=32, capacity=(4000, 4000, 8000, 400), deposit_on=1) as sim:
        dt_ = torch.float32
        E = [torch.tensor(a, dtype=dt_, device="cuda") for a in f[:3]]
        B = [torch.tensor(a, dtype=dt_, device="cuda") for a in f[3:]]
        J = [torch.zeros(len(f[0]), dtype=dt_, device="cuda") for _ in range(3)]
        sim.set_grid_fields(E, B, J)
        sim.set_all()
        stream = sim.stream
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * n)]
        for e_ in ev:
            e_.record(stream)
        torch.cuda.synchronize()
        with pytest.raises(qed.QedError) as e:
            qed.qed_profile_stages(sim.ctx, [x.cuda_event for x in ev[: n + 1]])
        assert e.value.status == qed.QED_ERR_ARG
        mark = torch.cuda.Event(enable_timing=True)
        mark.record(stream)
        qed.qed_profile_stages(sim.ctx, [x.cuda_event for x in ev[: 2 * n]])
        sim.step(3)
        qed.qed_profile_stages(sim.ctx, [])
        torch.cuda.synchronize()
        # steps 0 and 1 recorded after the mark, in order; the third block untouched (before the mark)
        seq = [mark] + ev[: 2 * n]
        for a_, b_ in zip(seq, seq[1:]):
            assert a_.elapsed_time(b_) >= 0.0
        assert mark.elapsed_time(ev[2 * n]) < 0.0
        assert sim.diag()["status"] == 0
