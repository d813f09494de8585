"""qed_particles_read_static: reading particles without any allocation.

Callers whose device memory all belongs to their own pool allocator, or
real-time loops that forbid allocation after start-up, read results with
this entry point; its scratch is a fixed array inside the library.  The
tests call it through the C ABI and check its output against
qed_particles_get on two calls in a row (so the second call starts from the
scratch contents the first one left), then again after more steps with
different counts; a read into a buffer shorter than the live count, a read
into page-locked host memory, an empty species, and a device failure it
reports (which must latch the context like qed_particles_get does).
This file is collected last.
"""
import numpy as np
import pytest

from paper_1412_6426_gb300 import qed, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1412_6426_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()


def buffers(cap, device="cuda"):
    import torch
    pin = device == "cpu"
    return (torch.empty((cap, 3), dtype=torch.float64, device=device, pin_memory=pin),
            torch.empty((cap, 3), dtype=torch.float64, device=device, pin_memory=pin),
            torch.empty(cap, dtype=torch.float64, device=device, pin_memory=pin),
            torch.empty(cap, dtype=torch.int64, device=device, pin_memory=pin))


def read_static(sim, sp, cap, device="cuda"):
    x, p, w, i = buffers(cap, device)
    n = qed.qed_particles_read_static(sim.ctx, sp, x.data_ptr(), p.data_ptr(), w.data_ptr(), i.data_ptr(), cap,
                                      sim.stream.cuda_stream)
    return (x[:n].cpu().numpy(), p[:n].cpu().numpy(), w[:n].cpu().numpy(), i[:n].cpu().numpy().view(np.uint64))


def cascade_sim(precision, caps):
    from paper_1412_6426_gb300.sim import Simulation
    w = workloads.test_particles_static_b(n_particles=3000, nsteps=6)
    w.fp = (0, 0, 0, 0, 0, 1e-2)       # chi ~ 10: photons convert to pairs, leaving dead records
    w.dt = 3e4
    return Simulation(w, precision=precision, capacity=caps)


@pytest.mark.parametrize("precision", [32, 64])
def test_read_static_matches_particles_get(precision):
    caps = (20000, 20000, 60000, 0)
    with cascade_sim(precision, caps) as sim:
        sim.set_all()
        for nsteps in (3, 2):
            sim.step(nsteps)
            assert sim.diag()["pairs"] > 0
            first = {sp: read_static(sim, sp, caps[sp]) for sp in range(3)}
            second = {sp: read_static(sim, sp, caps[sp]) for sp in range(3)}
            ref = {sp: sim.get(sp) for sp in range(3)}    # compacts the store
            for sp in range(3):
                assert len(ref[sp][3]) > 0
                for got in (first[sp], second[sp]):
                    for a, b in zip(got, ref[sp]):
                        assert np.array_equal(a, b), sp


def test_read_static_partial_pinned_and_empty():
    import torch
    caps = (20000, 20000, 60000, 0)
    with cascade_sim(32, caps) as sim:
        sim.set_all()
        sim.step(3)
        live = sim.diag()["count"]
        k = live[2] // 3
        assert k > 10
        # a buffer shorter than the live count: the first k records in store
        # order are written and the call reports the live count with QED_ERR_ARG
        x, p, w, i = buffers(k)
        with pytest.raises(qed.QedError) as e:
            qed.qed_particles_read_static(sim.ctx, 2, x.data_ptr(), p.data_ptr(), w.data_ptr(), i.data_ptr(), k,
                                          sim.stream.cuda_stream)
        assert e.value.status == qed.QED_ERR_ARG
        torch.cuda.synchronize()
        part = (x.cpu().numpy(), p.cpu().numpy(), w.cpu().numpy(), i.cpu().numpy().view(np.uint64))
        # page-locked host output through its device alias
        host = {sp: read_static(sim, sp, caps[sp], device="cpu") for sp in range(2)}
        # the ion store has no capacity and no particles: one empty read
        empty = read_static(sim, 3, 0)
        assert all(len(a) == 0 for a in empty)
        ref = {sp: sim.get(sp) for sp in range(3)}
        for a, b in zip(part, ref[2]):
            assert np.array_equal(a, b[:k])
        for sp in range(2):
            for a, b in zip(host[sp], ref[sp]):
                assert np.array_equal(a, b), sp


def test_read_static_refuses_pageable_and_small_buffers():
    from paper_1412_6426_gb300.sim import Simulation
    w = workloads.test_particles_static_b(n_particles=100, nsteps=1)
    with Simulation(w, precision=32, capacity=(200, 10, 500, 0)) as sim:
        sim.set_all()
        host = [np.zeros((200, 3)), np.zeros((200, 3)), np.zeros(200), np.zeros(200, dtype=np.uint64)]
        with pytest.raises(qed.QedError) as e:
            qed.qed_particles_read_static(sim.ctx, 0, *[a.ctypes.data for a in host], 200, sim.stream.cuda_stream)
        assert e.value.status == qed.QED_ERR_ARG
        with pytest.raises(qed.QedError) as e:
            read_static(sim, 0, 50)
        assert e.value.status == qed.QED_ERR_ARG


def test_read_static_latches_a_device_failure():
    from paper_1412_6426_gb300.sim import Simulation
    w = workloads.test_particles_static_b(n_particles=100, nsteps=1)
    x, p, wt, ids = w.particles[0]
    p = p.copy()
    p[7, 1] = np.nan                   # a non-finite momentum: the step reports it
    w.particles = {0: (x, p, wt, ids)}
    with Simulation(w, precision=32, capacity=(200, 10, 500, 0)) as sim:
        sim.set_all()
        sim.step(1)
        with pytest.raises(qed.QedError) as e:
            read_static(sim, 0, 200)
        assert e.value.status == qed.QED_ERR_NONFINITE
        # the context now refuses to step, as after qed_particles_get
        with pytest.raises(qed.QedError) as e:
            sim.step(1)
        assert e.value.status == qed.QED_ERR_STATE
