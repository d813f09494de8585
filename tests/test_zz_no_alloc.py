"""qed_particles_read_static: reading particles without any allocation.

Callers that cannot call cudaMalloc (inside CUDA graph capture, under their
own pool allocator, in allocation-free real-time loops) read results with
this entry point; its scratch is a fixed array inside the library.  The test
calls it through the C ABI and checks its output against qed_particles_get
on two calls in a row (so the second call starts from the scratch contents
the first one left), then again after more steps with different counts.
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


def read_static(sim, sp, cap):
    import torch
    x = torch.empty((cap, 3), dtype=torch.float64, device="cuda")
    p = torch.empty((cap, 3), dtype=torch.float64, device="cuda")
    w = torch.empty(cap, dtype=torch.float64, device="cuda")
    i = torch.empty(cap, dtype=torch.int64, device="cuda")
    n = qed.qed_particles_read_static(sim.ctx, sp, x.data_ptr(), p.data_ptr(), w.data_ptr(), i.data_ptr(), cap,
                                      sim.stream.cuda_stream)
    return (x[:n].cpu().numpy(), p[:n].cpu().numpy(), w[:n].cpu().numpy(), i[:n].cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("precision", [32, 64])
def test_read_static_matches_particles_get(precision):
    from paper_1412_6426_gb300.sim import Simulation
    w = workloads.test_particles_static_b(n_particles=3000, nsteps=6)
    w.fp = (0, 0, 0, 0, 0, 1e-2)       # chi ~ 10: photons convert to pairs, leaving dead records
    w.dt = 3e4
    caps = (20000, 20000, 60000, 0)
    with Simulation(w, precision=precision, capacity=caps) as sim:
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
