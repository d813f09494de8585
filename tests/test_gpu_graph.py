"""qed_step captured in a CUDA graph and replayed (GPU test).

The step index and time live in device memory and are advanced by the first
kernel of every step, so a captured sequence of steps can be replayed.  The
stores are double-buffered by compaction; a captured sequence with an even
number of compactions ends in the buffers it started from.  Replaying 8
captured steps twice must give exactly the particles of 16 eager steps.
"""
import numpy as np
import pytest

from paper_1412_6426_gb300 import qed, workloads
from tests.util import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1412_6426_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()


@pytest.mark.parametrize("precision", [32, 64])
def test_graph_replay_matches_eager(precision):
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    w = workloads.test_particles_static_b(n_particles=500, nsteps=16)
    w.fp = (0, 0, 0, 0, 0, 1e-2)          # chi ~ 10: ~7e4 emissions and ~1.3e3 pairs in 16 steps
    w.dt = 3e4
    caps = (20_000, 20_000, 300_000, 0)
    with Simulation(w, precision=precision, capacity=caps, compact_interval=4) as a:
        a.set_all()
        a.step(16)
        da = a.diag()
        ref = {sp: a.get(sp) for sp in range(4)}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with Simulation(w, precision=precision, capacity=caps, compact_interval=4, stream=stream) as b:
            b.set_all()
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                qed.qed_step(b.ctx, None, w.dt, 8, torch.cuda.current_stream().cuda_stream)
            g.replay()
            g.replay()
            torch.cuda.synchronize()
            db = b.diag()
            out = {sp: b.get(sp) for sp in range(4)}
    assert db["step"] == 16 and da["emissions"] == db["emissions"] > 1000 and da["pairs"] == db["pairs"] > 0
    rep = compare(out, ref, rtol_p=0.0 if precision == 64 else 1e-6, xtol=1e-6)
    assert rep["ok"], rep
