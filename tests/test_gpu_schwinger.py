"""Pairs from the vacuum per cell (Sec. V.B) on the GPU.

FP64 parity with the oracle: the cell-keyed draws make the same pairs in
the same cells at the same points; the pairs then accelerate, radiate and
convert like any particle.  An analytic uniform field and the Yee mesh
(with deposit and field update, so the new pairs' currents act back on E)
are both checked.  FP32: the pair count matches N_cells P_S.
"""
import math

import numpy as np
import pytest

from oracle import drive
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


def uniform_box(E0=0.25, n=24, d=60.0, dt=40.0, nsteps=3):
    return workloads.Workload(name="schwinger", n=(n, n, n), d=(d, d, d), x0=(0.0, 0.0, 0.0),
                              periodic=(1, 1, 1), field_mode=workloads.FIELD_UNIFORM, fp=(0, E0, 0, 0, 0, 0),
                              dt=dt, nsteps=nsteps, particles={}, seed=4, kappa=0.1)


def test_schwinger_fp64_parity_uniform_field():
    w = uniform_box()
    caps = (60_000, 60_000, 200_000, 1)
    ora, od, _, _ = run_oracle(w, caps=caps, schwinger_on=1)
    assert od["schwinger_pairs"] > 300 and od["emissions"] > 0
    gpu, gd = run_gpu(w, precision=64, caps=caps, schwinger_on=1)
    assert gd["status"] == 0
    for k in ("schwinger_pairs", "schwinger_gt1", "emissions", "pairs"):
        assert gd[k] == od[k], k
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w))
    assert rep["ok"], rep


def test_schwinger_fp64_parity_grid():
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    n, d = (8, 8, 8), (60.0, 60.0, 60.0)
    dt = 0.45 * d[0] / math.sqrt(3)
    nc = int(np.prod(n))
    f = [np.zeros(nc) for _ in range(6)]
    f[1][:] = 0.3                                  # uniform Ey
    w = workloads.Workload(name="schwinger_grid", n=n, d=d, x0=(0.0, 0.0, 0.0), periodic=(1, 1, 1),
                           field_mode=workloads.FIELD_GRID, fp=(), dt=dt, nsteps=3, particles={}, seed=6,
                           kappa=0.1)
    caps = (20_000, 20_000, 60_000, 1)
    fo = [a.copy() for a in f]
    Jo = [np.zeros(nc) for _ in range(3)]
    ora, od, _, _ = drive.run(w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt, 3, {}, kappa=w.kappa,
                              seed=w.seed, caps=caps, fields=fo, J=Jo, deposit_on=1, yee=True, schwinger_on=1)
    assert od["schwinger_pairs"] > 50
    E = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in f[:3]]
    B = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in f[3:]]
    J = [torch.zeros(nc, dtype=torch.float64, device="cuda") for _ in range(3)]
    with Simulation(w, precision=64, capacity=caps, deposit_on=1, schwinger_on=1) as s:
        s.set_grid_fields(E, B, J)
        s.step(3)
        gd = s.diag(check=False)
        gpu = {sp: s.get(sp) for sp in range(4)}
    assert gd["status"] == 0 and gd["schwinger_pairs"] == od["schwinger_pairs"]
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w))
    assert rep["ok"], rep
    fg = [t.cpu().numpy() for t in E + B]
    fscale = max(np.abs(a).max() for a in fo)
    for c in range(6):
        assert np.abs(fg[c] - fo[c]).max() <= 1e-12 * fscale, c


def test_schwinger_fp32_count():
    E0, n, d, dt = 0.25, 64, 60.0, 40.0
    w = uniform_box(E0=E0, n=n, d=d, dt=dt, nsteps=1)
    caps = (n ** 3, n ** 3, 1, 1)
    out, gd = run_gpu(w, precision=32, caps=caps, schwinger_on=1, emission_on=0, pairs_on=0)
    assert gd["status"] == 0
    p = E0 * E0 * math.exp(-math.pi / E0) / (4 * math.pi ** 3) * d ** 3 * dt
    N = n ** 3
    k = gd["schwinger_pairs"]
    assert abs(k - N * p) < 5 * math.sqrt(N * p * (1 - p))
    assert len(out[0][3]) == len(out[1][3]) == k
