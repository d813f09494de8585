"""The self-consistent cascade at full size (GPU test): 256^3 Yee mesh, two
counter-propagating CP pulses at 1e24 W/cm^2, 2e5 seeds, FP32.

The particles are coupled through the fields, so no sampled family can be
checked against the oracle; instead a property that holds at any size: the
current deposited in a step satisfies the discrete continuity equation with
the charge densities before and after it,
    (rho1 - rho0)/dt + div J = 0   at every node,
through the cell-block sort, the split advance / tiled deposit kernels,
the unsorted tail, the in-step products (pairs are born at one point, so
they carry no net charge) and the photons' straight flights.  The step
is taken at step 400, after the pulses have met and the cascade has begun.
"""
import numpy as np
import pytest

from oracle import oracle as o
from paper_1412_6426_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1412_6426_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()


def test_cascade_continuity_at_full_size():
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    w, f = workloads.self_consistent_cascade()
    n = w.n
    nc = len(f[0])
    E = [torch.from_numpy(a).cuda() for a in f[:3]]
    B = [torch.from_numpy(a).cuda() for a in f[3:]]
    J = [torch.zeros(nc, dtype=torch.float32, device="cuda") for _ in range(3)]
    caps = (4_000_000, 4_000_000, 200_000_000, 0)
    with Simulation(w, precision=32, capacity=caps, deposit_on=1, compact_interval=8) as s:
        s.set_grid_fields(E, B, J)
        s.set_all()
        s.step(400)
        d0 = s.diag()
        before = {sp: s.get(sp) for sp in (0, 1)}
        s.step(1)
        d1 = s.diag()
        after = {sp: s.get(sp) for sp in (0, 1)}
        Jh = [t.double().cpu().numpy() for t in J]
    assert d0["status"] == 0 and d1["status"] == 0
    assert d1["count"][0] > 1e5 and d1["count"][2] > 1e6 and d1["pairs"] > 0

    def rho(parts):
        acc = np.zeros(nc)
        for sp, q in ((0, -1.0), (1, 1.0)):
            x, _, wt, _ = parts[sp]
            acc += o.charge_density(n, w.d, w.x0, x[:, 0], x[:, 1], x[:, 2], q * wt)
        return acc
    r0, r1 = rho(before), rho(after)
    sh = (n[2], n[1], n[0])
    Jx, Jy, Jz = (a.reshape(sh) for a in Jh)
    div = ((Jx - np.roll(Jx, 1, axis=2)) / w.d[0] + (Jy - np.roll(Jy, 1, axis=1)) / w.d[1]
           + (Jz - np.roll(Jz, 1, axis=0)) / w.d[2])
    res = (r1 - r0).reshape(sh) / w.dt + div
    scale = np.abs(r1 - r0).max() / w.dt
    assert scale > 0
    assert np.abs(res).max() <= 1e-4 * scale, (np.abs(res).max(), scale)
