"""The large self-consistent cascade at full size (GPU test): 512^3 Yee
mesh, four CP pulses at 2e24 W/cm^2 (two along x, two along y), a hydrogen
slab of 1e22 cm^-3, 0.5 um thick, 8 particles per cell and species (4.2e7
electrons and 4.2e7 protons), thinning every 8 steps.

The particles share the mesh, so no sampled family can be checked against
the oracle; the property checked is the discrete continuity equation of the
deposit over one step,
    (rho1 - rho0)/dt + div J = 0,
at every node of a slab of the mesh around the target (rho from the oracle's
CIC charge density of the electrons, positrons and protons in and near the
slab), in FP32 and in FP64.  The FP64 run also checks that the store of
1.05e9 particles plus the FP64 mesh fits 180 GB.
"""
import numpy as np
import pytest

from oracle import oracle as o
from paper_1412_6426_gb300 import workloads

pytestmark = pytest.mark.gpu

MARGIN = 40        # cells either side of the target in the checked slab


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1412_6426_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()


@pytest.fixture(scope="module")
def case():
    return workloads.large_cascade()


def slab_particles(sim, sp, lo, hi, sign):
    """Positions and charges (sign x weight) of the species' particles with
    lo <= x < hi, read on the device and filtered there."""
    import torch
    from paper_1412_6426_gb300 import qed
    cap = max(sim.caps[sp], 1)
    x = torch.empty((cap, 3), dtype=torch.float64, device="cuda")
    p = torch.empty((cap, 3), dtype=torch.float64, device="cuda")
    wt = torch.empty(cap, dtype=torch.float64, device="cuda")
    ids = torch.empty(cap, dtype=torch.int64, device="cuda")
    n = qed.qed_particles_get(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(), ids.data_ptr(), cap,
                              sim.stream.cuda_stream)
    keep = (x[:n, 0] >= lo) & (x[:n, 0] < hi)
    xs = x[:n][keep].cpu().numpy()
    qs = (sign * wt[:n][keep]).cpu().numpy()
    del x, p, wt, ids
    torch.cuda.empty_cache()
    return xs, qs


def continuity_residual(w, sim, J, step_fn):
    """Takes one step with step_fn and returns (max |residual|, scale) over the
    interior nodes of the slab [i0 - MARGIN, i1 + MARGIN) along x."""
    import torch
    n = w.n
    i0, i1 = w.meta["target_cells"]
    a, b = i0 - MARGIN, i1 + MARGIN
    lo, hi = a * w.d[0], b * w.d[0]
    nsub = (b - a, n[1], n[2])
    x0 = (lo, 0.0, 0.0)

    def rho():
        acc = np.zeros(int(np.prod(nsub)))
        for sp, q in ((0, -1.0), (1, 1.0), (3, 1.0)):
            xs, qs = slab_particles(sim, sp, lo, hi, q)
            if len(qs):
                acc += o.charge_density(nsub, w.d, x0, xs[:, 0], xs[:, 1], xs[:, 2], qs)
        return acc.reshape(nsub[2], nsub[1], nsub[0])

    r0 = rho()
    step_fn()
    r1 = rho()
    sh = (n[2], n[1], n[0])
    Js = [t.reshape(sh)[:, :, a - 1:b].double().cpu().numpy() for t in J]     # one extra column for i - 1
    Jx, Jy, Jz = Js
    div = ((Jx[:, :, 1:] - Jx[:, :, :-1]) / w.d[0]
           + (Jy[:, :, 1:] - np.roll(Jy[:, :, 1:], 1, axis=1)) / w.d[1]
           + (Jz[:, :, 1:] - np.roll(Jz[:, :, 1:], 1, axis=0)) / w.d[2])
    res = (r1 - r0) / w.dt + div
    # nodes within 2 cells of the slab's x faces see particles that crossed them
    inner = res[:, :, 2:-2]
    scale = np.abs((r1 - r0)[:, :, 2:-2]).max() / w.dt
    return float(np.abs(inner).max()), float(scale)


def run_case(w, fx, fy, precision, caps, steps_before, check_footprint=None):
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    n = w.n[0]
    dt_ = torch.float32 if precision == 32 else torch.float64
    F = workloads.expand_profiles(fx, fy, n, xp=torch, dtype=dt_, device="cuda")
    J = [torch.zeros(n ** 3, dtype=dt_, device="cuda") for _ in range(3)]
    free0, _ = torch.cuda.mem_get_info()
    with Simulation(w, precision=precision, capacity=caps, deposit_on=1, compact_interval=8,
                    thin_interval=w.meta["thin_interval"], thin_limit=w.meta["thin_limit"],
                    pending_capacity=50_000_000) as s:
        free1, _ = torch.cuda.mem_get_info()
        footprint = free0 - free1
        s.set_grid_fields(F[:3], F[3:], J)
        s.set_all()
        s.step(steps_before)
        d0 = s.diag()
        res, scale = continuity_residual(w, s, J, lambda: s.step(1))
        d1 = s.diag()
    return footprint, d0, d1, res, scale


def test_large_cascade_fp32_continuity(case):
    w, fx, fy = case
    # step 42 is not a thinning step ((s + 1) % 8 != 0), so weights only move with currents
    _, d0, d1, res, scale = run_case(w, fx, fy, 32, w.meta["capacity32"], 42)
    assert d0["status"] == 0 and d1["status"] == 0
    assert scale > 0
    assert res <= 1e-4 * scale, (res, scale)
    assert d1["count"][2] > 1e7 and d1["count"][3] == 41943040


def test_large_cascade_fp64_footprint_and_continuity(case):
    w, fx, fy = case
    mesh = 9 * w.n[0] ** 3 * 8
    footprint, d0, d1, res, scale = run_case(w, fx, fy, 64, w.meta["capacity64"], 4)
    assert sum(w.meta["capacity64"][:3]) >= 1.0e9
    assert footprint + mesh <= 180e9, (footprint, mesh)
    assert d0["status"] == 0 and d1["status"] == 0 and d1["count"][2] > 0
    assert res <= 1e-10 * scale, (res, scale)
