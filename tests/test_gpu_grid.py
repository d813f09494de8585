"""Self-consistent grid mode on the GPU: CIC gather from the Yee mesh,
Esirkepov deposit and the symmetrised FDTD update, against the oracle.

FP64: particles (same ids, momenta 1e-12) and the fields E, B, J after a few
steps (1e-12 of the field scale and of the current scale; the deposit's
atomics sum in a different order).
FP32: the deposited current satisfies the discrete continuity equation with
the charge densities before and after the step, to FP32 rounding.
"""
import math

import numpy as np
import pytest

from oracle import drive
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


def grid_case(seed=5, npart=300):
    rng = np.random.default_rng(seed)
    n = (16, 12, 10)
    d = (2000.0, 2000.0, 2000.0)
    x0 = (0.0, 0.0, 0.0)
    dt = 0.45 * d[0] / math.sqrt(3)
    L = np.array(n) * np.array(d)
    nc = int(np.prod(n))
    E0 = 5e-3
    k = 2 * math.pi / L[0]
    I, J_, K = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    flat = ((K * n[1] + J_) * n[0] + I).ravel()
    f = [np.zeros(nc) for _ in range(6)]
    f[1][flat] = (E0 * np.cos(k * I * d[0])).ravel()                  # Ey at (i, j+1/2, k)
    f[5][flat] = (E0 * np.cos(k * (I + 0.5) * d[0])).ravel()          # Bz at (i+1/2, j+1/2, k)
    f[2][flat] = (0.3 * E0 * np.sin(2 * k * I * d[0])).ravel()
    parts = {}
    for sp in (0, 1):
        x = rng.uniform(0, 1, (npart, 3)) * L
        dirs = rng.standard_normal((npart, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        p = dirs * rng.uniform(50, 200, npart)[:, None]
        parts[sp] = (x, p, np.ones(npart), np.arange(npart, dtype=np.uint64) + 10_000 * sp)
    # ions (charge +1, mass 1836.15): pushed and deposited, never emit
    xi = rng.uniform(0, 1, (npart // 3, 3)) * L
    pi = rng.standard_normal((npart // 3, 3)) * 100.0
    parts[3] = (xi, pi, np.ones(len(xi)), np.arange(len(xi), dtype=np.uint64) + 50_000)
    w = workloads.Workload(name="grid", n=n, d=d, x0=x0, periodic=(1, 1, 1), field_mode=workloads.FIELD_GRID,
                           fp=(), dt=dt, nsteps=5, particles=parts, seed=seed, kappa=0.1)
    return w, f


def run_gpu_grid(w, f, precision, nsteps):
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    dtype = torch.float64 if precision == 64 else torch.float32
    E = [torch.tensor(a, dtype=dtype, device="cuda") for a in f[:3]]
    B = [torch.tensor(a, dtype=dtype, device="cuda") for a in f[3:]]
    J = [torch.zeros(len(f[0]), dtype=dtype, device="cuda") for _ in range(3)]
    caps = (4000, 4000, 8000, 400)
    with Simulation(w, precision=precision, capacity=caps, deposit_on=1) as s:
        s.set_grid_fields(E, B, J)
        s.set_all()
        s.step(nsteps)
        d = s.diag(check=False)
        out = {sp: s.get(sp) for sp in range(4)}
    fields = [t.double().cpu().numpy() for t in E + B + J]
    return out, d, fields


def test_fp64_grid_parity():
    from tests.util import compare
    w, f = grid_case()
    nsteps = 5
    fo = [a.copy() for a in f]
    Jo = [np.zeros_like(f[0]) for _ in range(3)]
    ora, od, _, _ = drive.run(w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt, nsteps, w.particles,
                              kappa=w.kappa, seed=w.seed, caps=(4000, 4000, 8000, 400), fields=fo, J=Jo,
                              deposit_on=1, yee=True)
    gpu, gd, fg = run_gpu_grid(w, f, 64, nsteps)
    assert gd["status"] == 0, gd
    assert gd["emissions"] == od["emissions"] > 10
    rep = compare(gpu, ora, rtol_p=1e-12, xtol=1e-9)
    assert rep["ok"], rep
    # E and B against the field scale: components that start at zero (Bx, Ex)
    # are differences of O(E0) neighbours, so their error is the ulp of E0
    fscale = max(np.abs(a).max() for a in fo)
    for c in range(6):
        assert np.abs(fg[c] - fo[c]).max() <= 1e-12 * fscale, c
    jscale = max(np.abs(a).max() for a in Jo)
    for c in range(3):
        assert np.abs(fg[6 + c] - Jo[c]).max() <= 1e-12 * jscale, c


def test_fp32_grid_continuity():
    w, f = grid_case(seed=9)
    gpu0 = {sp: w.particles[sp] for sp in (0, 1)}
    out, d, fg = run_gpu_grid(w, f, 32, 1)
    assert d["status"] == 0, d
    # charge densities from the start and end positions (products carry no
    # net charge: pairs are born at one point)
    def rho(parts, signs):
        acc = np.zeros(len(f[0]))
        for sp, q in signs:
            x, _, wt, _ = parts[sp]
            if len(x):
                acc += o.charge_density(w.n, w.d, w.x0, x[:, 0], x[:, 1], x[:, 2], q * wt)
        return acc
    gpu0[3] = w.particles[3]
    r0 = rho(gpu0, ((0, -1.0), (1, 1.0), (3, 1.0)))
    r1 = rho(out, ((0, -1.0), (1, 1.0), (3, 1.0)))
    Jx, Jy, Jz = fg[6], fg[7], fg[8]
    n = w.n
    idx = lambda i, j, k: ((k % n[2]) * n[1] + (j % n[1])) * n[0] + (i % n[0])
    worst = 0.0
    scale = np.abs(r1 - r0).max() / w.dt
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                c = idx(i, j, k)
                div = (Jx[c] - Jx[idx(i - 1, j, k)]) / w.d[0] + (Jy[c] - Jy[idx(i, j - 1, k)]) / w.d[1] \
                    + (Jz[c] - Jz[idx(i, j, k - 1)]) / w.d[2]
                worst = max(worst, abs((r1[c] - r0[c]) / w.dt + div))
    assert worst <= 1e-5 * scale
