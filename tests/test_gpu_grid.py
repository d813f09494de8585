"""Self-consistent grid mode on the GPU: CIC gather from the Yee mesh,
Esirkepov deposit and the symmetrised FDTD update, against the oracle.

FP64: particles (same ids, momenta 1e-12) and the fields E, B, J after a few
steps (1e-12 of the field scale and of the current scale; the deposit's
atomics sum in a different order), on a mesh the particles fill and in one
dense cell block whose current goes through the shared-memory tile.
FP32: the deposited current satisfies the discrete continuity equation with
the charge densities before and after the step, to FP32 rounding; emissions,
pairs and the photon spectrum agree with the oracle within 3 sigma.
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


def grid_case(seed=5, npart=300, n=(16, 12, 10), E0=5e-3, pmin=50.0, pmax=200.0, region=None, cell=2000.0):
    """A periodic Yee mesh with a plane wave (Ey, Bz) and an Ez harmonic, and
    electrons, positrons and ions with random directions and |p| in
    [pmin, pmax]; region = (lo, hi) in cells puts every particle inside that
    box (a dense cell block), else they fill the mesh."""
    rng = np.random.default_rng(seed)
    d = (cell, cell, cell)
    x0 = (0.0, 0.0, 0.0)
    dt = 0.45 * d[0] / math.sqrt(3)
    L = np.array(n) * np.array(d)
    nc = int(np.prod(n))
    k = 2 * math.pi / L[0]
    I, J_, K = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    flat = ((K * n[1] + J_) * n[0] + I).ravel()
    f = [np.zeros(nc) for _ in range(6)]
    f[1][flat] = (E0 * np.cos(k * I * d[0])).ravel()                  # Ey at (i, j+1/2, k)
    f[5][flat] = (E0 * np.cos(k * (I + 0.5) * d[0])).ravel()          # Bz at (i+1/2, j+1/2, k)
    f[2][flat] = (0.3 * E0 * np.sin(2 * k * I * d[0])).ravel()
    lo, hi = (np.zeros(3), L) if region is None else (np.array(region[0]) * d, np.array(region[1]) * d)

    def place(k):
        return lo + rng.uniform(0, 1, (k, 3)) * (hi - lo)
    parts = {}
    for sp in (0, 1):
        x = place(npart)
        dirs = rng.standard_normal((npart, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        p = dirs * rng.uniform(pmin, pmax, npart)[:, None]
        parts[sp] = (x, p, np.ones(npart), np.arange(npart, dtype=np.uint64) + 10_000 * sp)
    # ions (charge +1, mass 1836.15): pushed and deposited, never emit
    xi = place(npart // 3)
    pi = rng.standard_normal((npart // 3, 3)) * 100.0
    parts[3] = (xi, pi, np.ones(len(xi)), np.arange(len(xi), dtype=np.uint64) + 50_000)
    w = workloads.Workload(name="grid", n=n, d=d, x0=x0, periodic=(1, 1, 1), field_mode=workloads.FIELD_GRID,
                           fp=(), dt=dt, nsteps=5, particles=parts, seed=seed, kappa=0.1)
    return w, f


def run_gpu_grid(w, f, precision, nsteps, caps=(4000, 4000, 8000, 400), nbins=0, tuning=None):
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    dtype = torch.float64 if precision == 64 else torch.float32
    E = [torch.tensor(a, dtype=dtype, device="cuda") for a in f[:3]]
    B = [torch.tensor(a, dtype=dtype, device="cuda") for a in f[3:]]
    J = [torch.zeros(len(f[0]), dtype=dtype, device="cuda") for _ in range(3)]
    with Simulation(w, precision=precision, capacity=caps, deposit_on=1, nbins=nbins) as s:
        if tuning:
            s.set_tuning(**tuning)
        s.set_grid_fields(E, B, J)
        s.set_all()
        s.step(nsteps)
        d = s.diag(check=False)
        out = {sp: s.get(sp) for sp in range(4)}
    fields = [t.double().cpu().numpy() for t in E + B + J]
    return out, d, fields


def fp64_grid_parity(w, f, nsteps, caps=(4000, 4000, 8000, 400), tuning=None):
    from tests.util import compare
    fo = [a.copy() for a in f]
    Jo = [np.zeros_like(f[0]) for _ in range(3)]
    ora, od, _, _ = drive.run(w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt, nsteps, w.particles,
                              kappa=w.kappa, seed=w.seed, caps=caps, fields=fo, J=Jo, deposit_on=1, yee=True)
    gpu, gd, fg = run_gpu_grid(w, f, 64, nsteps, caps=caps, tuning=tuning)
    assert gd["status"] == 0, gd
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
    return gd, od


def test_fp64_grid_parity():
    w, f = grid_case()
    gd, od = fp64_grid_parity(w, f, 5)
    assert gd["emissions"] == od["emissions"] > 10


@pytest.mark.parametrize("n", [(12, 10, 7), (9, 13, 3), (8, 8, 2)])
def test_fp64_grid_parity_mesh_shapes(n):
    # ragged meshes for the field update's launch tiles (32 x 8 cells in x-y,
    # one z plane each) and the cell blocks (8^3): x below a warp, y not a
    # multiple of 8, odd plane counts, and two planes, where the periodic
    # wrap in z meets the neighbour plane from both sides
    w, f = grid_case(seed=17, npart=200, n=n)
    gd, od = fp64_grid_parity(w, f, 4)
    assert gd["emissions"] == od["emissions"]


def test_fp64_grid_parity_drifted_out_of_the_tile():
    # the dense block with a tile of one halo cell over 12 steps without a
    # re-sort: particles near the block's faces move more than a cell out of
    # its tile, are listed and deposited by the drift kernel, and J (like
    # E, B and the particles) still matches the oracle's to 1e-12
    w, f = grid_case(seed=11, npart=2500, n=(16, 16, 16), region=((2, 2, 2), (6, 6, 6)))
    gd, od = fp64_grid_parity(w, f, 12, caps=(20_000, 20_000, 40_000, 2_000), tuning={"deposit_halo": 1})
    assert gd["emissions"] == od["emissions"] > 10
    assert 0.5 * gd["block_steps"] < gd["tile_deposits"] < 0.995 * gd["block_steps"], \
        (gd["tile_deposits"], gd["block_steps"])


@pytest.mark.parametrize("halo", [1, 4, 0])
def test_fp64_grid_parity_dense_cell_block(halo):
    # 2 x 2500 leptons and 830 ions inside one 8^3 cell block of a 16^3 mesh
    # (cells 2..6, so that a few steps' drift keeps every stencil inside the
    # block's current tile): with a tile (halo 1: the block alone; 4: the
    # widest) the deposit goes through shared memory, without one (halo 0)
    # through global atomics, and J must match the oracle's to 1e-12 of its
    # scale either way
    w, f = grid_case(seed=11, npart=2500, n=(16, 16, 16), region=((2, 2, 2), (6, 6, 6)))
    gd, od = fp64_grid_parity(w, f, 3, caps=(20_000, 20_000, 40_000, 2_000), tuning={"deposit_halo": halo})
    assert gd["emissions"] == od["emissions"] > 10
    assert gd["block_steps"] >= 3 * 5800
    if halo:
        assert gd["tile_deposits"] >= 0.99 * gd["block_steps"], (gd["tile_deposits"], gd["block_steps"])
    else:
        assert gd["tile_deposits"] == 0


def test_fp32_grid_statistics():
    # chi ~ 15-60 on the mesh (E0 = 3e-2 E_S, |p| 500-2000, cells of 2e4
    # Compton lengths so that a step of the Courant limit holds about one
    # emission per lepton): emissions, pairs, yields and the photon spectrum
    # of the FP32 path within 3 sigma of the FP64 oracle's; every particle
    # that shares its event history within the FP32 bound (at most 30 events
    # in any ancestry in these 3 steps)
    from tests.test_gpu_parity import fp32_momentum_bounds
    w, f = grid_case(seed=13, npart=3000, E0=3e-2, pmin=500.0, pmax=2000.0, cell=2e4)
    nsteps, caps, nbins = 3, (60_000, 60_000, 200_000, 1_000), 24
    fo = [a.copy() for a in f]
    Jo = [np.zeros_like(f[0]) for _ in range(3)]
    ora, od, spo, _ = drive.run(w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt, nsteps, w.particles,
                                kappa=w.kappa, seed=w.seed, caps=caps, fields=fo, J=Jo, deposit_on=1, yee=True,
                                nbins=nbins)
    gpu, gd, fg = run_gpu_grid(w, f, 32, nsteps, caps=caps, nbins=nbins)
    assert gd["status"] == 0 and od["overflow"] == 0
    assert od["emissions"] > 4000 and od["pairs"] > 30, (od["emissions"], od["pairs"])
    for k in ("emissions", "pairs"):
        assert abs(gd[k] - od[k]) <= 3 * math.sqrt(gd[k] + od[k]), (k, gd[k], od[k])
    for sp in range(3):
        n_o, n_g = len(ora[sp][3]), len(gpu[sp][3])
        assert abs(n_g - n_o) <= 3 * math.sqrt(n_g + n_o), (sp, n_g, n_o)
    sg = np.array(gd["spectrum"])
    assert np.all(np.abs(sg - spo) <= 3 * np.sqrt(np.maximum(sg + spo, 1.0)) + 1e-9), (sg, spo)
    # the field adds at most E0 dt per step to the seeds' largest |p|
    p_max = 2000.0 + 2 * nsteps * 3e-2 * w.dt
    matched, worst = fp32_momentum_bounds(gpu, ora, p_max, n_ev=30)
    assert matched >= 0.9 * sum(len(ora[sp][3]) for sp in range(3))
    assert worst <= 1.0, worst


def continuity_residual(w, f, out, fg):
    """Largest |d rho/dt + div J| over the mesh, and its scale max |d rho|/dt:
    charge densities from the start and end positions (products carry no
    net charge: pairs are born at one point)."""
    def rho(parts, signs):
        acc = np.zeros(len(f[0]))
        for sp, q in signs:
            x, _, wt, _ = parts[sp]
            if len(x):
                acc += o.charge_density(w.n, w.d, w.x0, x[:, 0], x[:, 1], x[:, 2], q * wt)
        return acc
    signs = ((0, -1.0), (1, 1.0), (3, 1.0))
    r0 = rho(w.particles, signs)
    r1 = rho(out, signs)
    Jx, Jy, Jz = fg[6], fg[7], fg[8]
    n = w.n
    idx = lambda i, j, k: ((k % n[2]) * n[1] + (j % n[1])) * n[0] + (i % n[0])
    worst = 0.0
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                c = idx(i, j, k)
                div = (Jx[c] - Jx[idx(i - 1, j, k)]) / w.d[0] + (Jy[c] - Jy[idx(i, j - 1, k)]) / w.d[1] \
                    + (Jz[c] - Jz[idx(i, j, k - 1)]) / w.d[2]
                worst = max(worst, abs((r1[c] - r0[c]) / w.dt + div))
    return worst, np.abs(r1 - r0).max() / w.dt


def test_fp32_grid_continuity():
    w, f = grid_case(seed=9)
    out, d, fg = run_gpu_grid(w, f, 32, 1)
    assert d["status"] == 0, d
    worst, scale = continuity_residual(w, f, out, fg)
    assert worst <= 1e-5 * scale


def test_fp32_grid_continuity_dense_cell_block():
    # 5,800 particles in one 8^3 cell block: every deposit goes through the
    # block's fixed-point current tile, and the discrete continuity equation
    # holds to the same 1e-5 of its scale as with FP32 sums
    w, f = grid_case(seed=11, npart=2500, n=(16, 16, 16), region=((2, 2, 2), (6, 6, 6)))
    out, d, fg = run_gpu_grid(w, f, 32, 1, caps=(20_000, 20_000, 40_000, 2_000))
    assert d["status"] == 0, d
    assert d["tile_deposits"] >= 0.99 * d["block_steps"] >= 0.99 * 5800
    worst, scale = continuity_residual(w, f, out, fg)
    assert worst <= 1e-5 * scale
