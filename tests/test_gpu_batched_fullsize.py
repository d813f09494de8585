"""The batched-ensemble workload at full size (GPU tests).

512 ensembles, 8.4e7 seed electrons (the workload the batched bench line
times).  Thinning couples the particles of an ensemble, so sampled families
are compared with the oracle over the first three steps, before the first
thinning (after step index 3): FP64 must match the oracle family by family
(same ids, momenta within 1e-12); FP32 on whole small ensembles, yields
within 3 sigma and every particle with a shared history within its bound.  Thinning itself is
checked through properties that hold at any size: run four steps with and
without it; every (ensemble, species) group keeps its total weight, the
survivors are a subset of the unthinned particles with the same momenta and
one common weight factor, and a group above its limit L keeps about L.
Finally the bench's launch configuration (autotuned, then CUDA-graph
replays) runs to step 64 without a device error and with every group
within its thinning budget.
"""
import math

import numpy as np
import pytest

from paper_1412_6426_gb300 import qed, workloads
from tests.util import box_scale, compare, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    import torch
    from paper_1412_6426_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    return workloads.batched_ensembles()


def thin_opts(w, on=True):
    return dict(thin_interval=w.meta["thin_interval"] if on else 0, thin_limit=w.meta["thin_limit"])


def run_full(w, precision, nsteps, caps, thin=True):
    from paper_1412_6426_gb300.sim import Simulation
    with Simulation(w, precision=precision, capacity=caps, compact_interval=4, **thin_opts(w, thin)) as s:
        s.set_all()
        s.step(nsteps)
        d = s.diag(check=False)
        out = {sp: s.get(sp) for sp in range(3)} if d["status"] == 0 else None
    return out, d


def sampled(w, n_per, ensembles, seed):
    rng = np.random.default_rng(seed)
    x, p, wt, ids = w.particles[0]
    ens_of = (ids >> np.uint64(64 - w.ens_bits)).astype(np.int64)
    pick = []
    for e in ensembles:
        idx = np.flatnonzero(ens_of == e)
        pick.append(rng.choice(idx, min(n_per, len(idx)), replace=False))
    return np.sort(np.concatenate(pick))


def families(w, index, nsteps):
    ws = workloads.subset(w, 0, index)
    ora, od, _, _ = run_oracle(ws, nsteps, caps=(200_000, 200_000, 800_000, 1), thin_interval=0)
    assert od["overflow"] == 0
    ids = np.concatenate([ora[sp][3] for sp in range(4)])
    return ora, od, ids


def small_caps(w):
    n = w.n_initial()
    return (int(1.3 * n) + 4096, int(0.4 * n) + 4096, int(4 * n) + 4096, 0)


def strongest_and_weakest(w, k=6):
    order = np.argsort(w.meta["chi"])
    return list(order[:k]) + list(order[len(order) // 2:len(order) // 2 + k]) + list(order[-k:])


def test_full_size_fp64_sampled_families_match(w):
    gpu, gd = run_full(w, 64, 3, small_caps(w))
    assert gd["status"] == 0
    index = sampled(w, 3, strongest_and_weakest(w), seed=21)
    ora, od, ids = families(w, index, 3)
    gpu4 = dict(gpu)
    gpu4[3] = (np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0, dtype=np.uint64))
    rep = compare(gpu4, ora, rtol_p=1e-12, xtol=1e-12 * box_scale(w), subset_ids=ids)
    assert rep["ok"], rep
    assert rep["matched"] > len(index)


def whole_small_ensembles(w, k=8, max_count=3000):
    """k ensembles of at most max_count seeds, spread over the chi range."""
    small = np.flatnonzero(w.meta["counts"] <= max_count)
    small = small[np.argsort(w.meta["chi"][small])]
    return [int(e) for e in small[np.linspace(0, len(small) - 1, k).round().astype(int)]]


def test_full_size_fp32_whole_ensembles_statistics(w):
    # Whole ensembles (every seed and every product, told apart on the GPU by
    # the ensemble bits of the ids): yields per species within 3 sigma of the
    # oracle's, and every particle that shares its event history within the
    # FP32 bound (1e-5 plus the quantisation of the FP32 event draws in its
    # ancestry, tests/test_gpu_parity.py)
    from tests.test_gpu_parity import fp32_momentum_bounds
    gpu, gd = run_full(w, 32, 3, small_caps(w))
    assert gd["status"] == 0
    ens = whole_small_ensembles(w)
    x, p, wt, ids = w.particles[0]
    shift = np.uint64(64 - w.ens_bits)
    index = np.flatnonzero(np.isin((ids >> shift).astype(np.int64), ens))
    ora, od, _ = families(w, index, 3)
    sub = {}
    for sp in range(3):
        xg, pg, wg, ig = gpu[sp]
        keep = np.isin((ig >> shift).astype(np.int64), ens)
        sub[sp] = (xg[keep], pg[keep], wg[keep], ig[keep])
        n_g, n_o = int(keep.sum()), len(ora[sp][3])
        assert abs(n_g - n_o) <= 3 * math.sqrt(max(n_g + n_o, 1)), (sp, n_g, n_o)
    assert len(ora[2][3]) > 1000
    p_max = 1.05 * float(np.linalg.norm(p[index], axis=1).max())
    matched, worst = fp32_momentum_bounds(sub, ora, p_max, n_ev=60)
    assert matched >= 0.9 * sum(len(ora[sp][3]) for sp in range(3))
    assert worst <= 1.0, worst


def test_full_size_thinning_properties(w):
    caps = small_caps(w)
    thin, dt_ = run_full(w, 32, 4, caps, thin=True)
    base, db = run_full(w, 32, 4, caps, thin=False)
    assert dt_["status"] == 0 and db["status"] == 0 and dt_["thinned"] > 0 and db["thinned"] == 0
    shift = np.uint64(64 - w.ens_bits)
    counts = w.meta["counts"]
    n_ens = len(counts)
    sel = np.array(strongest_and_weakest(w, 16))
    for sp in range(3):
        xa, pa, wa, ia = thin[sp]
        xb, pb, wb, ib = base[sp]
        ea, eb = (ia >> shift).astype(np.int64), (ib >> shift).astype(np.int64)
        # every group keeps its total weight (all 512)
        sa = np.bincount(ea, weights=wa, minlength=n_ens)
        sb = np.bincount(eb, weights=wb, minlength=n_ens)
        assert np.allclose(sa, sb, rtol=1e-5, atol=0)
        na = np.bincount(ea, minlength=n_ens)
        nb = np.bincount(eb, minlength=n_ens)
        L = w.meta["thin_limit"][sp] * counts
        for e in range(n_ens):
            if nb[e] <= L[e]:
                assert na[e] == nb[e]
            else:
                q = L[e] / nb[e]
                assert abs(na[e] - L[e]) < 5 * math.sqrt(nb[e] * q * (1 - q)) + 1
        # on 48 ensembles (weakest, middle, strongest): survivors are a subset
        # with untouched momenta and one common weight factor per group
        ka, kb = np.isin(ea, sel), np.isin(eb, sel)
        common, a, b = np.intersect1d(ia[ka], ib[kb], return_indices=True)
        assert len(common) == int(ka.sum())
        assert np.array_equal(pa[ka][a], pb[kb][b])
        ratio = wa[ka][a] / wb[kb][b]
        eg = ea[ka][a]
        for e in sel:
            r = ratio[eg == e]
            if len(r):
                assert np.allclose(r, r[0], rtol=2e-7)


def test_full_size_bench_configuration(w):
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with Simulation(w, precision=32, capacity=w.capacity, compact_interval=4, stream=stream,
                        **thin_opts(w)) as s:
            s.set_all()
            tuned, n = s.autotune(1, 32)
            assert n <= 32
            s.set_tuning(**tuned)
            G = math.lcm(w.meta["thin_interval"], 2 * tuned["compact_interval"])
            left = 64 - n
            s.step(left % G)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                qed.qed_step(s.ctx, None, w.dt, G, stream.cuda_stream)
            for _ in range(left // G):
                g.replay()
            torch.cuda.synchronize()
            d = s.diag()
            out = {sp: s.get(sp) for sp in range(3)}
    assert d["step"] == 64 and d["status"] == 0 and d["thinned"] > 0
    shift = np.uint64(64 - w.ens_bits)
    counts = w.meta["counts"]
    for sp in range(3):
        e = (out[sp][3] >> shift).astype(np.int64)
        assert e.max() < len(counts)
        n = np.bincount(e, minlength=len(counts))
        L = w.meta["thin_limit"][sp] * counts
        # step 64 ended with a thinning: every group is at most its limit plus noise
        assert np.all(n <= L + 5 * np.sqrt(L) + 1)
