"""Helpers shared by the parity tests: run a workload through the oracle and
the CUDA library, and compare the two particle by particle (matched by id)."""
from __future__ import annotations

import numpy as np

from oracle import drive


def default_caps(w):
    base = w.n_initial()
    n_ion = len(w.particles[3][3]) if 3 in w.particles else 0
    return (40 * base + 1024,) * 3 + (max(n_ion, 1),)


def run_oracle(w, nsteps=None, *, caps=None, nbins=0, step0=0, t0=0.0, **opts):
    caps = default_caps(w) if caps is None else caps
    if getattr(w, "ens", None) is not None:
        opts.setdefault("ens", w.ens)
    if getattr(w, "ens_bits", 0):
        opts.setdefault("ens_bits", w.ens_bits)
    return drive.run(w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt,
                     w.nsteps if nsteps is None else nsteps, w.particles, kappa=opts.pop("kappa", w.kappa),
                     seed=opts.pop("seed", w.seed), caps=caps, nbins=nbins, step0=step0, t0=t0, **opts)


def run_gpu(w, nsteps=None, *, precision=64, caps=None, nbins=0, step0=0, t0=0.0, **opts):
    from paper_1412_6426_gb300.sim import Simulation
    caps = default_caps(w) if caps is None else caps
    with Simulation(w, precision=precision, capacity=caps, nbins=nbins, **opts) as sim:
        if step0 or t0:
            sim.set_clock(step0, t0)
        sim.set_all()
        sim.step(w.nsteps if nsteps is None else nsteps)
        d = sim.diag(check=False)
        out = {sp: sim.get(sp) for sp in range(4)} if d["status"] == 0 else None
    return out, d


def box_scale(w):
    return float(max(np.array(w.n) * np.array(w.d)))


def compare(gpu: dict, ora: dict, *, rtol_p: float, xtol: float, species=(0, 1, 2, 3), subset_ids=None,
            rtol_w: float = 0.0, p_floor: float = 0.0):
    """Match particles by id; returns a report dict.  With subset_ids the GPU
    side is restricted to those ids (sampled families at full size).  Weights
    must agree exactly unless rtol_w is given (thinning rescales them by
    ratios of sums whose rounding depends on the summation order).  Momenta
    agree to rtol_p relative to max(|p|, p_floor): p_floor is the momentum
    scale of an external field for particles slower than it (0: plain
    relative error)."""
    rep = {"missing": 0, "extra": 0, "matched": 0, "max_rel_p": 0.0, "max_dx": 0.0}
    for sp in species:
        xg, pg, wg, ig = gpu[sp]
        xo, po, wo, io = ora[sp]
        if subset_ids is not None:
            keep = np.isin(ig, subset_ids)
            xg, pg, wg, ig = xg[keep], pg[keep], wg[keep], ig[keep]
        common, a, b = np.intersect1d(ig, io, return_indices=True)
        rep["missing"] += len(io) - len(common)
        rep["extra"] += len(ig) - len(common)
        rep["matched"] += len(common)
        if len(common) == 0:
            continue
        pa, pb = pg[a], po[b]
        scale = np.maximum(np.linalg.norm(pb, axis=1), max(p_floor, 1e-300))
        rel = np.linalg.norm(pa - pb, axis=1) / scale
        rep["max_rel_p"] = max(rep["max_rel_p"], float(rel.max()))
        rep["max_dx"] = max(rep["max_dx"], float(np.abs(xg[a] - xo[b]).max()))
        if rtol_w > 0.0:
            assert np.allclose(wg[a], wo[b], rtol=rtol_w, atol=0.0), "weights differ"
        else:
            assert np.array_equal(wg[a], wo[b]), "weights differ"
    rep["ok"] = (rep["missing"] == 0 and rep["extra"] == 0 and rep["max_rel_p"] <= rtol_p
                 and rep["max_dx"] <= xtol)
    return rep
