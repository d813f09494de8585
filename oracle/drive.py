"""Drive the FP64 oracle through whole steps from plain arrays.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  Imports
nothing from the product package: inputs arrive as plain numbers and numpy
arrays.
"""
from __future__ import annotations

import numpy as np

from . import oracle as o


def run(n, d, x0, periodic, field_mode, fp, dt, nsteps, particles: dict, *, kappa: float, seed: int,
        nsub_max: int = 1000, emission_on: int = 1, pairs_on: int = 1, same_step_children: int = 1,
        caps=None, nbins: int = 0, lg_lo: float = -12.0, lg_hi: float = 0.0, step0: int = 0,
        t0: float = 0.0, fields=None, J=None, deposit_on: int = 0, yee: bool = False,
        ion_charge: float = 1.0, ion_mass: float = 1836.15267343, time_from: int = 0,
        ens_bits: int = 0, ens=None, emit_fg: float = 1.0, emit_ng: int = 1, pair_fg: float = 1.0,
        pair_ng: int = 1, thin_interval: int = 0, thin_limit=(0, 0, 0, 0), generator: int = 0,
        schwinger_on: int = 0, schwinger_weight: float = 1.0, expect: bool = False):
    """Advance the given particles by nsteps steps of dt.

    particles: {species: (x[n,3], p[n,3], w[n], id[n])}.  Returns
    ({species: (x, p, w, id)}, diagnostics dict, spectrum, spectrum_energy).
    With yee=True the grid fields (list of 6 arrays, modified in place) are
    advanced by one FDTD step after the particles, using the deposited J.
    Steps from index time_from on are timed (diag "timed_seconds" and
    "timed_particle_steps").  With thin_interval > 0 the stores are thinned
    after every step s with (s + 1) % thin_interval == 0 (Sec. VI).  With
    schwinger_on, pairs from the vacuum are created per cell after the
    particles of each step, before the field update (Sec. V.B).  With expect
    (and nbins), diag also holds "expected" and "expected_var": the photon
    spectrum expected along the realised trajectories, and its variance.
    """
    import time
    P = o.make_params(n=n, d=d, x0=x0, periodic=periodic, field_mode=field_mode, fp=fp, kappa=kappa,
                      nsub_max=nsub_max, emission_on=emission_on, pairs_on=pairs_on,
                      same_step_children=same_step_children, deposit_on=deposit_on, seed=seed,
                      lg_lo=lg_lo, lg_hi=lg_hi, ion_charge=ion_charge, ion_mass=ion_mass,
                      ens_bits=ens_bits, ens=ens, emit_fg=emit_fg, emit_ng=emit_ng, pair_fg=pair_fg,
                      pair_ng=pair_ng, thin_interval=thin_interval, thin_limit=thin_limit,
                      generator=generator, schwinger_on=schwinger_on, schwinger_weight=schwinger_weight)
    if caps is None:
        base = sum(len(v[3]) for v in particles.values())
        caps = (4 * base + 64,) * 4
    run_ = o.Run(P, caps=caps, nbins=nbins, expect=expect)
    absorbed_at_set = 0
    for sp, (x, p, w, ids) in particles.items():
        # a particle placed outside an open lattice is removed before any step
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        inside = np.ones(len(x), dtype=bool)
        for c in range(3):
            if not periodic[c]:
                lo, hi = x0[c], x0[c] + d[c] * n[c]
                inside &= (x[:, c] >= lo) & (x[:, c] < hi)
        absorbed_at_set += int((~inside).sum())
        run_.sp[sp].set(x[inside], np.asarray(p).reshape(-1, 3)[inside], np.asarray(w)[inside],
                        np.asarray(ids, dtype=np.uint64)[inside])
    if fields is not None:
        run_.set_grid_fields(fields, J)
    psteps = 0
    timed_ps = 0
    t_start = time.perf_counter()
    for k in range(nsteps):
        if k == time_from:
            t_start = time.perf_counter()
        live = sum(sp.n for sp in run_.sp)
        psteps += live
        if k >= time_from:
            timed_ps += live
        if J is not None:
            for a in J:
                a[:] = 0.0
        run_.step(step0 + k, t0 + k * dt, dt)
        if schwinger_on:
            run_.schwinger(step0 + k, t0 + k * dt, dt)
        if yee:
            o.yee_step(n, d, dt, fields, J)
        if thin_interval > 0 and (step0 + k + 1) % thin_interval == 0:
            run_.thin(step0 + k)
    t_end = time.perf_counter()
    out = {sp: run_.sp[sp].get() for sp in range(4)}
    spec = run_.spectrum[:nbins].copy() if nbins else None
    spec_e = run_.spectrum_energy[:nbins].copy() if nbins else None
    diag = run_.diag()
    diag["absorbed"] += absorbed_at_set
    diag["particle_steps"] = psteps
    diag["timed_particle_steps"] = timed_ps
    diag["timed_seconds"] = t_end - t_start if nsteps > time_from else 0.0
    if expect and nbins:
        diag["expected"] = run_.expected[:nbins].copy()
        diag["expected_var"] = run_.expected_var[:nbins].copy()
    return out, diag, spec, spec_e
