"""Convenience layer over the C ABI: numpy/PyTorch arrays in and out.

Marshalling only; the particle path runs in the CUDA library.  PyTorch
provides device memory and the stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import qed


def _dev(a: np.ndarray, dtype) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


class Simulation:
    """One library context (one GPU, one precision)."""

    def __init__(self, workload, precision: int = 64, capacity=None, emission_on: int = 1,
                 pairs_on: int = 1, same_step_children: int = 1, deposit_on: int = 0, nbins: int = 0,
                 lg_lo: float = -12.0, lg_hi: float = 0.0, nsub_max: int = 1000, kappa=None,
                 compact_interval: int = 0, pending_capacity: int = 0, seed=None, pm_strict: int = 0,
                 ion_charge: float = 1.0, ion_mass: float = 1836.15267343, stream=None, tables=None,
                 thin_interval: int = 0, thin_limit=(0, 0, 0, 0), emit_fg: float = 1.0, emit_ng: int = 1,
                 pair_fg: float = 1.0, pair_ng: int = 1, generator: int = 0, schwinger_on: int = 0,
                 schwinger_weight: float = 1.0):
        w = workload
        self.w = w
        self.prec = precision
        self.nbins = nbins
        g = qed.QedGridDesc()
        g.n[:] = list(w.n)
        g.periodic[:] = list(w.periodic)
        g.d[:] = list(w.d)
        g.x0[:] = list(w.x0)
        g.field_mode = w.field_mode
        g.fp[:] = list(w.fp) + [0.0] * (16 - len(w.fp))
        s = qed.QedSpeciesDesc()
        caps = capacity if capacity is not None else w.capacity
        s.capacity[:] = [int(c) for c in caps]
        s.charge[:] = [-1.0, 1.0, 0.0, ion_charge]
        s.mass[:] = [1.0, 1.0, 0.0, ion_mass]
        p = qed.QedParams()
        p.precision = precision
        p.nsub_max = nsub_max
        p.emission_on = emission_on
        p.pairs_on = pairs_on
        p.same_step_children = same_step_children
        p.deposit_on = deposit_on
        p.pm_strict = pm_strict
        p.seed = w.seed if seed is None else seed
        p.nbins = nbins
        p.compact_interval = compact_interval
        p.kappa = w.kappa if kappa is None else kappa
        p.lg_lo, p.lg_hi = lg_lo, lg_hi
        p.pending_capacity = pending_capacity
        p.ens_bits = int(getattr(w, "ens_bits", 0))
        p.thin_interval = int(thin_interval)
        p.thin_limit[:] = [int(v) for v in thin_limit]
        p.emit_fg, p.pair_fg = float(emit_fg), float(pair_fg)
        p.emit_ng, p.pair_ng = int(emit_ng), int(pair_ng)
        p.generator = int(generator)
        p.schwinger_on = int(schwinger_on)
        p.schwinger_weight = float(schwinger_weight)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = qed.qed_init(g, s, p, tables=tables, stream=self.stream.cuda_stream)
        self.caps = list(s.capacity)
        self.fields = None
        if getattr(w, "ens", None) is not None:
            self.set_ensembles(w.ens)

    # -- particles ------------------------------------------------------------
    def set(self, species: int, x, p, w, ids) -> None:
        n = len(ids)
        if n == 0:
            qed.qed_particles_set(self.ctx, species, 0, 0, 0, 0, 0, self.stream.cuda_stream)
            return
        tx, tp, tw = _dev(x, np.float64), _dev(p, np.float64), _dev(w, np.float64)
        ti = torch.from_numpy(np.ascontiguousarray(ids, dtype=np.uint64).view(np.int64)).cuda()
        qed.qed_particles_set(self.ctx, species, tx.data_ptr(), tp.data_ptr(), tw.data_ptr(), ti.data_ptr(),
                              n, self.stream.cuda_stream)
        self.stream.synchronize()

    def set_all(self) -> None:
        for sp in range(4):
            if sp in self.w.particles:
                self.set(sp, *self.w.particles[sp])

    def get(self, species: int):
        cap = max(self.caps[species], 1)
        x = torch.empty((cap, 3), dtype=torch.float64, device="cuda")
        p = torch.empty((cap, 3), dtype=torch.float64, device="cuda")
        w = torch.empty(cap, dtype=torch.float64, device="cuda")
        i = torch.empty(cap, dtype=torch.int64, device="cuda")
        n = qed.qed_particles_get(self.ctx, species, x.data_ptr(), p.data_ptr(), w.data_ptr(), i.data_ptr(),
                                  cap, self.stream.cuda_stream)
        return (x[:n].cpu().numpy(), p[:n].cpu().numpy(), w[:n].cpu().numpy(),
                i[:n].cpu().numpy().view(np.uint64))

    # -- stepping --------------------------------------------------------------
    def set_grid_fields(self, E, B, J) -> None:
        f = qed.QedFields()
        for k in range(3):
            f.E[k] = E[k].data_ptr()
            f.B[k] = B[k].data_ptr()
            f.J[k] = J[k].data_ptr()
        self.fields = f
        self._field_refs = (E, B, J)

    def step(self, nsteps: int = 1, dt: float | None = None) -> None:
        qed.qed_step(self.ctx, self.fields, self.w.dt if dt is None else dt, nsteps, self.stream.cuda_stream)

    def set_ensembles(self, table) -> None:
        qed.qed_ensembles_set(self.ctx, np.asarray(table, dtype=np.float64), self.stream.cuda_stream)

    def tuning(self) -> dict:
        return qed.qed_get_tuning(self.ctx).as_dict()

    def set_tuning(self, **kw) -> None:
        t = qed.qed_get_tuning(self.ctx)
        for k, v in kw.items():
            setattr(t, k, int(v))
        qed.qed_set_tuning(self.ctx, t)

    def autotune(self, steps_per_trial: int, max_steps: int, dt: float | None = None) -> tuple[dict, int]:
        """Advance by real steps while picking the tuning; returns (tuning, steps taken)."""
        t, n = qed.qed_autotune(self.ctx, self.fields, self.w.dt if dt is None else dt, steps_per_trial,
                                max_steps, self.stream.cuda_stream)
        return t.as_dict(), n

    def set_clock(self, step: int, time: float) -> None:
        qed.qed_set_clock(self.ctx, step, time)

    def diag(self, check: bool = True) -> dict:
        return qed.qed_diagnostics(self.ctx, self.nbins, self.stream.cuda_stream, check=check)

    def close(self) -> None:
        if self.ctx:
            qed.qed_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
