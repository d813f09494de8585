"""Thin ctypes binding of the C ABI declared in ``include/qed.h``.

Argument marshalling only: every step of the particle path runs in the CUDA
library ``_build/libqed_gb300.so``.  There is no fallback; if the library is
missing, ``load()`` raises.  PyTorch is used only for device memory and
streams (``torch.Tensor.data_ptr()``, ``torch.cuda.Stream.cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqed_gb300.so")

QED_OK, QED_ERR_ARG, QED_ERR_CUDA, QED_ERR_CAPACITY, QED_ERR_NONFINITE = 0, 1, 2, 3, 4
QED_ERR_TIMEOUT, QED_ERR_PMGT1, QED_ERR_STATE, QED_ERR_COURANT = 5, 6, 7, 8
QED_ELECTRON, QED_POSITRON, QED_PHOTON, QED_ION = 0, 1, 2, 3
QED_FIELD_GRID, QED_FIELD_UNIFORM, QED_FIELD_GAUSSIAN_LP, QED_FIELD_ROTATING_E, QED_FIELD_ENSEMBLE, QED_FIELD_STANDING_WAVE = (
    0, 1, 2, 3, 4, 5)
QED_ENS_STRIDE = 10
QED_GEN_MODIFIED, QED_GEN_ALTERNATIVE, QED_GEN_STANDARD = 0, 1, 2
QED_MAX_ENS_BITS = 16
# qed_stage: the points of a step at which qed_profile_stages records events
(QED_STAGE_BEGIN, QED_STAGE_CONSTANTS, QED_STAGE_PHOTONS, QED_STAGE_BLOCKS, QED_STAGE_DEPOSIT, QED_STAGE_MASSIVE,
 QED_STAGE_PRODUCTS, QED_STAGE_SCHWINGER, QED_STAGE_FIELD, QED_STAGE_END, QED_NSTAGES) = range(11)

# every entry point the header declares (checked by the CPU tests)
EXPORTS = ("qed_init", "qed_tables_export", "qed_particles_set", "qed_particles_get", "qed_step",
           "qed_set_clock", "qed_profile_events", "qed_diagnostics", "qed_destroy", "qed_error_string",
           "qed_particles_read_static", "qed_ensembles_set", "qed_get_tuning", "qed_set_tuning",
           "qed_autotune", "qed_profile_stages", "qed_selftest_barrier")


class QedGridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("periodic", ctypes.c_int32 * 3),
                ("d", ctypes.c_double * 3), ("x0", ctypes.c_double * 3),
                ("field_mode", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("fp", ctypes.c_double * 16)]


class QedSpeciesDesc(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64 * 4), ("charge", ctypes.c_double * 4),
                ("mass", ctypes.c_double * 4)]


class QedParams(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("nsub_max", ctypes.c_int32),
                ("emission_on", ctypes.c_int32), ("pairs_on", ctypes.c_int32),
                ("same_step_children", ctypes.c_int32), ("deposit_on", ctypes.c_int32),
                ("pm_strict", ctypes.c_int32), ("seed", ctypes.c_uint32),
                ("nbins", ctypes.c_int32), ("compact_interval", ctypes.c_int32),
                ("kappa", ctypes.c_double), ("lg_lo", ctypes.c_double), ("lg_hi", ctypes.c_double),
                ("pending_capacity", ctypes.c_int64),
                ("ens_bits", ctypes.c_int32), ("thin_interval", ctypes.c_int32),
                ("thin_limit", ctypes.c_int64 * 4),
                ("emit_fg", ctypes.c_double), ("pair_fg", ctypes.c_double),
                ("emit_ng", ctypes.c_int32), ("pair_ng", ctypes.c_int32),
                ("generator", ctypes.c_int32), ("reserved_gen", ctypes.c_int32),
                ("schwinger_on", ctypes.c_int32), ("reserved_s", ctypes.c_int32),
                ("schwinger_weight", ctypes.c_double)]


class QedTuning(ctypes.Structure):
    _fields_ = [("photon_blocks_per_sm", ctypes.c_int32), ("massive_blocks_per_sm", ctypes.c_int32),
                ("work_chunk", ctypes.c_int32), ("compact_interval", ctypes.c_int32),
                ("sort_massive", ctypes.c_int32), ("concurrent", ctypes.c_int32),
                ("deposit_halo", ctypes.c_int32), ("refill_lanes", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class QedFields(ctypes.Structure):
    _fields_ = [("E", ctypes.c_void_p * 3), ("B", ctypes.c_void_p * 3), ("J", ctypes.c_void_p * 3)]


class QedDiag(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64 * 4), ("particle_steps", ctypes.c_int64),
                ("species_steps", ctypes.c_int64 * 4)] + [(k, ctypes.c_int64) for k in (
        "emissions", "pairs", "substeps_lepton", "substeps_photon", "pm_gt1",
        "pp_gt1", "capped", "absorbed", "overflow", "nonfinite", "photons_created", "pairs_created",
        "thinned", "schwinger_pairs", "schwinger_gt1", "kernel_launches", "step")] + [
        ("time", ctypes.c_double), ("status", ctypes.c_int32), ("nbins", ctypes.c_int32),
        ("spectrum", ctypes.POINTER(ctypes.c_double)),
        ("spectrum_energy", ctypes.POINTER(ctypes.c_double)), ("block_steps", ctypes.c_int64),
        ("tile_deposits", ctypes.c_int64)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    lib.qed_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(QedGridDesc), ctypes.POINTER(QedSpeciesDesc),
                             vp, ctypes.c_size_t, ctypes.POINTER(QedParams), vp]
    lib.qed_tables_export.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.qed_particles_set.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp, i64, vp]
    lib.qed_particles_get.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp, i64, ctypes.POINTER(i64), vp]
    lib.qed_step.argtypes = [vp, ctypes.POINTER(QedFields), ctypes.c_double, i32, vp]
    lib.qed_particles_read_static.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp, i64, ctypes.POINTER(i64), vp]
    lib.qed_set_clock.argtypes = [vp, i64, ctypes.c_double]
    lib.qed_profile_events.argtypes = [vp, vp, vp, vp]
    lib.qed_profile_stages.argtypes = [vp, ctypes.POINTER(vp), i32]
    lib.qed_selftest_barrier.argtypes = [vp, i32, i64, vp]
    lib.qed_diagnostics.argtypes = [vp, ctypes.POINTER(QedDiag), vp]
    lib.qed_destroy.argtypes = [vp]
    lib.qed_ensembles_set.argtypes = [vp, i32, dp, vp]
    lib.qed_get_tuning.argtypes = [vp, ctypes.POINTER(QedTuning)]
    lib.qed_set_tuning.argtypes = [vp, ctypes.POINTER(QedTuning)]
    lib.qed_autotune.argtypes = [vp, ctypes.POINTER(QedFields), ctypes.c_double, i32, i64, vp,
                                 ctypes.POINTER(QedTuning), ctypes.POINTER(i64)]
    lib.qed_error_string.argtypes = [ctypes.c_int]
    lib.qed_error_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "qed_error_string":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class QedError(RuntimeError):
    def __init__(self, call: str, status: int):
        self.status = status
        super().__init__(f"{call}: {qed_error_string(status)} ({status})")


def _check(call: str, rc: int) -> int:
    if rc != QED_OK:
        raise QedError(call, rc)
    return rc


def qed_error_string(status: int) -> str:
    return load().qed_error_string(int(status)).decode()


def qed_init(grid: QedGridDesc, species: QedSpeciesDesc, params: QedParams, tables: bytes | None = None,
             stream: int = 0) -> int:
    ctx = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(tables, len(tables)) if tables else None
    _check("qed_init", load().qed_init(ctypes.byref(ctx), ctypes.byref(grid), ctypes.byref(species),
                                       ctypes.cast(buf, ctypes.c_void_p) if buf else None,
                                       len(tables) if tables else 0, ctypes.byref(params),
                                       ctypes.c_void_p(stream)))
    return ctx.value


def qed_tables_export(ctx: int) -> bytes:
    need = ctypes.c_size_t()
    _check("qed_tables_export", load().qed_tables_export(ctypes.c_void_p(ctx), None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check("qed_tables_export", load().qed_tables_export(ctypes.c_void_p(ctx), buf, need.value, ctypes.byref(need)))
    return buf.raw


def qed_particles_set(ctx: int, species: int, x_ptr: int, p_ptr: int, w_ptr: int, id_ptr: int, n: int,
                      stream: int = 0) -> None:
    _check("qed_particles_set", load().qed_particles_set(
        ctypes.c_void_p(ctx), int(species), ctypes.c_void_p(x_ptr), ctypes.c_void_p(p_ptr),
        ctypes.c_void_p(w_ptr), ctypes.c_void_p(id_ptr), int(n), ctypes.c_void_p(stream)))


def qed_particles_get(ctx: int, species: int, x_ptr: int, p_ptr: int, w_ptr: int, id_ptr: int, max_n: int,
                      stream: int = 0) -> int:
    n = ctypes.c_int64()
    rc = load().qed_particles_get(ctypes.c_void_p(ctx), int(species), ctypes.c_void_p(x_ptr),
                                  ctypes.c_void_p(p_ptr), ctypes.c_void_p(w_ptr), ctypes.c_void_p(id_ptr),
                                  int(max_n), ctypes.byref(n), ctypes.c_void_p(stream))
    _check("qed_particles_get", rc)
    return n.value


def qed_particles_read_static(ctx: int, species: int, x_ptr: int, p_ptr: int, w_ptr: int, id_ptr: int,
                              max_n: int, stream: int = 0) -> int:
    """Read one species into device or page-locked buffers without allocating."""
    n = ctypes.c_int64()
    rc = load().qed_particles_read_static(ctypes.c_void_p(ctx), int(species), ctypes.c_void_p(x_ptr),
                                          ctypes.c_void_p(p_ptr), ctypes.c_void_p(w_ptr), ctypes.c_void_p(id_ptr),
                                          int(max_n), ctypes.byref(n), ctypes.c_void_p(stream))
    _check("qed_particles_read_static", rc)
    return n.value


def qed_step(ctx: int, fields: QedFields | None, dt: float, nsteps: int = 1, stream: int = 0) -> None:
    _check("qed_step", load().qed_step(ctypes.c_void_p(ctx), ctypes.byref(fields) if fields else None,
                                       float(dt), int(nsteps), ctypes.c_void_p(stream)))


def qed_set_clock(ctx: int, step: int, time: float) -> None:
    _check("qed_set_clock", load().qed_set_clock(ctypes.c_void_p(ctx), int(step), float(time)))


def qed_profile_events(ctx: int, start_event: int, photon_event: int, stop_event: int) -> None:
    _check("qed_profile_events", load().qed_profile_events(ctypes.c_void_p(ctx), ctypes.c_void_p(start_event),
                                                           ctypes.c_void_p(photon_event),
                                                           ctypes.c_void_p(stop_event)))


def qed_profile_stages(ctx: int, events) -> None:
    """events: raw cudaEvent_t handles (ints or 0), entry k for stage k, or
    m blocks of QED_NSTAGES for steps 0..m-1 of each following call; []
    stops recording."""
    arr = (ctypes.c_void_p * max(len(events), 1))(*[ctypes.c_void_p(e or None) for e in events])
    _check("qed_profile_stages", load().qed_profile_stages(ctypes.c_void_p(ctx), arr, len(events)))


def qed_selftest_barrier(ctx: int, absent_block: int, spin_limit: int, stream: int = 0) -> int:
    """Run the bounded grid barrier with block absent_block (-1: none) never
    arriving; returns the status (QED_OK or QED_ERR_TIMEOUT) without raising."""
    return load().qed_selftest_barrier(ctypes.c_void_p(ctx), int(absent_block), int(spin_limit), ctypes.c_void_p(stream))


def qed_diagnostics(ctx: int, nbins: int = 0, stream: int = 0, check: bool = True) -> dict:
    d = QedDiag()
    spec = np.zeros(max(nbins, 1))
    spec_e = np.zeros(max(nbins, 1))
    d.nbins = nbins
    if nbins:
        d.spectrum = spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.spectrum_energy = spec_e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = load().qed_diagnostics(ctypes.c_void_p(ctx), ctypes.byref(d), ctypes.c_void_p(stream))
    if check:
        _check("qed_diagnostics", rc)
    out = {k: getattr(d, k) for k, _ in QedDiag._fields_[3:21]}
    out["count"] = list(d.count)
    out["particle_steps"] = d.particle_steps
    out["species_steps"] = list(d.species_steps)
    out["time"] = d.time
    out["status"] = d.status
    out["block_steps"] = d.block_steps
    out["tile_deposits"] = d.tile_deposits
    if nbins:
        out["spectrum"] = spec[:nbins].copy()
        out["spectrum_energy"] = spec_e[:nbins].copy()
    return out


def qed_ensembles_set(ctx: int, table: np.ndarray, stream: int = 0) -> None:
    """table: (n_ens, QED_ENS_STRIDE) rows {E0, omega, phase, Eu[3], Bu[3], thin_scale} (host, copied)."""
    tab = np.ascontiguousarray(table, dtype=np.float64).reshape(-1, QED_ENS_STRIDE)
    _check("qed_ensembles_set", load().qed_ensembles_set(ctypes.c_void_p(ctx), len(tab),
                                                         ctypes.c_void_p(tab.ctypes.data),
                                                         ctypes.c_void_p(stream)))


def qed_get_tuning(ctx: int) -> QedTuning:
    t = QedTuning()
    _check("qed_get_tuning", load().qed_get_tuning(ctypes.c_void_p(ctx), ctypes.byref(t)))
    return t


def qed_set_tuning(ctx: int, tuning: QedTuning) -> None:
    _check("qed_set_tuning", load().qed_set_tuning(ctypes.c_void_p(ctx), ctypes.byref(tuning)))


def qed_autotune(ctx: int, fields: QedFields | None, dt: float, steps_per_trial: int, max_steps: int,
                 stream: int = 0) -> tuple[QedTuning, int]:
    t = QedTuning()
    taken = ctypes.c_int64()
    _check("qed_autotune", load().qed_autotune(ctypes.c_void_p(ctx), ctypes.byref(fields) if fields else None,
                                               float(dt), int(steps_per_trial), int(max_steps),
                                               ctypes.c_void_p(stream), ctypes.byref(t), ctypes.byref(taken)))
    return t, taken.value


def qed_destroy(ctx: int) -> None:
    if ctx:
        load().qed_destroy(ctypes.c_void_p(ctx))
