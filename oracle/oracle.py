"""ctypes wrapper of the FP64 CPU oracle (``qed_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product library never imports it.  It shares no code with the CUDA path.

The oracle works in Compton units (momentum m c, time hbar/mc^2, length
hbar/mc, fields E_S) and keeps particles at absolute FP64 positions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qed_oracle.c")
LIB = os.path.join(HERE, "libqed_oracle.so")

ELECTRON, POSITRON, PHOTON, ION = 0, 1, 2, 3
FIELD_GRID, FIELD_UNIFORM, FIELD_GAUSSIAN_LP, FIELD_ROTATING_E, FIELD_ENSEMBLE, FIELD_STANDING_WAVE = 0, 1, 2, 3, 4, 5
PURPOSE_EMIT, PURPOSE_PAIR, PURPOSE_CHILD, PURPOSE_KEEP, PURPOSE_THIN = 1, 2, 3, 4, 5
ENS_STRIDE = 10  # per ensemble: E0, omega, phase, Eu[3], Bu[3], thin_scale
GEN_MODIFIED, GEN_ALTERNATIVE, GEN_STANDARD = 0, 1, 2


def compile_library(src: str, out: str) -> None:
    """Compile one copy of the oracle's C source into a shared library."""
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", out, src, "-lm"])


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        compile_library(SRC, LIB + ".tmp")
        os.replace(LIB + ".tmp", LIB)
    return LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("periodic", ctypes.c_int32 * 3),
        ("field_mode", ctypes.c_int32),
        ("nsub_max", ctypes.c_int32),
        ("emission_on", ctypes.c_int32),
        ("pairs_on", ctypes.c_int32),
        ("same_step_children", ctypes.c_int32),
        ("deposit_on", ctypes.c_int32),
        ("seed", ctypes.c_uint32),
        ("nbins", ctypes.c_int32),
        ("d", ctypes.c_double * 3),
        ("x0", ctypes.c_double * 3),
        ("kappa", ctypes.c_double),
        ("lg_lo", ctypes.c_double),
        ("lg_hi", ctypes.c_double),
        ("charge", ctypes.c_double * 4),
        ("mass", ctypes.c_double * 4),
        ("fp", ctypes.c_double * 16),
        ("ens_bits", ctypes.c_int32),
        ("n_ens", ctypes.c_int32),
        ("ens", ctypes.POINTER(ctypes.c_double)),
        ("emit_fg", ctypes.c_double),
        ("pair_fg", ctypes.c_double),
        ("emit_ng", ctypes.c_int32),
        ("pair_ng", ctypes.c_int32),
        ("thin_interval", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("thin_limit", ctypes.c_int64 * 4),
        ("generator", ctypes.c_int32),
        ("reserved2", ctypes.c_int32),
        ("schwinger_on", ctypes.c_int32),
        ("reserved3", ctypes.c_int32),
        ("schwinger_weight", ctypes.c_double),
    ]


class Store(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cap", ctypes.c_int64)] + [
        (k, ctypes.POINTER(ctypes.c_double)) for k in ("x", "y", "z", "px", "py", "pz", "w")
    ] + [("id", ctypes.POINTER(ctypes.c_uint64))]


class Diag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "emissions", "pairs", "substeps_lepton", "substeps_photon", "pm_gt1", "pp_gt1",
        "capped", "absorbed", "overflow", "nonfinite", "photons_created", "pairs_created",
        "thinned", "schwinger_pairs", "schwinger_gt1")] + [
        ("energy_defect", ctypes.c_double),
        ("spectrum", ctypes.POINTER(ctypes.c_double)),
        ("spectrum_energy", ctypes.POINTER(ctypes.c_double)),
        ("expected", ctypes.POINTER(ctypes.c_double)),
        ("expected_var", ctypes.POINTER(ctypes.c_double))]


_lib = None


def lib():
    """The loaded oracle library.  QED_ORACLE_LIB names another build of the
    same source to load instead (the planted-mistake tests use it)."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(os.environ.get("QED_ORACLE_LIB") or build())
        d, i64, u32, u64, i32 = (ctypes.c_double, ctypes.c_int64, ctypes.c_uint32,
                                 ctypes.c_uint64, ctypes.c_int32)
        pd = ctypes.POINTER(d)
        for name in ("or_F1", "or_F2"):
            getattr(_lib, name).restype = d
            getattr(_lib, name).argtypes = [d]
        _lib.or_synchrotron.argtypes = [d, pd, pd]
        _lib.or_G.restype = d; _lib.or_G.argtypes = [d, d]
        _lib.or_P.restype = d; _lib.or_P.argtypes = [d, d, d, d]
        _lib.or_Pm.restype = d; _lib.or_Pm.argtypes = [d, d, d, d]
        _lib.or_Pp.restype = d; _lib.or_Pp.argtypes = [d, d, d, d]
        for name in ("or_chi", "or_heff", "or_heff_photon", "or_chi_photon"):
            getattr(_lib, name).restype = d
            getattr(_lib, name).argtypes = [pd, pd, pd]
        _lib.or_dtq_lepton.restype = d; _lib.or_dtq_lepton.argtypes = [d, d, d]
        _lib.or_dtq_photon.restype = d; _lib.or_dtq_photon.argtypes = [d, d]
        _lib.or_nsub.restype = ctypes.c_int; _lib.or_nsub.argtypes = [d, d, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        _lib.or_boris.argtypes = [pd, pd, pd, d, d, d]
        _lib.or_field.argtypes = [ctypes.c_int, pd, pd, d, pd, pd]
        _lib.or_u52.restype = d; _lib.or_u52.argtypes = [u32, u32]
        _lib.or_philox4x32_10.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
        _lib.or_draw.argtypes = [u64, u32, u32, u32, u32, pd, pd]
        _lib.or_child_id.restype = u64; _lib.or_child_id.argtypes = [u64, u32, u32, u32, u32]
        _lib.or_step.restype = ctypes.c_int
        _lib.or_step.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Store), ctypes.POINTER(Diag),
                                 ctypes.POINTER(pd), ctypes.POINTER(pd), u32, d, d]
        _lib.or_schwinger.restype = ctypes.c_int
        _lib.or_schwinger.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Store), ctypes.POINTER(Diag),
                                      ctypes.POINTER(pd), u32, d, d]
        _lib.or_Wnorm.restype = d; _lib.or_Wnorm.argtypes = [d, d]
        _lib.or_gauss_legendre8.argtypes = [pd, pd]
        _lib.or_Pstd.restype = d; _lib.or_Pstd.argtypes = [d, d, d]
        _lib.or_delta_std.restype = d; _lib.or_delta_std.argtypes = [d, d]
        _lib.or_sample_frozen_gen.restype = i64
        _lib.or_sample_frozen_gen.argtypes = [i32, d, d, d, i64, u32, d, d, i32, pd, ctypes.POINTER(i64)]
        _lib.or_field_ensemble.argtypes = [ctypes.POINTER(Params), u64, d, pd, pd]
        _lib.or_thin.restype = ctypes.c_int
        _lib.or_thin.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Store), ctypes.POINTER(Diag), u32]
        _lib.or_sample_frozen.restype = i64
        _lib.or_sample_frozen.argtypes = [d, d, d, i64, u32, d, d, i32, pd, ctypes.POINTER(i64)]
        _lib.or_philox_block.argtypes = [u64, u32, u32, u32, u32, i64, ctypes.POINTER(u32)]
        _lib.or_yee_step.restype = ctypes.c_int
        _lib.or_yee_step.argtypes = [ctypes.POINTER(i32), pd, d, ctypes.POINTER(pd), ctypes.POINTER(pd)]
        _lib.or_gather.argtypes = [ctypes.POINTER(i32), pd, pd, ctypes.POINTER(pd), pd, pd, pd]
        _lib.or_deposit.argtypes = [ctypes.POINTER(i32), pd, pd, ctypes.POINTER(pd), pd, pd, d, d]
        _lib.or_charge_density.argtypes = [ctypes.POINTER(i32), pd, pd, pd, pd, pd, pd, pd, i64]
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _v3(v):
    return (ctypes.c_double * 3)(*[float(a) for a in v])


# ---- scalar physics ------------------------------------------------------

def F1(x: float) -> float:
    return lib().or_F1(float(x))


def F2(x: float) -> float:
    return lib().or_F2(float(x))


def G(delta, chi):
    return lib().or_G(float(delta), float(chi))


def P(delta, chi, gamma, dt):
    return lib().or_P(float(delta), float(chi), float(gamma), float(dt))


def Pm(r1, chi, gamma, dt):
    return lib().or_Pm(float(r1), float(chi), float(gamma), float(dt))


def Pp(de, chig, eps, dt):
    return lib().or_Pp(float(de), float(chig), float(eps), float(dt))


def chi(p, E, B):
    return lib().or_chi(_v3(p), _v3(E), _v3(B))


def heff(p, E, B):
    return lib().or_heff(_v3(p), _v3(E), _v3(B))


def chi_photon(k, E, B):
    return lib().or_chi_photon(_v3(k), _v3(E), _v3(B))


def heff_photon(k, E, B):
    return lib().or_heff_photon(_v3(k), _v3(E), _v3(B))


def dtq_lepton(gamma, heff_, kappa):
    return lib().or_dtq_lepton(float(gamma), float(heff_), float(kappa))


def dtq_photon(heff_g, kappa):
    return lib().or_dtq_photon(float(heff_g), float(kappa))


def nsub(t_span, dtq, nmax):
    c = ctypes.c_int(0)
    n = lib().or_nsub(float(t_span), float(dtq), int(nmax), ctypes.byref(c))
    return n, bool(c.value)


def boris(p, E, B, q, m, h):
    pp = _v3(p)
    lib().or_boris(pp, _v3(E), _v3(B), float(q), float(m), float(h))
    return np.array(pp[:])


def field(mode, fp, x, t):
    fpa = (ctypes.c_double * 16)(*(list(fp) + [0.0] * (16 - len(fp))))
    E, B = _v3((0, 0, 0)), _v3((0, 0, 0))
    lib().or_field(int(mode), fpa, _v3(x), float(t), E, B)
    return np.array(E[:]), np.array(B[:])


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def philox_block(pid, step, sub0, purpose, seed, n):
    out = np.zeros((n, 4), dtype=np.uint32)
    lib().or_philox_block(pid, step, sub0, purpose, seed, n,
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def u52(a, b):
    return lib().or_u52(a, b)


def draw(pid, step, sub, purpose, seed):
    r1, r2 = ctypes.c_double(), ctypes.c_double()
    lib().or_draw(pid, step, sub, purpose, seed, ctypes.byref(r1), ctypes.byref(r2))
    return r1.value, r2.value


def child_id(parent, step, sub, kind, seed):
    return lib().or_child_id(parent, step, sub, kind, seed)


def sample_frozen(chi_, gamma, h, ndraw, seed, lo, hi, nbins):
    hist = np.zeros(nbins)
    viol = ctypes.c_int64(0)
    acc = lib().or_sample_frozen(float(chi_), float(gamma), float(h), int(ndraw), int(seed),
                                 float(lo), float(hi), int(nbins), _dp(hist), ctypes.byref(viol))
    return acc, hist, viol.value


def sample_frozen_gen(generator, chi_, gamma, h, ndraw, seed, lo, hi, nbins):
    hist = np.zeros(nbins)
    viol = ctypes.c_int64(0)
    acc = lib().or_sample_frozen_gen(int(generator), float(chi_), float(gamma), float(h), int(ndraw), int(seed),
                                     float(lo), float(hi), int(nbins), _dp(hist), ctypes.byref(viol))
    return acc, hist, viol.value


def gauss_legendre8():
    """The 8-point Gauss-Legendre nodes and weights on [-1, 1] that W is
    integrated with."""
    x, w = np.zeros(8), np.zeros(8)
    lib().or_gauss_legendre8(_dp(x), _dp(w))
    return x, w


def Wnorm(x, chi_):
    return lib().or_Wnorm(float(x), float(chi_))


def Pstd(chi_, gamma, dt):
    return lib().or_Pstd(float(chi_), float(gamma), float(dt))


def delta_std(chi_, r2):
    return lib().or_delta_std(float(chi_), float(r2))


# ---- Yee mesh, gather, deposit -------------------------------------------

def yee_step(n, d, dt, f, J):
    """f: list of 6 arrays (Ex..Bz), J: list of 3 arrays; modified in place."""
    n3 = (ctypes.c_int32 * 3)(*n)
    fp = (ctypes.POINTER(ctypes.c_double) * 6)(*[_dp(a) for a in f])
    jp = (ctypes.POINTER(ctypes.c_double) * 3)(*[_dp(a) for a in J])
    if lib().or_yee_step(n3, _v3(d), float(dt), fp, jp) != 0:
        raise MemoryError("or_yee_step")


def gather(n, d, x0, f, x):
    n3 = (ctypes.c_int32 * 3)(*n)
    fp = (ctypes.POINTER(ctypes.c_double) * 6)(*[_dp(a) for a in f])
    E, B = _v3((0, 0, 0)), _v3((0, 0, 0))
    lib().or_gather(n3, _v3(d), _v3(x0), fp, _v3(x), E, B)
    return np.array(E[:]), np.array(B[:])


def deposit(n, d, x0, J, xa, xb, qw, dt):
    n3 = (ctypes.c_int32 * 3)(*n)
    jp = (ctypes.POINTER(ctypes.c_double) * 3)(*[_dp(a) for a in J])
    lib().or_deposit(n3, _v3(d), _v3(x0), jp, _v3(xa), _v3(xb), float(qw), float(dt))


def charge_density(n, d, x0, x, y, z, qw):
    rho = np.zeros(int(np.prod(n)))
    n3 = (ctypes.c_int32 * 3)(*n)
    x, y, z, qw = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, qw))
    lib().or_charge_density(n3, _v3(d), _v3(x0), _dp(rho), _dp(x), _dp(y), _dp(z), _dp(qw), len(x))
    return rho


# ---- the particle step ---------------------------------------------------

class Species:
    """Numpy-backed store of one species (absolute FP64 positions)."""

    def __init__(self, cap: int):
        self.cap = int(cap)
        self.a = {k: np.zeros(self.cap) for k in ("x", "y", "z", "px", "py", "pz", "w")}
        self.a["id"] = np.zeros(self.cap, dtype=np.uint64)
        self.n = 0

    def set(self, x, p, w, ids):
        n = len(ids)
        if n > self.cap:
            raise ValueError("capacity")
        x = np.asarray(x, dtype=np.float64).reshape(n, 3)
        p = np.asarray(p, dtype=np.float64).reshape(n, 3)
        for c, k in enumerate("xyz"):
            self.a[k][:n] = x[:, c]
            self.a["p" + k][:n] = p[:, c]
        self.a["w"][:n] = w
        self.a["id"][:n] = ids
        self.n = n

    def get(self):
        n = self.n
        x = np.stack([self.a[k][:n] for k in "xyz"], axis=1).copy()
        p = np.stack([self.a["p" + k][:n] for k in "xyz"], axis=1).copy()
        return x, p, self.a["w"][:n].copy(), self.a["id"][:n].copy()

    def cstore(self) -> Store:
        s = Store()
        s.n, s.cap = self.n, self.cap
        for k in ("x", "y", "z", "px", "py", "pz", "w"):
            setattr(s, k, _dp(self.a[k]))
        s.id = self.a["id"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        return s


class Run:
    """One oracle simulation: four species stores, parameters, diagnostics."""

    def __init__(self, params: Params, caps, nbins: int = 0, expect: bool = False):
        self.P = params
        self.P.nbins = nbins
        self.sp = [Species(c) for c in caps]
        self.spectrum = np.zeros(max(nbins, 1))
        self.spectrum_energy = np.zeros(max(nbins, 1))
        self.D = Diag()
        self.D.spectrum = _dp(self.spectrum)
        self.D.spectrum_energy = _dp(self.spectrum_energy)
        # the expected spectrum along the realised trajectories (and its variance)
        self.expected = np.zeros(max(nbins, 1))
        self.expected_var = np.zeros(max(nbins, 1))
        if expect:
            self.D.expected = _dp(self.expected)
            self.D.expected_var = _dp(self.expected_var)
        self.fields = None
        self.J = None

    def set_grid_fields(self, f, J):
        self.fields = f
        self.J = J

    def step(self, step: int, t: float, dt: float):
        stores = (Store * 4)(*[s.cstore() for s in self.sp])
        fp = jp = None
        if self.fields is not None:
            fp = (ctypes.POINTER(ctypes.c_double) * 6)(*[_dp(a) for a in self.fields])
        if self.J is not None:
            jp = (ctypes.POINTER(ctypes.c_double) * 3)(*[_dp(a) for a in self.J])
        rc = lib().or_step(ctypes.byref(self.P), stores, ctypes.byref(self.D), fp, jp,
                           int(step), float(t), float(dt))
        if rc != 0:
            raise MemoryError("or_step")
        for s, c in zip(self.sp, stores):
            s.n = int(c.n)

    def schwinger(self, step: int, t: float, dt: float):
        stores = (Store * 4)(*[s.cstore() for s in self.sp])
        fp = None
        if self.fields is not None:
            fp = (ctypes.POINTER(ctypes.c_double) * 6)(*[_dp(a) for a in self.fields])
        lib().or_schwinger(ctypes.byref(self.P), stores, ctypes.byref(self.D), fp, int(step), float(t), float(dt))
        for s, c in zip(self.sp, stores):
            s.n = int(c.n)

    def thin(self, step: int):
        stores = (Store * 4)(*[s.cstore() for s in self.sp])
        if lib().or_thin(ctypes.byref(self.P), stores, ctypes.byref(self.D), int(step)) != 0:
            raise MemoryError("or_thin")
        for s, c in zip(self.sp, stores):
            s.n = int(c.n)

    def diag(self) -> dict:
        return {k: getattr(self.D, k) for k, _ in Diag._fields_[:16]}


def make_params(*, n=(1, 1, 1), d=(1.0, 1.0, 1.0), x0=(0.0, 0.0, 0.0), periodic=(0, 0, 0),
                field_mode=FIELD_UNIFORM, fp=(), kappa=0.1, nsub_max=1000, emission_on=1,
                pairs_on=1, same_step_children=1, deposit_on=0, seed=1, lg_lo=-12.0,
                lg_hi=0.0, ion_charge=1.0, ion_mass=1836.15267343, ens_bits=0, ens=None,
                emit_fg=1.0, emit_ng=1, pair_fg=1.0, pair_ng=1, thin_interval=0,
                thin_limit=(0, 0, 0, 0), generator=0, schwinger_on=0, schwinger_weight=1.0) -> Params:
    """Oracle parameters.  ens: (n_ens, ENS_STRIDE) float64 table of the
    ensemble fields (field_mode FIELD_ENSEMBLE); the returned Params keeps a
    reference to it."""
    P = Params()
    P.n[:] = list(n)
    P.periodic[:] = list(periodic)
    P.field_mode = field_mode
    P.nsub_max = nsub_max
    P.emission_on = emission_on
    P.pairs_on = pairs_on
    P.same_step_children = same_step_children
    P.deposit_on = deposit_on
    P.seed = seed
    P.d[:] = list(d)
    P.x0[:] = list(x0)
    P.kappa = kappa
    P.lg_lo, P.lg_hi = lg_lo, lg_hi
    P.charge[:] = [-1.0, 1.0, 0.0, ion_charge]
    P.mass[:] = [1.0, 1.0, 0.0, ion_mass]
    fpl = list(fp) + [0.0] * (16 - len(fp))
    P.fp[:] = fpl
    P.ens_bits = int(ens_bits)
    if ens is not None:
        tab = np.ascontiguousarray(ens, dtype=np.float64).reshape(-1, ENS_STRIDE)
        P._ens_keep = tab
        P.n_ens = len(tab)
        P.ens = _dp(tab)
    P.emit_fg, P.pair_fg = float(emit_fg), float(pair_fg)
    P.emit_ng, P.pair_ng = int(emit_ng), int(pair_ng)
    P.thin_interval = int(thin_interval)
    P.thin_limit[:] = [int(v) for v in thin_limit]
    P.generator = int(generator)
    P.schwinger_on = int(schwinger_on)
    P.schwinger_weight = float(schwinger_weight)
    return P


def field_ensemble(P: Params, pid: int, t: float):
    E = np.zeros(3)
    B = np.zeros(3)
    lib().or_field_ensemble(ctypes.byref(P), int(pid), float(t), _dp(E), _dp(B))
    return E, B
