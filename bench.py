"""Throughput of the QED particle step: particle-steps/s with QED events.

Workload (default, --workload cascade512): the large self-consistent 3D
cascade -- a 512^3 periodic Yee mesh (dx = lambda/32, lambda = 0.8 um,
dt = T_L/64), four circularly polarised plane-wave pulses at 2e24 W/cm^2
(two along x, two along y), a cold hydrogen slab of 1e22 cm^-3, 0.5 um
thick, with 8 macro-electrons and 8 macro-protons per cell (4.2e7 each),
photon emission and Breit-Wheeler pairs, Esirkepov deposit, FDTD update,
thinning every 8 steps.  A window of K steps starting at step 40 is timed
(W warm-up steps right before it), each step bracketed by CUDA events on its
stream; the stages of every timed step (photon pass, cell-block pass,
deposit, FDTD, ...) are recorded on the same stream (qed_profile_stages),
and the roofline object is for the stage that takes the most time.  The
FP64 form runs side by side over the same window.  The mesh alone (4.8 GB in
FP32) is far larger than L2.

One bench step = one qed_step (every live particle of every species advanced
by dt, then the field update).  Prints one JSON line on rank 0.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload instead (a 32^3 box of the same recipe, one core).

--workload collision times the head-on collision of a 1 GeV electron beam
(1e6 electrons, 1% energy spread, 1 um rms radius, 3 um rms length) with a
counter-propagating linearly polarised Gaussian pulse (lambda = 0.8 um,
a0 = 200, 30 fs FWHM, 2 um waist), test particles in the analytic field,
dt = T_laser/100, 600 steps: W warm-up steps and K timed steps in a window
centred on the collision, a 256 MiB buffer written between timed steps to
flush L2.

--workload batched times the batched-ensemble workload: 512 independent
test-particle instances in uniform rotating E fields (chi log-uniform in
[0.1, 100], electron counts log-uniform in [1e3, 1e6]), with per-ensemble
thinning, 500 steps of dt = T_laser/100 in FP32; the first steps run under
the autotuner, the rest are replays of a CUDA graph.

--workload cascade times the self-consistent 256^3 cascade (2000 steps).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RUN_STEPS = 600
N_ELECTRONS = 1_000_000
TUNING: dict = {}          # qed_tuning fields applied to the collision runs (--tuning)
GENERATOR = 0              # photon-emission generator: 0 modified, 1 alternative, 2 standard
CAPS = (1_300_000, 200_000, 60_000_000, 0)
COMPACT_INTERVAL = 32       # measured: 8 -> 4.21e10, 16 -> 4.52e10, 32 -> 4.65e10 particle-steps/s
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes per particle-step (read cell + offset + p + w + id, write
# cell + offset + p) and per appended particle record, FP32 / FP64 forms
BYTES_PER_STEP = {32: 68, 64: 120}
BYTES_PER_APPEND = {32: 40, 64: 68}
# DRAM bytes (read + write) per photon-step of the photon kernel, from one ncu
# capture of k_photons at the collision step (step 300) of the 2.5e5-electron
# beam: (dram__bytes_read.sum + dram__bytes_write.sum) / live photons.  The
# kernel's traffic is proportional to the records it touches, so the bench
# scales it by the photons of its own launches.  Remove an entry when the
# kernel changes until it is measured again.  (Empty: the FP32 photon kernel
# changed, photon norms by the reciprocal square root, after its last
# capture, 247.68e6 / 5.567e6 = 44.5 B per photon-step.)
PHOTON_DRAM_BYTES_PER_STEP: dict = {}
METRIC = "particle-steps/s with QED events, FP32 vs FP64 GPU path; % of HBM roofline"
WORKLOAD_NAME = ("beam-laser head-on collision: 1e6 e- at 1 GeV (1% spread, 1 um x 3 um rms), "
                 "LP Gaussian pulse lambda=0.8 um a0=200 30 fs FWHM w0=2 um, analytic field, "
                 "emission + Breit-Wheeler pairs, dt=T_L/100, 600 steps")


def window(K: int, W: int) -> int:
    """First step of the warm-up + timed window, centred on the collision."""
    meet = RUN_STEPS // 2
    return max(0, min(RUN_STEPS - K - W, meet - (K + W) // 2))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
def make_workload(seed: int):
    from paper_1412_6426_gb300 import workloads
    return workloads.beam_laser_collision(n_particles=N_ELECTRONS, seed=seed, nsteps=RUN_STEPS)


def rank_seed(rank: int) -> int:
    """Weak scaling: rank r runs its own workload, drawn with seed 1 + r."""
    return 1 + rank


def combine_ranks(items):
    """[(value, "sum" | "max"), ...] -> the values summed or maximised over
    the ranks of the current process group (one rank, or none: unchanged).
    The only collective of a run: the data path has none."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return [float(v) for v, _ in items]
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    out = []
    for v, op in items:
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.SUM if op == "sum" else tdist.ReduceOp.MAX)
        out.append(float(t.item()))
    return out


def scale_workload(n_electrons: int) -> None:
    """Shrink the beam (and capacities) for profiling captures."""
    global N_ELECTRONS, CAPS
    f = n_electrons / N_ELECTRONS
    N_ELECTRONS = n_electrons
    CAPS = tuple(int(c * f) + (1024 if c else 0) for c in CAPS)


def time_device(w, prec: int, K: int, W: int, dist_barrier) -> dict:
    """K timed steps of the device-resident path (inputs already in HBM)."""
    import torch
    from paper_1412_6426_gb300 import qed
    from paper_1412_6426_gb300.sim import Simulation

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    s0 = window(K, W)
    with Simulation(w, precision=prec, capacity=CAPS, compact_interval=COMPACT_INTERVAL,
                    generator=GENERATOR) as sim:
        sim.set_all()
        if TUNING:
            sim.set_tuning(**TUNING)
        if s0:
            sim.step(s0)                      # untimed: advance to the window
        sim.step(W)                           # warm-up steps
        d0 = sim.diag()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        kev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(K)]
        for trio in kev:                      # materialise the events before the library records them
            for e_ in trio:
                e_.record(stream)
        torch.cuda.synchronize()
        dist_barrier()
        sampler = ClockSampler(int(os.environ.get("BENCH_GPU_INDEX", torch.cuda.current_device())))
        torch.cuda.synchronize()
        for k in range(K):
            flush.zero_()                     # L2 flush, outside the timed events
            qed.qed_profile_events(sim.ctx, kev[k][0].cuda_event, kev[k][1].cuda_event, kev[k][2].cuda_event)
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        dist_barrier()
        qed.qed_profile_events(sim.ctx, 0, 0, 0)
        d1 = sim.diag()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(c) for a, _, c in kev]
    phot_ms = [a.elapsed_time(b) for a, b, _ in kev]
    psteps = d1["particle_steps"] - d0["particle_steps"]
    photon_steps = d1["species_steps"][2] - d0["species_steps"][2]
    appended = (d1["emissions"] - d0["emissions"]) + 2 * (d1["pairs"] - d0["pairs"])
    algo_bytes = BYTES_PER_STEP[prec] * psteps + BYTES_PER_APPEND[prec] * appended
    return {"precision": prec, "window_start": s0, "particle_steps": psteps, "seconds": sum(step_ms) / 1e3,
            "kernel_seconds": sum(kern_ms) / 1e3, "ms_per_step": sum(step_ms) / K, "algo_bytes": algo_bytes,
            "photon_seconds": sum(phot_ms) / 1e3, "photon_steps": photon_steps,
            "photon_algo_bytes": BYTES_PER_STEP[prec] * photon_steps,
            "emissions": d1["emissions"] - d0["emissions"], "pairs": d1["pairs"] - d0["pairs"],
            "launches": d1["kernel_launches"] - d0["kernel_launches"], "live_end": d1["count"],
            "substeps": (d1["substeps_lepton"] - d0["substeps_lepton"])
                        + (d1["substeps_photon"] - d0["substeps_photon"]),
            "clocks": clocks}


def time_e2e(w, prec: int, K: int, W: int) -> dict:
    """The same steps through the public API with host buffers: each step
    copies every species in from pinned host memory (qed_particles_set),
    advances it (qed_step) and copies it back out (qed_particles_get)."""
    import numpy as np
    import torch
    from paper_1412_6426_gb300 import qed
    from paper_1412_6426_gb300.sim import Simulation

    stream = torch.cuda.current_stream()
    s0 = window(K, W)
    host = {}
    for sp in range(3):
        cap = CAPS[sp]
        host[sp] = (torch.empty((cap, 3), dtype=torch.float64, pin_memory=True),
                    torch.empty((cap, 3), dtype=torch.float64, pin_memory=True),
                    torch.empty(cap, dtype=torch.float64, pin_memory=True),
                    torch.empty(cap, dtype=torch.int64, pin_memory=True))
    n = {sp: 0 for sp in range(3)}
    with Simulation(w, precision=prec, capacity=CAPS, compact_interval=COMPACT_INTERVAL) as sim:
        sim.set_all()
        if s0 + W:
            sim.step(s0 + W)

        def get_all():
            for sp in range(3):
                x, p, wt, i = host[sp]
                n[sp] = qed.qed_particles_get(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(),
                                              i.data_ptr(), CAPS[sp], stream.cuda_stream)

        get_all()
        torch.cuda.synchronize()
        h2d = d2h = 0
        psteps = 0
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(K):
            for sp in range(3):
                x, p, wt, i = host[sp]
                qed.qed_particles_set(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(), i.data_ptr(),
                                      n[sp], stream.cuda_stream)
                h2d += 64 * n[sp]
                psteps += n[sp]
            sim.step(1)
            get_all()                          # synchronises: the step's result is on the host
            d2h += 64 * sum(n.values())
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    secs = e0.elapsed_time(e1) / 1e3
    return {"value": psteps / secs, "seconds": secs, "wall_seconds": wall, "particle_steps": psteps,
            "h2d_bytes_per_step": h2d // K, "d2h_bytes_per_step": d2h // K}


# ----------------------------------------------------------------------------
# the FP64 CPU oracle on a bounded sample of the same workload
def _oracle_worker(args):
    (x, p, w, ids, wl_fields, W, K) = args
    from oracle import drive
    n, d, x0, periodic, field_mode, fp, dt, kappa, seed = wl_fields
    out, diag, _, _ = drive.run(n, d, x0, periodic, field_mode, fp, dt, W + K, {0: (x, p, w, ids)},
                                kappa=kappa, seed=seed, caps=(len(ids) * 3 + 64, 4096 + len(ids), 80 * len(ids) + 4096, 1),
                                time_from=W)
    return diag["timed_particle_steps"], diag["timed_seconds"], diag["overflow"]


def oracle_sample(K: int, W: int, per_worker: int, workers: int) -> dict:
    """Time the oracle on the first workers*per_worker electrons of the same
    beam (same seed, same run) over the same step window, one process per
    host core used."""
    w = make_workload(seed=1)
    s0 = window(K, W)
    x, p, wt, ids = w.particles[0]
    fields = (w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt, w.kappa, w.seed)
    jobs = []
    for k in range(workers):
        sl = slice(k * per_worker, (k + 1) * per_worker)
        jobs.append((x[sl].copy(), p[sl].copy(), wt[sl].copy(), ids[sl].copy(), fields, s0 + W, K))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    ps = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    return {"value": ps / secs, "unit": "particle-steps/s", "cores": workers, "kind": "oracle",
            "sample": (f"{workers * per_worker} of the 1e6 electrons (same beam, same seed) and all their "
                       f"products, steps {s0 + W}..{s0 + W + K - 1} of the 600-step run, FP64 oracle, "
                       f"{workers} processes x {per_worker} electrons"),
            "particle_steps": ps, "seconds": secs, "wall_seconds": wall,
            "overflow": sum(r[2] for r in res)}


def cpu_workers() -> int:
    return max(1, min(os.cpu_count() or 1, 32))


# ----------------------------------------------------------------------------
# batched ensembles
BATCH_STEPS = 500
BATCH_TUNE_MAX = 96
BATCH_NAME = ("batched ensembles: 512 independent test-particle instances in uniform rotating E (drift-free "
              "circular orbits), chi log-uniform in [0.1, 100], e- counts log-uniform in [1e3, 1e6] (seed 1), "
              "emission + Breit-Wheeler pairs, per-ensemble thinning every 4 steps (e-, e+ to N_e, photons to "
              "2 N_e), dt=T_L/100, 500 steps")


BATCH_SCALE = 1.0     # electron counts x this (profiling captures only)
BATCH_AUTOTUNE = True


def make_batched(seed: int):
    from paper_1412_6426_gb300 import workloads
    return workloads.batched_ensembles(seed=seed, nsteps=BATCH_STEPS,
                                       count_range=(1e3 * BATCH_SCALE, 1e6 * BATCH_SCALE))


def batched_device(w, prec: int, K: int, W: int, dist_barrier) -> dict:
    """Autotune on the first steps, then replay a captured CUDA graph of G
    steps; W warm-up steps (whole replays) and then up to K timed steps."""
    import torch
    from paper_1412_6426_gb300 import qed
    from paper_1412_6426_gb300.sim import Simulation

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = Simulation(w, precision=prec, capacity=w.capacity, compact_interval=4, stream=stream,
                         thin_interval=w.meta["thin_interval"], thin_limit=w.meta["thin_limit"])
        try:
            sim.set_all()
            if BATCH_AUTOTUNE:
                tuned, n_tune = sim.autotune(2, BATCH_TUNE_MAX)
            else:
                tuned, n_tune = sim.tuning(), 0
            sim.set_tuning(**tuned)                 # restarts the compaction phase
            ci = tuned["compact_interval"]
            G = math.lcm(w.meta["thin_interval"], 2 * ci)
            left = BATCH_STEPS - n_tune
            n_warm = max(1, -(-W // G))
            n_timed = max(1, min(K // G, left // G - n_warm))
            torch.cuda.synchronize()
            l0 = sim.diag()["kernel_launches"]
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                qed.qed_step(sim.ctx, None, w.dt, G, stream.cuda_stream)
            # minus the live-count kernels of the first diagnostics call (one per species store)
            per_replay = sim.diag()["kernel_launches"] - l0 - sum(1 for c in w.capacity if c > 0)
            for _ in range(n_warm):
                graph.replay()
            torch.cuda.synchronize()
            d0 = sim.diag()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(n_timed)]
            dist_barrier()
            sampler = ClockSampler(int(os.environ.get("BENCH_GPU_INDEX", torch.cuda.current_device())))
            torch.cuda.synchronize()
            for k in range(n_timed):
                ev[k][0].record(stream)
                graph.replay()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            clocks = sampler.stop()
            dist_barrier()
            d1 = sim.diag()
            del graph
        finally:
            sim.close()
    rep_ms = [a.elapsed_time(b) for a, b in ev]
    psteps = d1["particle_steps"] - d0["particle_steps"]
    made = (d1["photons_created"] - d0["photons_created"]) + 2 * (d1["pairs_created"] - d0["pairs_created"])
    lepton_steps = sum(d1["species_steps"][k] - d0["species_steps"][k] for k in (0, 1))
    return {"precision": prec, "particle_steps": psteps, "seconds": sum(rep_ms) / 1e3,
            "steps": n_timed * G, "warmup": n_tune + n_warm * G, "graph_steps": G, "replays": n_timed,
            "ms_per_step": sum(rep_ms) / (n_timed * G), "tuning": tuned, "tune_steps": n_tune,
            "algo_bytes": BYTES_PER_STEP[prec] * psteps + BYTES_PER_APPEND[prec] * made,
            "launches": per_replay * n_timed,
            "emissions": d1["emissions"] - d0["emissions"], "pairs": d1["pairs"] - d0["pairs"],
            "thinned": d1["thinned"] - d0["thinned"], "live_end": d1["count"],
            "substeps_per_lepton_step": (d1["substeps_lepton"] - d0["substeps_lepton"]) / max(lepton_steps, 1),
            "clocks": clocks, "step_end": d1["step"]}


def batched_e2e(w, prec: int, n_steps: int) -> dict:
    """n_steps through the public API with pinned host buffers, right after
    the thinning that ends step 8: per step every species is copied in
    (qed_particles_set), advanced (qed_step) and copied out
    (qed_particles_get).  The host buffers hold 3x (photons) and 2x
    (leptons) the live particles at the start, which bounds two steps of
    growth."""
    import torch
    from paper_1412_6426_gb300 import qed
    from paper_1412_6426_gb300.sim import Simulation

    stream = torch.cuda.current_stream()
    with Simulation(w, precision=prec, capacity=w.capacity, compact_interval=4,
                    thin_interval=w.meta["thin_interval"], thin_limit=w.meta["thin_limit"]) as sim:
        sim.set_all()
        sim.step(8)
        live = sim.diag()["count"]
        host, n = {}, {}
        for sp in range(3):
            cap = max(1, int(live[sp] * (3.0 if sp == 2 else 2.0)) + 4096)
            host[sp] = (torch.empty((cap, 3), dtype=torch.float64, pin_memory=True),
                        torch.empty((cap, 3), dtype=torch.float64, pin_memory=True),
                        torch.empty(cap, dtype=torch.float64, pin_memory=True),
                        torch.empty(cap, dtype=torch.int64, pin_memory=True))

        def get_all():
            for sp in range(3):
                x, p, wt, i = host[sp]
                n[sp] = qed.qed_particles_get(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(),
                                              i.data_ptr(), len(wt), stream.cuda_stream)

        get_all()
        torch.cuda.synchronize()
        h2d = d2h = psteps = 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_steps):
            for sp in range(3):
                x, p, wt, i = host[sp]
                qed.qed_particles_set(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(), i.data_ptr(),
                                      n[sp], stream.cuda_stream)
                h2d += 64 * n[sp]
                psteps += n[sp]
            sim.step(1)
            get_all()
            d2h += 64 * sum(n.values())
        e1.record(stream)
        torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    return {"value": psteps / secs, "particle_steps": psteps, "seconds": secs,
            "h2d_bytes_per_step": h2d // n_steps, "d2h_bytes_per_step": d2h // n_steps}


def _batched_oracle_worker(args):
    (parts, fields, nsteps) = args
    from oracle import drive
    n, d, x0, periodic, dt, kappa, seed, ens, bits, thin_interval, thin_limit = fields
    base = len(parts[0][3])
    out, diag, _, _ = drive.run(n, d, x0, periodic, 4, (), dt, nsteps, parts, kappa=kappa, seed=seed,
                                caps=(60 * base + 4096, 60 * base + 4096, 200 * base + 4096, 1),
                                ens=ens, ens_bits=bits, thin_interval=thin_interval, thin_limit=thin_limit)
    return diag["timed_particle_steps"], diag["timed_seconds"], diag["overflow"]


def batched_oracle_sample(nsteps: int, workers: int) -> dict:
    """The oracle on whole ensembles (thinning couples the particles of an
    ensemble): the smallest ensembles of the same workload, one per process,
    over its first nsteps steps."""
    import numpy as np
    w = make_batched(seed=1)
    counts = w.meta["counts"]
    order = np.argsort(counts)[:workers]
    x, p, wt, ids = w.particles[0]
    ens_of = (ids >> np.uint64(64 - w.ens_bits)).astype(np.int64)
    fields = (w.n, w.d, w.x0, w.periodic, w.dt, w.kappa, w.seed, w.ens, w.ens_bits,
              w.meta["thin_interval"], w.meta["thin_limit"])
    jobs = []
    for e in order:
        m = ens_of == e
        jobs.append(({0: (x[m], p[m], wt[m], ids[m])}, fields, nsteps))
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(jobs)) as pool:
        res = pool.map(_batched_oracle_worker, jobs)
    ps = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    return {"value": ps / secs, "unit": "particle-steps/s", "cores": len(jobs), "kind": "oracle",
            "sample": (f"the {len(jobs)} smallest of the 512 ensembles ({int(counts[order].sum())} seed electrons "
                       f"and all their products, with their thinning), steps 0..{nsteps - 1}, FP64 oracle, "
                       f"one process per ensemble"),
            "overflow": sum(r[2] for r in res)}


# ----------------------------------------------------------------------------
# the self-consistent cascade on the 256^3 Yee mesh
CASCADE_STEPS = 2000
CASCADE_CAPS = (30_000_000, 30_000_000, 1_200_000_000, 0)
CASCADE_NAME = ("self-consistent 3D QED cascade: 256^3 periodic Yee mesh, dx = lambda/32 (lambda = 0.8 um), "
                "dt = T_L/64, two counter-propagating CP plane-wave pulses at 1e24 W/cm^2 (sin^2 envelope, "
                "2 lambda FWHM), seed 1e5 e- + 1e5 e+ cold in a 1 um cube, Esirkepov deposit + FDTD, "
                "emission + Breit-Wheeler pairs, 2000 steps")


def cascade_run(K: int, W: int, dist_barrier, e2e_at: int = 1200, e2e_steps: int = 2) -> dict:
    """The 2000-step cascade: W warm-up steps, then K timed steps (each with
    CUDA events on the stream; the fields alone, 600 MB, exceed L2).  The
    step kernels are bracketed separately (qed_profile_events)."""
    import numpy as np
    import torch
    from paper_1412_6426_gb300 import qed, workloads
    from paper_1412_6426_gb300.sim import Simulation

    w, f = workloads.self_consistent_cascade(nsteps=CASCADE_STEPS)
    nc = len(f[0])
    E = [torch.from_numpy(a).cuda() for a in f[:3]]
    B = [torch.from_numpy(a).cuda() for a in f[3:]]
    J = [torch.zeros(nc, dtype=torch.float32, device="cuda") for _ in range(3)]
    stream = torch.cuda.current_stream()
    K = min(K, CASCADE_STEPS - W)
    with Simulation(w, precision=32, capacity=CASCADE_CAPS, deposit_on=1, compact_interval=8) as sim:
        sim.set_grid_fields(E, B, J)
        sim.set_all()
        sim.step(W)
        d0 = sim.diag()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        kev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(K)]
        for trio in kev:
            for e_ in trio:
                e_.record(stream)
        torch.cuda.synchronize()
        dist_barrier()
        sampler = ClockSampler(int(os.environ.get("BENCH_GPU_INDEX", torch.cuda.current_device())))
        for k in range(K):
            qed.qed_profile_events(sim.ctx, kev[k][0].cuda_event, kev[k][1].cuda_event, kev[k][2].cuda_event)
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        dist_barrier()
        qed.qed_profile_events(sim.ctx, 0, 0, 0)
        d1 = sim.diag()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(c) for a, _, c in kev]
    psteps = d1["particle_steps"] - d0["particle_steps"]
    appended = (d1["photons_created"] - d0["photons_created"]) + 2 * (d1["pairs_created"] - d0["pairs_created"])
    out = {"particle_steps": psteps, "seconds": sum(step_ms) / 1e3, "kernel_seconds": sum(kern_ms) / 1e3,
           "ms_per_step": sum(step_ms) / K, "steps": K, "ncell": nc, "appended": appended,
           "launches": d1["kernel_launches"] - d0["kernel_launches"], "live_end": d1["count"],
           "emissions": d1["emissions"] - d0["emissions"], "pairs": d1["pairs"] - d0["pairs"], "clocks": clocks,
           "last_ms": step_ms[-50:]}
    # end to end through the C ABI with host buffers, a few steps into the cascade
    out["e2e"] = None
    if e2e_steps:
        w2, f2 = workloads.self_consistent_cascade(nsteps=CASCADE_STEPS)
        E2 = [torch.from_numpy(a).cuda() for a in f2[:3]]
        B2 = [torch.from_numpy(a).cuda() for a in f2[3:]]
        J2 = [torch.zeros(nc, dtype=torch.float32, device="cuda") for _ in range(3)]
        with Simulation(w2, precision=32, capacity=CASCADE_CAPS, deposit_on=1, compact_interval=8) as sim:
            sim.set_grid_fields(E2, B2, J2)
            sim.set_all()
            sim.step(e2e_at)
            live = sim.diag()["count"]
            host, n = {}, {}
            for sp in range(3):
                cap = max(1, int(live[sp] * 1.5) + 4096)
                host[sp] = tuple(torch.empty(sh, dtype=dt_, pin_memory=True) for sh, dt_ in
                                 (((cap, 3), torch.float64), ((cap, 3), torch.float64), ((cap,), torch.float64),
                                  ((cap,), torch.int64)))
            def get_all():
                for sp in range(3):
                    x, p, wt, i = host[sp]
                    n[sp] = qed.qed_particles_get(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(),
                                                  i.data_ptr(), len(wt), stream.cuda_stream)
            get_all()
            torch.cuda.synchronize()
            h2d = d2h = ps = 0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(e2e_steps):
                for sp in range(3):
                    x, p, wt, i = host[sp]
                    qed.qed_particles_set(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(), i.data_ptr(),
                                          n[sp], stream.cuda_stream)
                    h2d += 64 * n[sp]
                    ps += n[sp]
                sim.step(1)
                get_all()
                d2h += 64 * sum(n.values())
            e1.record(stream)
            torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        out["e2e"] = {"value": ps / secs, "unit": "particle-steps/s", "h2d_bytes_per_step": h2d // e2e_steps,
                      "d2h_bytes_per_step": d2h // e2e_steps, "steps": e2e_steps, "at_step": e2e_at}
    return out


def cascade_oracle_sample(nsteps: int) -> dict:
    """The oracle on the same cascade, one core (the particles share the
    mesh), over its first nsteps steps: all 2e5 seeds and the full 256^3
    Yee mesh."""
    import numpy as np
    from oracle import drive
    from paper_1412_6426_gb300 import workloads
    w, f = workloads.self_consistent_cascade(nsteps=CASCADE_STEPS, precision=64)
    fo = [a.astype(np.float64) for a in f]
    Jo = [np.zeros_like(fo[0]) for _ in range(3)]
    n0 = w.n_initial()
    t0 = time.perf_counter()
    _, diag, _, _ = drive.run(w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt, nsteps, w.particles,
                              kappa=w.kappa, seed=w.seed, caps=(4 * n0, 4 * n0, 40 * n0, 1), fields=fo, J=Jo,
                              deposit_on=1, yee=True)
    secs = time.perf_counter() - t0
    return {"value": diag["particle_steps"] / secs, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": (f"steps 0..{nsteps - 1} of the cascade (all 2e5 seeds and their products, the full 256^3 "
                       f"Yee mesh with deposit and field update), FP64 oracle, one process (the particles share "
                       f"the mesh)")}


def cascade_profile_window(start: int, count: int, caps) -> None:
    """For profiling captures: run the cascade to step `start`, then `count`
    steps inside a CUDA profiler range (ncu --profile-from-start off)."""
    import torch
    from paper_1412_6426_gb300 import workloads
    from paper_1412_6426_gb300.sim import Simulation
    w, f = workloads.self_consistent_cascade(nsteps=CASCADE_STEPS)
    nc = len(f[0])
    E = [torch.from_numpy(a).cuda() for a in f[:3]]
    B = [torch.from_numpy(a).cuda() for a in f[3:]]
    J = [torch.zeros(nc, dtype=torch.float32, device="cuda") for _ in range(3)]
    with Simulation(w, precision=32, capacity=caps, deposit_on=1, compact_interval=8) as sim:
        sim.set_grid_fields(E, B, J)
        sim.set_all()
        sim.step(start)
        torch.cuda.synchronize()
        live0 = sim.diag()["count"]
        torch.cuda.profiler.start()
        sim.step(count)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        d = sim.diag()
    print(json.dumps({"profile_window": [start, count], "live_before": live0, "live_after": d["count"],
                      "status": d["status"]}))


def main_cascade(args, world, rank, local):
    import torch
    import torch.distributed as tdist
    from paper_1412_6426_gb300 import build
    if args.profile_window:
        build.build()
        torch.cuda.set_device(local)
        a, b = (int(v) for v in args.profile_window.split(":"))
        caps = tuple(int(float(v)) for v in args.cascade_caps.split(",")) + (0,) if args.cascade_caps \
            else CASCADE_CAPS
        cascade_profile_window(a, b, caps)
        return

    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            tdist.barrier()

    build.build()
    W = args.warmup
    K = CASCADE_STEPS - W if args.steps == RUN_STEPS - 3 else args.steps
    r = cascade_run(K, W, barrier, e2e_steps=0 if args.no_e2e else 2)
    tot, mx = combine_ranks([(r["particle_steps"], "sum"), (r["seconds"], "max")])
    if rank != 0:
        if world > 1:
            tdist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    # algorithmic bytes: particles (68 B per particle-step, 40 B per append)
    # and the mesh (FDTD: 9 reads + 6 writes of 4 B per cell-step; J zeroed
    # and accumulated: 12 + 12 B per cell-step)
    algo = 68 * r["particle_steps"] + 40 * r["appended"] + (60 + 24) * r["ncell"] * r["steps"]
    ach = algo / r["seconds"] / 1e9
    line = {"metric": METRIC, "value": tot / mx, "unit": "particle-steps/s", "n_gpus": world, "steps": r["steps"],
            "warmup": W, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": CASCADE_NAME, "precision": "fp32 fields, particles, push/rates; fp64 tables",
                       "parallelism": f"independent boxes x{world}",
                       "l2": "fields alone 600 MB, larger than L2 (no flush)", "compact_and_sort_interval": 8},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": None, "peak_source": peak_kind,
                         "kernel": "whole step (all kernels: particles, deposit, FDTD, sort)",
                         "algorithmic_bytes_per_step": algo / r["steps"]},
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "events": {"emissions": r["emissions"], "pairs": r["pairs"], "live_at_end": r["live_end"],
                       "step_kernels_ms_per_step": r["kernel_seconds"] * 1e3 / r["steps"],
                       "last_steps_ms": round(sum(r["last_ms"]) / len(r["last_ms"]), 3)}}
    if r["e2e"] is not None:
        line["e2e"] = r["e2e"]
    if not args.no_cpu:
        cb = cascade_oracle_sample(6)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()


LARGE_NAME = ("large self-consistent 3D QED cascade: 512^3 periodic Yee mesh, dx = lambda/32 (lambda = 0.8 um), "
              "dt = T_L/64, four CP plane-wave pulses at 2e24 W/cm^2 (two along x, two along y; sin^2 envelope "
              "of half the box), hydrogen slab 1e22 cm^-3, 0.5 um thick, 8 ppc e- and p+ (4.2e7 each), "
              "Esirkepov deposit + FDTD, emission + Breit-Wheeler pairs, thinning every 8 steps")
LARGE_START, LARGE_STEPS = 40, 20   # the timed window starts at step 40 (W warm-ups right before it)
# The stages of a step (qed_profile_stages) and the kernels each one holds.
STAGES = ("constants", "photons", "blocks", "deposit", "massive", "products", "schwinger", "field", "end")
STAGE_KERNELS = {"constants": "J and count resets, k_grid_max (first step of a call), k_step_constants", "photons": "k_photons",
                 "blocks": "k_blocks (e-/e+, then ions)", "deposit": "k_deposit_blocks", "massive": "k_pass0",
                 "products": "k_products", "schwinger": "k_schwinger", "field": "k_yee_b, k_yee_e",
                 "end": "thinning, compaction and cell-block sort"}
# Algorithmic bytes per unit of each stage, FP32 / FP64:
#  photons, blocks, massive: the particle step, 68 / 120 B per particle-step
#    (read cell, offsets, p, w, id; write cell, offsets, p);
#  deposit: the start point and the end record of each particle the cell-block
#    pass advanced, 16 + 32 = 48 / 96 B (the current tiles are flushed once);
#  field: the Yee update, 9 reads + 6 writes a cell, 60 / 120 B per cell-step;
#  constants: J zeroed (3 values), 12 / 24 B per cell-step (the mesh maxima
#    are read off the fields at the first step of a qed_step call only; the
#    field update forms them for the steps after it).
STAGE_BYTES = {"photons": (68, 120), "blocks": (68, 120), "massive": (68, 120), "deposit": (48, 96),
               "field": (60, 120), "constants": (12, 24)}
# DRAM bytes (read + write) per unit of a kernel from one ncu capture of that
# kernel on the large-cascade recipe; the bench scales them by the units of
# its own launches.  Remove an entry when the kernel changes until it is
# measured again.
# "blocks" (k_blocks, e-/e+ and ions): 489.5 MB read + written over 5.289e6
# particle-steps at step 40 of the same recipe on a 128^3 mesh; "deposit"
# (k_deposit_blocks and k_deposit_drift): 298.1 MB over the same particle-steps.
LARGE_DRAM_BYTES_PER_UNIT: dict = {("blocks", 32): 489.50e6 / 5.289e6, ("deposit", 32): 298.08e6 / 5.289e6}


def large_setup(precision: int, n: int = 512):
    import torch
    from paper_1412_6426_gb300 import workloads
    w, fx, fy = workloads.large_cascade(n=n)
    dt_ = torch.float32 if precision == 32 else torch.float64
    F = workloads.expand_profiles(fx, fy, n, xp=torch, dtype=dt_, device="cuda")
    J = [torch.zeros(n ** 3, dtype=dt_, device="cuda") for _ in range(3)]
    opts = dict(precision=precision, capacity=w.meta["capacity%d" % precision], deposit_on=1,
                compact_interval=8, thin_interval=w.meta["thin_interval"], thin_limit=w.meta["thin_limit"],
                pending_capacity=50_000_000)
    return w, F, J, opts


def large_device(precision: int, K: int, W: int, dist_barrier, start: int = LARGE_START) -> dict:
    """Advance the 512^3 cascade to step max(start, W) - W untimed, take W
    warm-up steps, then K steps in one qed_step call bracketed by CUDA events
    on the stream (the mesh alone, 4.8 GB in FP32, exceeds L2), with the
    stages of every timed step recorded by qed_profile_stages on the same
    stream (one block of events per step of the call)."""
    import torch
    from paper_1412_6426_gb300 import qed
    from paper_1412_6426_gb300.sim import Simulation
    w, F, J, opts = large_setup(precision)
    stream = torch.cuda.current_stream()
    s0 = max(start, W)
    with Simulation(w, **opts) as sim:
        sim.set_grid_fields(F[:3], F[3:], J)
        sim.set_all()
        if TUNING:
            sim.set_tuning(**TUNING)
        tuning = sim.tuning()
        if s0 - W:
            sim.step(s0 - W)
        sim.step(W)
        d0 = sim.diag()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        sev = [[torch.cuda.Event(enable_timing=True) for _ in range(qed.QED_NSTAGES)] for _ in range(K)]
        for row in sev:                       # materialise the events before the library records them
            for e_ in row:
                e_.record(stream)
        qed.qed_profile_stages(sim.ctx, [e_.cuda_event for row in sev for e_ in row] if K > 1
                               else [e_.cuda_event for e_ in sev[0]])
        torch.cuda.synchronize()
        dist_barrier()
        sampler = ClockSampler(int(os.environ.get("BENCH_GPU_INDEX", torch.cuda.current_device())))
        ev[0].record(stream)
        sim.step(K)
        ev[1].record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        dist_barrier()
        qed.qed_profile_stages(sim.ctx, [])
        d1 = sim.diag()
    total_ms = ev[0].elapsed_time(ev[1])
    step_ms = [sev[k][0].elapsed_time(sev[k][-1]) for k in range(K)]
    stage_ms = {name: sum(sev[k][j].elapsed_time(sev[k][j + 1]) for k in range(K)) / K
                for j, name in enumerate(STAGES)}
    psteps = d1["particle_steps"] - d0["particle_steps"]
    sp = [d1["species_steps"][i] - d0["species_steps"][i] for i in range(4)]
    blk = d1["block_steps"] - d0["block_steps"]
    appended = (d1["photons_created"] - d0["photons_created"]) + 2 * (d1["pairs_created"] - d0["pairs_created"])
    ncell = w.n[0] * w.n[1] * w.n[2]
    units = {"photons": sp[2], "blocks": blk, "deposit": blk, "massive": sp[0] + sp[1] + sp[3] - blk,
             "field": ncell * K, "constants": ncell * K}
    pi = 0 if precision == 32 else 1
    r = 4 if precision == 32 else 8
    # particles (68 / 120 B per particle-step, 40 / 68 B per append) and the mesh
    # (FDTD: 9 reads + 6 writes a cell-step; J zeroed and accumulated: 3 + 3)
    algo = (BYTES_PER_STEP[precision] * psteps + BYTES_PER_APPEND[precision] * appended
            + 21 * r * ncell * K)
    return {"particle_steps": psteps, "seconds": total_ms / 1e3, "ms_per_step": total_ms / K,
            "step_ms_min_max": [min(step_ms), max(step_ms)],
            "steps": K, "warmup": W, "window": [s0, s0 + K], "appended": appended, "algo_bytes": algo,
            "clocks": clocks, "stage_ms": stage_ms, "stage_units": units,
            "stage_bytes": {k: STAGE_BYTES[k][pi] for k in STAGE_BYTES},
            "launches": d1["kernel_launches"] - d0["kernel_launches"], "live_end": d1["count"],
            "emissions": d1["emissions"] - d0["emissions"], "pairs": d1["pairs"] - d0["pairs"],
            "substeps_lepton": d1["substeps_lepton"] - d0["substeps_lepton"],
            "thinned": d1["thinned"] - d0["thinned"], "precision": precision, "tuning": tuning,
            "tile_fraction": (d1["tile_deposits"] - d0["tile_deposits"]) / blk if blk else None}


def dominant_roofline(rr: dict, peak: float, peak_kind: str) -> dict:
    """The roofline of the kernel that takes the most time per step (among the
    stages with a byte model): algorithmic bytes per launch over its own
    launch time, measured by the stage events on its stream."""
    K = rr["steps"]
    name = max(STAGE_BYTES, key=lambda k: rr["stage_ms"][k])
    ms = rr["stage_ms"][name]
    units = rr["stage_units"][name] / K
    per = rr["stage_bytes"][name]
    ach = per * units / (ms * 1e-3) / 1e9
    dram = LARGE_DRAM_BYTES_PER_UNIT.get((name, rr["precision"]))
    traffic = dram * units if dram else None
    out = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "traffic": traffic, "peak_source": peak_kind, "kernel": STAGE_KERNELS[name], "stage": name,
           "kernel_ms_per_launch": ms, "algorithmic_bytes_per_launch": per * units, "units_per_launch": units,
           "bytes_per_unit": per,
           "share_of_step": ms / rr["ms_per_step"]}
    if traffic:
        out["frac_traffic"] = traffic / (ms * 1e-3) / 1e9 / peak
    return out


def large_e2e(at: int = 1, steps: int = 3) -> dict:
    """Steps at..at+steps-1 through the C ABI with page-locked host buffers:
    before each step every species' records are copied in, after it they
    are read back (the next step starts from what was read); the copies
    cross the host link, whose rate varies, so several steps are timed."""
    import torch
    from paper_1412_6426_gb300 import qed
    from paper_1412_6426_gb300.sim import Simulation
    w, F, J, opts = large_setup(32)
    stream = torch.cuda.current_stream()
    with Simulation(w, **opts) as sim:
        sim.set_grid_fields(F[:3], F[3:], J)
        sim.set_all()
        sim.step(at)
        live = sim.diag()["count"]
        host, n = {}, {}
        for sp in range(4):
            # early in the run the photons grow by millions a step
            cap = int(live[sp] * 1.3) + (30_000_000 if sp == 2 else 1_000_000) * steps
            host[sp] = tuple(torch.empty(sh, dtype=dt_, pin_memory=True) for sh, dt_ in
                             (((cap, 3), torch.float64), ((cap, 3), torch.float64), ((cap,), torch.float64),
                              ((cap,), torch.int64)))

        def get_all():
            for sp in range(4):
                x, p, wt, i = host[sp]
                n[sp] = qed.qed_particles_get(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(),
                                              i.data_ptr(), len(wt), stream.cuda_stream)
        get_all()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h2d = d2h = ps = 0
        for _ in range(steps):
            for sp in range(4):
                x, p, wt, i = host[sp]
                qed.qed_particles_set(sim.ctx, sp, x.data_ptr(), p.data_ptr(), wt.data_ptr(), i.data_ptr(),
                                      n[sp], stream.cuda_stream)
                h2d += 64 * n[sp]
                ps += n[sp]
            sim.step(1)
            get_all()
            d2h += 64 * sum(n.values())
        e1.record(stream)
        torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    return {"value": ps / secs, "unit": "particle-steps/s", "h2d_bytes_per_step": h2d // steps,
            "d2h_bytes_per_step": d2h // steps, "steps": steps, "at_step": at}


def large_oracle_sample(nsteps: int = 1, n: int = 64, time_from: int = 0) -> dict:
    """The oracle on an n^3 box of the same recipe (box n/32 lambda, the same
    density, ppc, intensity and thinning), one core, over its first nsteps
    steps (those from index time_from on timed)."""
    import numpy as np
    from oracle import drive
    from paper_1412_6426_gb300 import workloads
    w, fx, fy = workloads.large_cascade(n=n)
    fo = [np.array(a, dtype=np.float64) for a in workloads.expand_profiles(fx, fy, n)]
    Jo = [np.zeros_like(fo[0]) for _ in range(3)]
    _, diag, _, _ = drive.run(w.n, w.d, w.x0, w.periodic, w.field_mode, w.fp, w.dt, nsteps, w.particles,
                              kappa=w.kappa, seed=w.seed, caps=w.meta["capacity64"], fields=fo, J=Jo,
                              deposit_on=1, yee=True, thin_interval=w.meta["thin_interval"],
                              thin_limit=w.meta["thin_limit"], time_from=time_from)
    secs = diag["timed_seconds"]
    ne = len(w.particles[workloads.ELECTRON][3])
    return {"value": diag["timed_particle_steps"] / secs, "unit": "particle-steps/s", "cores": 1,
            "kind": "oracle", "seconds": secs, "steps": nsteps - time_from,
            "sample": (f"steps {time_from}..{nsteps - 1} of the same recipe on a {n}^3 box ({n / 32:g} lambda; "
                       f"{ne:.2g} e- and as many p+ at the start), FP64 oracle with deposit and field update, "
                       f"one process (the particles share the mesh)")}


def large_profile_window(start: int, count: int, n: int = 512, caps=None) -> None:
    """For profiling captures: run the large cascade (FP32; n^3 mesh, the
    same recipe) to step `start`, then `count` steps inside a CUDA profiler
    range (ncu --profile-from-start off)."""
    import torch
    from paper_1412_6426_gb300.sim import Simulation
    w, F, J, opts = large_setup(32, n)
    if caps is not None:
        opts["capacity"] = caps
        opts["pending_capacity"] = 0
    with Simulation(w, **opts) as sim:
        sim.set_grid_fields(F[:3], F[3:], J)
        sim.set_all()
        sim.step(start)
        torch.cuda.synchronize()
        live0 = sim.diag()["count"]
        torch.cuda.profiler.start()
        sim.step(count)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        d = sim.diag()
    print(json.dumps({"profile_window": [start, count], "live_before": live0, "live_after": d["count"],
                      "status": d["status"]}))


def workloads_target(n: int) -> int:
    """Protons of the large cascade's target on an n^3 mesh."""
    from paper_1412_6426_gb300 import workloads
    return len(workloads.large_cascade(n=n)[0].particles[workloads.ION][3])


def main_large(args, world, rank, local):
    import torch
    import torch.distributed as tdist
    from paper_1412_6426_gb300 import build
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            tdist.barrier()

    build.build()
    if args.profile_window:
        a, b = (int(v) for v in args.profile_window.split(":"))
        caps = None
        if args.cascade_caps:
            caps = tuple(int(float(v)) for v in args.cascade_caps.split(","))
            caps = caps + (workloads_target(args.box),)
        large_profile_window(a, b, args.box, caps)
        return
    K, W = args.steps, args.warmup
    r = large_device(32, K, W, barrier)
    r64 = None if args.no_fp64 else large_device(64, max(2, K // 4), W, barrier)
    e2e = None if args.no_e2e else large_e2e()
    tot, mx = combine_ranks([(r["particle_steps"], "sum"), (r["seconds"], "max")])
    if rank != 0:
        if world > 1:
            tdist.destroy_process_group()
        return
    peak, peak_kind = peaks()

    def roof_step(rr):
        ach = rr["algo_bytes"] / rr["seconds"] / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": peak_kind,
                "kernel": "whole step (all kernels: particles, deposit, FDTD, thinning, sort)",
                "algorithmic_bytes_per_step": rr["algo_bytes"] / rr["steps"]}

    def stages(rr):
        return {k: round(v, 4) for k, v in rr["stage_ms"].items()}

    line = {"metric": METRIC, "value": tot / mx, "unit": "particle-steps/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": LARGE_NAME, "precision": "fp32 fields, particles, push/rates; fp64 tables",
                       "parallelism": f"independent boxes x{world}",
                       "l2": "the mesh alone, 4.8 GB, is larger than L2 (no flush)",
                       "compact_and_sort_interval": 8, "window": r["window"], "tuning": r["tuning"]},
            "roofline": dominant_roofline(r, peak, peak_kind), "roofline_step": roof_step(r),
            "stages_ms_per_step": stages(r), "gpu_launches": r["launches"], "clocks": r["clocks"],
            "events": {"emissions": r["emissions"], "pairs": r["pairs"], "thinned": r["thinned"],
                       "live_at_end": r["live_end"], "deposits_through_tiles": r["tile_fraction"],
                       "lepton_substeps_per_step": r["substeps_lepton"] / K}}
    if r64 is not None:
        v64 = r64["particle_steps"] / r64["seconds"]
        line["fp64"] = {"value": v64, "ms_per_step": r64["ms_per_step"], "steps": r64["steps"],
                        "window": r64["window"], "roofline": dominant_roofline(r64, peak, peak_kind),
                        "roofline_step": roof_step(r64), "stages_ms_per_step": stages(r64),
                        "speedup_fp32_over_fp64": line["value"] / v64, "live_at_end": r64["live_end"],
                        "clocks": r64["clocks"]}
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu:
        cb = large_oracle_sample(1)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()


def main_batched(args, world, rank, local):
    import torch
    import torch.distributed as tdist
    from paper_1412_6426_gb300 import build

    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            tdist.barrier()

    build.build()
    w = make_batched(seed=rank_seed(rank))    # weak scaling: each rank its own 512 ensembles
    r = batched_device(w, 32, args.steps, args.warmup, barrier)
    r64 = None if args.no_fp64 else batched_device(w, 64, args.steps, args.warmup, barrier)
    e2e = None if args.no_e2e else batched_e2e(w, 32, 2)
    tot, mx = combine_ranks([(r["particle_steps"], "sum"), (r["seconds"], "max")])
    if rank != 0:
        if world > 1:
            tdist.destroy_process_group()
        return
    value = tot / mx
    peak, peak_kind = peaks()

    def roof(rr):
        ach = rr["algo_bytes"] / rr["seconds"] / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": None, "peak_source": peak_kind,
                "kernel": "whole step (graph replay: step kernels, thinning, compaction, sort)",
                "algorithmic_bytes_per_step": rr["algo_bytes"] / rr["steps"],
                "bytes_per_unit": BYTES_PER_STEP[rr["precision"]]}

    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": r["steps"], "warmup": r["warmup"], "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": BATCH_NAME, "precision": "fp32 push/rates, fp64 tables",
                       "parallelism": f"independent ensemble sets x{world}",
                       "l2": "working set of several GB, larger than L2 (no flush)",
                       "graph_steps": r["graph_steps"], "timed_replays": r["replays"],
                       "autotune_steps": r["tune_steps"], "tuning": r["tuning"],
                       "steps_taken": r["step_end"]},
            "roofline": roof(r), "gpu_launches": r["launches"], "clocks": r["clocks"],
            "events": {"emissions": r["emissions"], "pairs": r["pairs"], "thinned": r["thinned"],
                       "substeps_per_lepton_step": r["substeps_per_lepton_step"],
                       "live_at_end": r["live_end"]}}
    if r64 is not None:
        line["fp64"] = {"value": r64["particle_steps"] / r64["seconds"], "ms_per_step": r64["ms_per_step"],
                        "roofline": roof(r64), "tuning": r64["tuning"],
                        "speedup_fp32_over_fp64": value / (r64["particle_steps"] / r64["seconds"])}
    if e2e is not None:
        line["e2e"] = {"value": e2e["value"], "unit": "particle-steps/s",
                       "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": e2e["d2h_bytes_per_step"], "steps": 2}
    if not args.no_cpu:
        cb = batched_oracle_sample(40, min(16, cpu_workers()))
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()


# ----------------------------------------------------------------------------
def main():
    global COMPACT_INTERVAL, BATCH_SCALE, BATCH_STEPS, BATCH_AUTOTUNE, GENERATOR
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20 for cascade512, 597 for collision)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 side-by-side run")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-per-worker", type=int, default=600)
    ap.add_argument("--compact-interval", type=int, default=COMPACT_INTERVAL,
                    help="steps between compactions (which also regroup photons that cannot pair)")
    ap.add_argument("--electrons", type=int, default=N_ELECTRONS,
                    help="beam size (smaller beams are for profiling captures, not bench lines)")
    ap.add_argument("--generator", type=int, default=0, choices=(0, 1, 2),
                    help="collision: emission generator (0 modified, 1 alternative, 2 standard)")
    ap.add_argument("--tuning", default="",
                    help="collision, cascade512: qed_tuning fields, e.g. deposit_halo=3,refill_lanes=16")
    ap.add_argument("--workload", choices=("collision", "batched", "cascade", "cascade512"), default="cascade512",
                    help="cascade512: the large 512^3 cascade with its slab target, a window of its run (the "
                         "headline line); collision: the beam-laser collision; batched: 512 ensembles; "
                         "cascade: the self-consistent 256^3 cascade")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="batched: electron counts x this (smaller sets are for profiling captures)")
    ap.add_argument("--batch-steps", type=int, default=BATCH_STEPS, help="batched: steps of the run")
    ap.add_argument("--no-autotune", action="store_true", help="batched: keep the default tuning")
    ap.add_argument("--profile-window", default="",
                    help="cascade, cascade512: START:COUNT, run to START and profile COUNT steps "
                         "(for ncu captures)")
    ap.add_argument("--cascade-caps", default="", help="cascade, cascade512: e-,e+,photon capacities (profiling)")
    ap.add_argument("--box", type=int, default=512,
                    help="cascade512 --profile-window: mesh edge of the same recipe (small profiling cases)")
    args = ap.parse_args()
    if args.electrons != N_ELECTRONS:
        scale_workload(args.electrons)
    COMPACT_INTERVAL = args.compact_interval
    GENERATOR = args.generator
    for kv in filter(None, args.tuning.split(",")):
        k, v = kv.split("=")
        TUNING[k.strip()] = int(v)
    if args.steps is None:
        args.steps = LARGE_STEPS if args.workload == "cascade512" else RUN_STEPS - 3
    K, W = args.steps, args.warmup
    if K < 1 or W < 0 or (args.workload == "collision" and K + W > RUN_STEPS):
        ap.error(f"need 1 <= steps, 0 <= warmup and (collision) steps + warmup <= {RUN_STEPS}")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "cascade":
        if args.impl == "reference":
            if rank == 0:
                cb = cascade_oracle_sample(6)
                print(json.dumps({"metric": METRIC, "value": cb["value"], "unit": "particle-steps/s",
                                  "n_gpus": args.gpus, "steps": 6, "warmup": 0, "higher_is_better": True,
                                  "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                                  "impl": "reference", "config": {"workload": CASCADE_NAME, "sample": cb["sample"]},
                                  "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                                  "e2e": {"value": cb["value"], "unit": "particle-steps/s",
                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
            return
        main_cascade(args, world, rank, local)
        return
    if args.workload == "cascade512":
        if args.impl == "reference":
            if rank == 0:
                # the oracle as it stands on a 32^3 box of the same recipe: W
                # untimed steps, then K timed steps (about 6 s each on one core)
                cb = large_oracle_sample(W + K, n=32, time_from=W)
                print(json.dumps({"metric": METRIC, "value": cb["value"], "unit": "particle-steps/s",
                                  "n_gpus": args.gpus, "steps": K, "warmup": W,
                                  "ms_per_step": cb["seconds"] * 1e3 / K, "higher_is_better": True,
                                  "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                                  "impl": "reference", "config": {"workload": LARGE_NAME, "sample": cb["sample"]},
                                  "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                                  "e2e": {"value": cb["value"], "unit": "particle-steps/s",
                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
            return
        main_large(args, world, rank, local)
        return
    if args.workload == "batched":
        BATCH_SCALE, BATCH_STEPS, BATCH_AUTOTUNE = args.batch_scale, args.batch_steps, not args.no_autotune
        if args.impl == "reference":
            if rank == 0:
                cb = batched_oracle_sample(40, min(16, cpu_workers()))
                print(json.dumps({"metric": METRIC, "value": cb["value"], "unit": "particle-steps/s",
                                  "n_gpus": args.gpus, "steps": 40, "warmup": 0, "higher_is_better": True,
                                  "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                                  "impl": "reference", "config": {"workload": BATCH_NAME, "sample": cb["sample"]},
                                  "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                                  "e2e": {"value": cb["value"], "unit": "particle-steps/s",
                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
            return
        main_batched(args, world, rank, local)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        ref = oracle_sample(K, W, args.cpu_per_worker, cpu_workers())
        line = {"metric": METRIC, "value": ref["value"], "unit": "particle-steps/s", "n_gpus": args.gpus,
                "steps": K, "warmup": W, "ms_per_step": ref["seconds"] * 1e3 / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": WORKLOAD_NAME, "sample": ref["sample"]},
                "cpu_baseline": {k: ref[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": ref["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import torch.distributed as tdist

    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            tdist.barrier()

    from paper_1412_6426_gb300 import build
    build.build()
    w = make_workload(seed=rank_seed(rank))   # weak scaling: each rank its own beam
    r32 = time_device(w, 32, K, W, barrier)
    r64 = None if args.no_fp64 else time_device(w, 64, K, W, barrier)
    e2e = None if args.no_e2e else time_e2e(w, 32, K, W)

    tot_ps, max_s = combine_ranks([(r32["particle_steps"], "sum"), (r32["seconds"], "max")])
    value = tot_ps / max_s
    out64 = None
    if r64 is not None:
        tot64, max64 = combine_ranks([(r64["particle_steps"], "sum"), (r64["seconds"], "max")])
        out64 = {"value": tot64 / max64, "ms_per_step": r64["ms_per_step"]}
    e2e_val = None
    if e2e is not None:
        tot_e, max_e = combine_ranks([(e2e["particle_steps"], "sum"), (e2e["seconds"], "max")])
        e2e_val = tot_e / max_e
    if rank != 0:
        if world > 1:
            tdist.destroy_process_group()
        return

    peak, peak_kind = peaks()

    def roof(r):
        # the dominant kernel: the photon pass-0 kernel (photons are most of the particles)
        ach = r["photon_algo_bytes"] / r["photon_seconds"] / 1e9
        per_unit = PHOTON_DRAM_BYTES_PER_STEP.get(r["precision"])
        traffic = per_unit * r["photon_steps"] / K if per_unit else None
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": traffic, "peak_source": peak_kind,
                "kernel": "k_photons<float>" if r["precision"] == 32 else "k_photons<double>",
                "kernel_ms_per_launch": r["photon_seconds"] * 1e3 / K,
                "algorithmic_bytes_per_launch": r["photon_algo_bytes"] / K,
                "units_per_launch": r["photon_steps"] / K, "bytes_per_unit": BYTES_PER_STEP[r["precision"]]}

    def roof_step(r):
        # every kernel of the step (photons, electrons/positrons/ions, in-step products)
        ach = r["algo_bytes"] / r["kernel_seconds"] / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "kernels_ms_per_step": r["kernel_seconds"] * 1e3 / K,
                "algorithmic_bytes_per_step": r["algo_bytes"] / K}

    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": r32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME if N_ELECTRONS == 1_000_000 else
                       WORKLOAD_NAME.replace("1e6 e-", f"{N_ELECTRONS:.0e} e-"), "window_steps": [r32["window_start"] + W,
                                                                   r32["window_start"] + W + K - 1],
                       "precision": "fp32 push/rates, fp64 tables", "parallelism": f"independent beams x{world}",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "compact_interval": COMPACT_INTERVAL, "tuning": TUNING or "default",
                       "generator": ("modified", "alternative", "standard")[GENERATOR]},
            "roofline": roof(r32),
            "roofline_step": roof_step(r32),
            "gpu_launches": r32["launches"],
            "clocks": r32["clocks"],
            "events": {"emissions": r32["emissions"], "pairs": r32["pairs"], "substeps": r32["substeps"],
                       "live_at_end": r32["live_end"]}}
    if out64 is not None:
        line["fp64"] = {"value": out64["value"], "ms_per_step": out64["ms_per_step"], "roofline": roof(r64),
                        "roofline_step": roof_step(r64),
                        "speedup_fp32_over_fp64": value / out64["value"], "clocks": r64["clocks"]}
    if e2e is not None:
        line["e2e"] = {"value": e2e_val, "unit": "particle-steps/s",
                       "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": e2e["d2h_bytes_per_step"]}
    if not args.no_cpu:
        cb = oracle_sample(K, W, args.cpu_per_worker, cpu_workers())
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
