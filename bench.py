"""Benchmark of the modified-Ehrenfest MD step on one or more GB300s.

Workload: the 96^3 precision workload -- 64 Si-like pseudo-atoms, 128 doubly
occupied orbitals, 0.25 bohr spacing, 8th-order stencil, mu = 10,
dt = 0.05 sqrt(10) -- with complex64 orbitals and FP64 density, energies,
forces and ions (the headline line), plus the same workload in FP64 (extra
key).  A "step" is one full MD step: velocity-Verlet positions, ionic tables
and potential, 8 Horner stages of AETRS with Taylor-4 halves, density,
Hartree + LDA, forces, velocity-Verlet velocities.

Metric: orbital grid-point H*psi updates/s = 8 * n_orb * N^3 * steps / time
(8 applications of H per orbital and point per step).

Multi-GPU: the path is run as independent replicas, one per GPU (the method
does shard by orbitals with one density/force reduction per step, which this
build does not implement); value = all ranks' updates / max-over-ranks time.

--impl reference: times the FP64 CPU oracle (the restated method, plain
numpy) on the same workload: each step is one AETRS step (8 H applications)
of a bounded orbital subset, scaled per orbital-point update.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "orbital grid-point H*psi updates/s"
UNIT = "updates/s"
# Algorithmic bytes of one Horner-stage update (read u_in, read psi0, write
# u_out); the potential and projector lists are shared across an orbital
# block and not counted.
BYTES_PER_UPDATE = {"f32": 24, "f64": 48}
# dram__bytes_read.sum + dram__bytes_write.sum of one Horner-stage launch on
# the 96^3 workload (one ncu capture), per precision, for the kernel as
# built; None until a capture exists for it.
TRAFFIC_PER_LAUNCH = {"f32": 3.147e9, "f64": None}


def max_over_ranks(x: float, device=None) -> float:
    """max of x over the ranks of the default process group (x itself when
    there is none); device: where the reduction tensor lives (cuda for NCCL,
    cpu for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, seconds_max: float) -> float:
    """Weak scaling: every rank processes units_per_rank; the job's rate is
    all ranks' units over the slowest rank's time."""
    return ws * units_per_rank / seconds_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.samples = []
        self._proc = None
        self._th = None

    def _read(self):
        for line in self._proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.samples.append(f)

    def __enter__(self):
        # one nvidia-smi in its own sampling loop, read line by line; it is
        # this process's child and is ended through its handle
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._th = threading.Thread(target=self._read, daemon=True)
            self._th.start()
        except OSError:
            self._proc = None
        return self

    def __exit__(self, *a):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=10)
            except subprocess.TimeoutExpired:
                self._proc.kill()
                self._proc.wait(timeout=10)
        if self._th:
            self._th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def cpu_oracle_rate(sysin, n_orb_sample: int, reps: int = 1):
    """Oracle AETRS step (two Taylor-4 exponentials = 8 H applications) on
    n_orb_sample orbitals of the workload, with the full potential of the
    workload's density.  Returns (updates/s, seconds, threads)."""
    import numpy as np
    from oracle import emd_oracle as O
    s = sysin
    tables = O.atom_tables(s.R, s.species, s.n, s.h)
    g = O.ion_charge(tables, s.species, s.n)
    v_loc = O.poisson(-g, s.h)
    rho = O.density(s.psi, s.occ)
    v_h = O.poisson(rho, s.h)
    _, vxc = O.lda_pz81(rho)
    H = O.Hamiltonian(v_loc + v_h + vxc, tables, s.species, s.h, s.fd_order)
    psi = np.ascontiguousarray(s.psi[:n_orb_sample])
    tau = 0.5 * (s.dt / s.mu)
    c0 = os.times()
    t0 = time.perf_counter()
    for _ in range(reps):
        out = O.taylor4(O.taylor4(psi, tau, H), tau, H)
    dt = time.perf_counter() - t0
    c1 = os.times()
    upd = 8.0 * n_orb_sample * s.n ** 3 * reps
    # cores the oracle kept busy: process CPU time over wall time (numpy's
    # element-wise work and FFTs run on one thread, its BLAS calls on more)
    cores = ((c1.user - c0.user) + (c1.system - c0.system)) / dt
    return upd / dt, dt, round(cores, 2)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_0812_2801_gb300 import inputs
    s = inputs.precision_c96(mu=10.0)
    n_sample = 1
    for _ in range(args.warmup):
        cpu_oracle_rate(s, n_sample)
    times = []
    for _ in range(args.steps):
        _, dt, cores = cpu_oracle_rate(s, n_sample)
        times.append(dt)
    tot = sum(times)
    value = 8.0 * n_sample * s.n ** 3 * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "precision-64at-96^3 (Si-like, 128 orbitals, order 8, mu 10)",
                   "sample": f"{n_sample} of 128 orbitals per step, full potential"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one AETRS step (8 H applications) on {n_sample} of 128 orbitals of the 96^3 workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def time_md(emd, torch, sysin, precision, steps, warmup, profile=True):
    """Device-resident timing of `steps` MD steps; returns dict."""
    sysg = emd.System(sysin, precision)
    h = sysg.handle
    for _ in range(warmup):
        sysg.propagate(1)
    torch.cuda.synchronize()
    emd.emd_set_option(h, emd.EMD_OPT_PROFILE, 1 if profile else 0)
    emd.emd_kernel_stats(h, emd.EMD_KERNEL_HORNER)
    emd.emd_kernel_stats(h, emd.EMD_KERNEL_ALL)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record()
    for _ in range(steps):
        sysg.propagate(1)
    stop.record()
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    k_ms, k_n = emd.emd_kernel_stats(h, emd.EMD_KERNEL_HORNER)
    _, launches = emd.emd_kernel_stats(h, emd.EMD_KERNEL_ALL)
    emd.emd_set_option(h, emd.EMD_OPT_PROFILE, 0)
    e = sysg.energy()
    sysg.close()
    return {"ms": ms, "stage_ms": k_ms, "stage_launches": k_n, "launches": launches,
            "energy": e}


def energy_drift(emd, torch, sysin, precision, steps, every=20):
    """Relative change of the conserved energy E = T_ion + E_KS (eq. E_new)
    over `steps` MD steps of the 96^3 workload, sampled every `every` steps
    (graph replay between samples)."""
    sysg = emd.System(sysin, precision)
    e0 = sysg.energy()["total"]
    dev, done = 0.0, 0
    t0 = time.perf_counter()
    while done < steps:
        k = min(every, steps - done)
        sysg.propagate(k)
        done += k
        dev = max(dev, abs(sysg.energy()["total"] - e0))
    e1 = sysg.energy()["total"]
    wall = time.perf_counter() - t0
    sysg.close()
    return {"steps": steps, "mu": sysin.mu, "dt": sysin.dt, "sampled_every": every,
            "rel_change": abs(e1 - e0) / abs(e0), "max_rel_deviation": dev / abs(e0),
            "per_1000_steps_linear": abs(e1 - e0) / abs(e0) * 1000.0 / steps,
            "wall_s": wall}


def time_e2e(emd, torch, sysin, precision, steps):
    """Through the public API with host buffers: every step uploads orbitals
    (complex64, the precision the system keeps them in) and ions from pinned
    memory, propagates one MD step and reads back the orbitals, forces and
    energy.  Timed with CUDA events on the default stream (every call either
    synchronises it or enqueues on it), with a per-phase breakdown and the
    plain pinned-copy bandwidth of one orbital set each way for context."""
    import numpy as np
    s = sysin
    psi_pin = torch.empty(s.psi.shape, dtype=torch.complex64, pin_memory=True)
    psi_pin.numpy()[...] = s.psi
    out_pin = torch.empty(s.psi.shape, dtype=torch.complex64, pin_memory=True)
    R = np.ascontiguousarray(s.R)
    V = np.ascontiguousarray(s.V)
    h = emd.emd_init_system(emd.config_for(s, precision))
    psi_np = psi_pin.numpy()
    out_np = out_pin.numpy()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    phase = [0.0, 0.0, 0.0]

    def one(record=False):
        if record:
            ev[0].record()
        emd.emd_set_ions(h, R, V)
        emd.emd_set_orbitals_c64(h, psi_np)
        if record:
            ev[1].record()
        emd.emd_propagate(h, 1, s.dt, s.mu)
        if record:
            ev[2].record()
        emd.emd_get_orbitals_c64(h, s.n_orb, s.n, out=out_np)
        emd.emd_get_forces(h, s.n_atoms)
        emd.emd_get_energy(h)
        if record:
            ev[3].record()
            torch.cuda.synchronize()
            for k in range(3):
                phase[k] += ev[k].elapsed_time(ev[k + 1])

    one()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(steps):
        one()
    stop.record()
    torch.cuda.synchronize()
    dt = start.elapsed_time(stop) * 1e-3
    for _ in range(3):
        one(record=True)
    emd.emd_destroy(h)
    # plain pinned <-> device copies of one complex64 orbital set
    dev = torch.empty_like(psi_pin, device="cuda")
    bw = {}
    for name, dst, src in (("h2d_GBps", dev, psi_pin), ("d2h_GBps", out_pin, dev)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        start.record()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        stop.record()
        torch.cuda.synchronize()
        bw[name] = 3 * psi_np.nbytes / (start.elapsed_time(stop) * 1e-3) / 1e9
    del dev
    bi = psi_np.nbytes + R.nbytes + V.nbytes
    bo = psi_np.nbytes + 3 * 8 * s.n_atoms + 9 * 8
    breakdown = {"set_ms": phase[0] / 3, "propagate_ms": phase[1] / 3, "get_ms": phase[2] / 3}
    breakdown.update(bw)
    return dt, bi, bo, breakdown


def time_batched(emd, torch, steps, n_replicas=32):
    """32 ragged replicas (8-64 atoms, 48^3-80^3, 16-128 orbitals, order 8,
    complex64, mu = 10): one batch whose 6-step chunks replay a captured CUDA
    graph, against the same replicas propagated one after another; each
    replica runs the stage configuration (block width, tile variant,
    z-chunk) the autotuner measured fastest for its shape.  16 small 48^3
    replicas are also timed as a batch of their own, where launch overhead
    and an underfilled GPU are the larger share of a step."""
    from paper_0812_2801_gb300 import autotune, inputs
    specs = inputs.replica_specs(n_replicas, seed=5)
    sysins, cfgs = [], []
    tune_t0 = time.perf_counter()
    for i, spec in enumerate(specs):
        sysin = inputs.replica(spec, i)
        cfgs.append(autotune.best_config(sysin, emd.EMD_FP32_ORBITALS))
        sysins.append(sysin)
    tune_s = time.perf_counter() - tune_t0

    def run(idx):
        systems, upd = [], 0.0
        for i in idx:
            g = emd.System(sysins[i], emd.EMD_FP32_ORBITALS, block_orbitals=cfgs[i]["bo"])
            autotune.configure(g, cfgs[i])
            systems.append(g)
            upd += 8.0 * sysins[i].n_orb * sysins[i].n ** 3
        dt, mu = sysins[idx[0]].dt, sysins[idx[0]].mu
        b = emd.emd_batch_create([g.handle for g in systems])
        emd.emd_batch_propagate(b, 8, dt, mu)          # warm-up + graph capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        emd.emd_batch_propagate(b, steps, dt, mu)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        emd.emd_batch_destroy(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g in systems:
            g.propagate(steps, dt, mu)
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        for g in systems:
            g.close()
        return upd, t_batch, t_seq

    upd, t_batch, t_seq = run(list(range(len(sysins))))
    # 16 small replicas (8 atoms, 48^3, 16 orbitals) of another seed
    base = len(sysins)
    for spec in inputs.small_replica_specs(16, seed=6):
        sysin = inputs.replica(spec, len(sysins))
        cfgs.append(autotune.best_config(sysin, emd.EMD_FP32_ORBITALS))
        sysins.append(sysin)
    small = list(range(base, len(sysins)))
    s_upd, s_batch, s_seq = run(small) if small else (0.0, 1.0, 1.0)
    rep = autotune.report()
    chosen = {k: autotune.cfg_name(v["best"]) for k, v in rep.items()}
    timings = {k: {c: round(t["step_ms"], 3) for c, t in v["timings"].items()}
               for k, v in rep.items()}
    return {"value": upd * steps / t_batch, "unit": UNIT, "replicas": n_replicas,
            "steps": steps, "ms_per_step": 1e3 * t_batch / steps,
            "sequential_value": upd * steps / t_seq,
            "speedup_vs_sequential": t_seq / t_batch,
            "updates_per_step": upd,
            "small_48": {"replicas": len(small),
                         "workload": "8 Si-like atoms, 48^3, 16 orbitals each (seed 6)",
                         "value": s_upd * steps / s_batch,
                         "ms_per_step": 1e3 * s_batch / steps,
                         "speedup_vs_sequential": s_seq / s_batch},
            "configs": chosen, "tuning_step_ms": timings, "tuning_s": tune_s,
            "workload": "32 ragged replicas: 8-64 Si-like atoms, 48^3/64^3/80^3, "
                        "2 orbitals per atom, order 8, complex64, mu 10, dt 0.158"}


def time_adjoint(emd, torch, n_steps=200, ckpt=20):
    """Adjoint gradient of the final dipole with respect to the (initial) ion
    positions and 200 field amplitudes on the 64^3 field workload (16 atoms,
    32 orbitals, order 6, FP64, mu 10), fixed and moving ions, each against
    the plain forward run of the same dynamics."""
    from paper_0812_2801_gb300 import inputs
    s = inputs.field_c64(n_steps)
    upd = 8.0 * s.n_orb * s.n ** 3 * n_steps

    def fresh():
        h = emd.emd_init_system(emd.config_for(s))
        emd.emd_set_option(h, emd.EMD_OPT_FROZEN_IONS, 1)
        emd.emd_set_ions(h, s.R, s.V * 0.0)
        emd.emd_set_orbitals(h, s.psi)
        return h

    h = fresh()
    emd.emd_propagate(h, 2, s.dt, s.mu, s.field[:2])
    torch.cuda.synchronize()
    emd.emd_destroy(h)
    h = fresh()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    emd.emd_propagate(h, n_steps, s.dt, s.mu, s.field)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    emd.emd_destroy(h)
    h = fresh()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    emd.emd_propagate_adjoint(h, n_steps, s.dt, s.mu, s.field, ckpt,
                              emd.EMD_OBS_DIPOLE_Z, s.n_atoms)
    t_adj = time.perf_counter() - t0
    emd.emd_destroy(h)

    # moving ions (the workload's thermal velocities)
    def fresh_md():
        h = emd.emd_init_system(emd.config_for(s))
        emd.emd_set_ions(h, s.R, s.V)
        emd.emd_set_orbitals(h, s.psi)
        return h

    h = fresh_md()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    emd.emd_propagate(h, n_steps, s.dt, s.mu, s.field)
    torch.cuda.synchronize()
    t_fwd_md = time.perf_counter() - t0
    emd.emd_destroy(h)
    h = fresh_md()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    emd.emd_propagate_adjoint(h, n_steps, s.dt, s.mu, s.field, ckpt,
                              emd.EMD_OBS_DIPOLE_Z, s.n_atoms)
    t_adj_md = time.perf_counter() - t0
    emd.emd_destroy(h)
    return {"workload": "field-16at-64^3: 16 Si-like atoms (bcc), 32 orbitals, 64^3 at 0.3, "
                        "order 6, FP64, mu 10, 200 steps, checkpoints every 20",
            "fixed_ions": {"forward_s": t_fwd, "gradient_s": t_adj,
                           "gradient_over_forward": t_adj / t_fwd,
                           "forward_updates_per_s": upd / t_fwd},
            "moving_ions": {"forward_s": t_fwd_md, "gradient_s": t_adj_md,
                            "gradient_over_forward": t_adj_md / t_fwd_md,
                            "forward_updates_per_s": upd / t_fwd_md},
            "unit": UNIT}


def time_large(emd, torch, steps, warmup):
    """The 160^3 workload (512 atoms, 1024 orbitals, order 8, complex64,
    mu 50, dt 0.354): input built with GEMMs on the device, uploaded as
    complex64, then `steps` MD steps timed with CUDA events."""
    from paper_0812_2801_gb300 import inputs
    t0 = time.perf_counter()
    s = inputs.large_c160(device="cuda")
    torch.cuda.empty_cache()          # the GEMMs' blocks: the system needs ~115 GB
    build_s = time.perf_counter() - t0
    h = emd.emd_init_system(emd.config_for(s, emd.EMD_FP32_ORBITALS))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals_c64(h, s.psi)
    n_orb = s.n_orb
    s.psi = None                      # 33.5 GB of host memory
    for _ in range(warmup):
        emd.emd_propagate(h, 1, s.dt, s.mu)
    e0 = emd.emd_get_energy(h)
    torch.cuda.synchronize()
    emd.emd_set_option(h, emd.EMD_OPT_PROFILE, 1)
    emd.emd_kernel_stats(h, emd.EMD_KERNEL_HORNER)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(steps):
        emd.emd_propagate(h, 1, s.dt, s.mu)
    stop.record()
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    k_ms, k_n = emd.emd_kernel_stats(h, emd.EMD_KERNEL_HORNER)
    emd.emd_set_option(h, emd.EMD_OPT_PROFILE, 0)
    e1 = emd.emd_get_energy(h)
    emd.emd_destroy(h)
    n3 = s.n ** 3
    upd = 8.0 * n_orb * n3 * steps
    stage_s = k_ms * 1e-3 / max(1, k_n)
    peak, _ = measured_peaks()
    achieved = BYTES_PER_UPDATE["f32"] * n_orb * n3 / stage_s / 1e9
    return {"workload": "large-512at-160^3: 512 atoms, 1024 orbitals, 160^3 at 0.3 bohr, "
                        "order 8, mu 50, dt 0.354, complex64",
            "value": upd / (ms * 1e-3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "horner_stage_avg_ms": stage_s * 1e3,
            "horner_stage_frac_hbm": achieved / peak,
            "energy_change_rel": abs(e1["total"] - e0["total"]) / abs(e0["total"]),
            "input_build_s": build_s}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--batched-steps", type=int, default=12)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--large-steps", type=int, default=4,
                    help="timed steps of the 160^3 / 1024-orbital workload (0: skip; "
                         "one GPU only: ~115 GB on the device, 33.5 GB of host input)")
    ap.add_argument("--drift-steps", type=int, default=200,
                    help="steps of the energy-drift run on the 96^3 workload (0: skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_0812_2801_gb300 import emd, inputs
    emd.load()

    s = inputs.precision_c96(mu=10.0)
    n3 = s.n ** 3
    upd_per_step = 8.0 * s.n_orb * n3

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # headline: FP32 orbitals
    barrier()
    with ClockSampler(local) as clk:
        r32 = time_md(emd, torch, s, emd.EMD_FP32_ORBITALS, args.steps, args.warmup)
    barrier()
    ms = max_over_ranks(r32["ms"], device="cuda")
    value = whole_job_rate(upd_per_step * args.steps, ws, ms * 1e-3)

    # FP64 form on the same workload
    r64 = time_md(emd, torch, s, emd.EMD_FP64, args.fp64_steps, 1)
    v64 = upd_per_step * args.fp64_steps / (r64["ms"] * 1e-3)

    # end to end through the C ABI with host buffers
    barrier()
    e2e_dt, bi, bo, e2e_parts = time_e2e(emd, torch, s, emd.EMD_FP32_ORBITALS, args.e2e_steps)
    e2e_dt = max_over_ranks(e2e_dt, device="cuda")
    e2e_val = whole_job_rate(upd_per_step * args.e2e_steps, ws, e2e_dt)

    batched = None if args.no_batched else time_batched(emd, torch, args.batched_steps)
    adjoint = None if (args.no_adjoint or ws > 1) else time_adjoint(emd, torch)
    drift = (energy_drift(emd, torch, s, emd.EMD_FP32_ORBITALS, args.drift_steps)
             if args.drift_steps > 0 and ws == 1 else None)
    large = (time_large(emd, torch, args.large_steps, 1)
             if args.large_steps > 0 and ws == 1 else None)

    peak, peak_kind = measured_peaks()
    stage_avg_s = r32["stage_ms"] * 1e-3 / max(1, r32["stage_launches"])
    bytes_launch = BYTES_PER_UPDATE["f32"] * s.n_orb * n3
    achieved = bytes_launch / stage_avg_s / 1e9
    stage64_s = r64["stage_ms"] * 1e-3 / max(1, r64["stage_launches"])
    # FP64 form's stage: double-float arithmetic on the FP32 pipes, real and
    # imaginary parts in one FP32x2 instruction.  Packed operations per
    # update (one orbital at one point): dv u 13, each x/y shell 36 (three
    # double-float adds of the four neighbours, the weight's TwoProduct and
    # one add), each z shell 20 (TwoProduct, two adds into the delay line),
    # the epilogue 65 (the scale and four projector entries): 78 + 56 M,
    # i.e. 2 (78 + 56 M) FP32 lane operations.  Peak: 128 FP32 lanes x 152
    # SMs x 2.07 GHz (an FMA counts once).
    M = s.fd_order // 2
    df_ops = 2.0 * (78 + 56 * M)
    f32_peak = 128 * 152 * 2.07e9 / 1e12          # T FP32 lane operations/s
    df_achieved = df_ops * s.n_orb * n3 / stage64_s / 1e12
    f64_hbm = BYTES_PER_UPDATE["f64"] * s.n_orb * n3 / stage64_s / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "precision-64at-96^3: 64 Si-like atoms, 128 orbitals, "
                               "96^3 at 0.25 bohr, order 8, mu 10, dt 0.158; complex64 "
                               "orbitals, FP64 rho/energy/forces/ions",
                   "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (orbital set 906 MB)",
                   "md_steps_per_s": ws * args.steps / (ms * 1e-3)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": TRAFFIC_PER_LAUNCH["f32"],
                     "kernel": "horner_stage (FP32)",
                     "bytes_per_launch": bytes_launch,
                     "avg_launch_ms": stage_avg_s * 1e3},
        "fp64": {"value": v64, "unit": UNIT, "ms_per_step": r64["ms"] / args.fp64_steps,
                 "horner_stage_avg_ms": stage64_s * 1e3,
                 "speedup_fp32_over_fp64": value / ws / v64,
                 "roofline": {"bound": "alu", "unit": "T FP32 lane operations/s",
                              "achieved": df_achieved, "peak": f32_peak,
                              "frac": df_achieved / f32_peak, "peak_kind": "nominal",
                              "ops_per_update": df_ops,
                              "kernel": "horner_stage (FP64 form, double-float on FP32 pipes)",
                              "peak_note": "128 FP32 lanes x 152 SMs x 2.07 GHz; the plain "
                                           "FP64 stage (EMD_OPT_STAGE_VARIANT 1) is bound by "
                                           "2 FP64 lanes per SM",
                              "hbm_achieved_GBps": f64_hbm, "hbm_frac": f64_hbm / peak}},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo, "steps": args.e2e_steps,
                "ms_per_step": 1e3 * e2e_dt / args.e2e_steps, "breakdown": e2e_parts,
                "note": "per step: set_ions + set_orbitals_c64 (pinned host, complex64), "
                        "propagate 1 MD step, get_orbitals_c64 + get_forces + get_energy; "
                        "CUDA events"},
        "drift": drift,
        "batched": batched,
        "adjoint": adjoint,
        "large": large,
        "gpu_launches": r32["launches"],
        "clocks": clk.summary(),
        "energy_total": r32["energy"]["total"],
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, secs, cores = cpu_oracle_rate(s, 8)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"one AETRS step (8 H applications) on 8 of 128 "
                                          f"orbitals of the 96^3 workload ({secs:.1f} s)"}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
