#!/usr/bin/env python3
"""Benchmark of the EC PIC/MCC hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

A step is one pass of the whole hot path (gather, push, electrode absorption,
null-collision MCC with births, S_2 charge assignment, field solve; plus the
counting sort every sort_period steps) over all particles of the production
explicit workload: 6.7 cm gap, 512 cells, 2,048,000 macro-particles per
species, 450 V at 13.56 MHz, 30 mTorr.  Inputs are resident in HBM; each
timed step is bracketed by CUDA events on the run's stream and the L2 is
flushed (a 256 MB write) between timed steps, outside the events.

--impl reference times the CPU oracle (FP64, one core) on a bounded sample
of the same workload.  N > 1 runs independent replicas, one per GPU (the
method's runs do not exchange data): value = particles of all ranks / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "particle-steps/s (push+deposit+MCC)"
UNIT = "particle-steps/s"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "dominant_kernel_traffic.json")

WORKLOADS = {
    "ccp_512cells_2048000ppsp": workloads.CFG_WIDE_EXPLICIT,
    "ccp_128cells_implicit": workloads.CFG_IMPLICIT,
    "ccp_64cells_12800ppsp": workloads.CFG_SMALL_CCP,
    # the production explicit workload with the m = 3 scheme
    "ccp_512cells_2048000ppsp_m3": dict(workloads.CFG_WIDE_EXPLICIT, scheme="ec3_explicit"),
    # the same on a stretched grid (Sec. 4's multi-scale grid)
    "ccp_512cells_2048000ppsp_stretched": workloads.CFG_WIDE_STRETCHED,
    "ccp_128cells_implicit_stretched": workloads.CFG_IMPLICIT_STRETCHED,
}


def kernel_source_sha() -> str:
    p = os.path.join(ROOT, "paper_1310_5284_gb300", "csrc", "pic_kernels.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def algorithmic_bytes_per_particle(scheme: str) -> dict:
    """Bytes one launch must move per particle (structure of arrays, 4 B per
    field): explicit reads cell word, offset and vx and writes them back (the
    cell word carries the wait to the particle's next null-collision
    selection); a particle whose wait runs out also reads its id, vy and vz
    and writes vx, vy, vz and its cell word (new wait).  The implicit
    corrector reads cell word, offset, vx and abar and writes them; its
    predictor reads cell word, offset, vx and abar."""
    if scheme in ("ec_implicit", "mc_implicit"):
        return {"per_particle": 32, "per_selected": 28, "predictor_per_particle": 16}
    return {"per_particle": 24, "per_selected": 28}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def replica_config(cfg: dict, rank: int) -> dict:
    """Rank r's replica: an independent discharge of the same workload (its
    own load seed and Philox run index); replicas exchange no data."""
    return dict(cfg, seed=cfg.get("seed", 1) + 1000 * rank, run=rank)


def job_totals(total_ms: float, particle_steps: float, world: int, device=None):
    """Whole-job aggregate over `world` ranks of the initialised process
    group: the slowest rank's timed total and the sum of all ranks'
    particle-steps (value = the latter over the former)."""
    if world <= 1:
        return total_ms, particle_steps
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([particle_steps], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def run_gpu(args, wl_name, cfg, rank, world):
    import torch
    from paper_1310_5284_gb300.sim import Sim
    from paper_1310_5284_gb300 import _abi

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg = replica_config(cfg, rank)
    sim = Sim(cfg, device=dev)
    stream = sim.stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    K, W = args.steps, args.warmup
    sort_period = int(cfg.get("sort_period", 16))
    implicit = cfg["scheme"] in ("ec_implicit", "mc_implicit")

    with torch.cuda.stream(stream):
        sim.step(W)
        torch.cuda.synchronize(dev)
        d0 = sim.diag()
        step0 = d0["step"]
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(dev.index)
        clocks.start()
        t_wall = time.perf_counter()
        for k in range(K):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            sim.step(1)
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
        clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in evs]  # ms
    d1 = sim.diag()
    n_avg = 0.5 * (sum(d0["count"]) + sum(d1["count"]))

    # dominant kernel: the fused particle launch (non-sort steps hold exactly it,
    # or the implicit predictor + corrector pair)
    sort_idx = [k for k in range(K) if sort_period > 0 and (step0 + k + 1) % sort_period == 0]
    plain = [times[k] for k in range(K) if k not in set(sort_idx)]
    t_push = sum(plain) / len(plain) if plain else min(times)
    sort_times = [times[k] for k in sort_idx]
    if sort_period > 0 and not sort_times:
        # the window held no sort step: time steps after it, flushed alike,
        # up to and including the next one (outside the window's totals)
        with torch.cuda.stream(stream):
            extra = []
            while True:
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.fill_(-1.0)
                a_.record(stream)
                sim.step(1)
                b_.record(stream)
                torch.cuda.synchronize(dev)
                extra.append(a_.elapsed_time(b_))
                if (step0 + K + len(extra)) % sort_period == 0:
                    break
            sort_times = extra[-1:]
    t_sort = (sum(sort_times) / len(sort_times) - t_push) if sort_times else 0.0
    # every step carries 1/sort_period of a sort: the K steps are charged their
    # plain launches plus that share, whatever share of sorts the window held
    ms_amortised = t_push + (t_sort / sort_period if sort_period > 0 else 0.0)
    total_ms = ms_amortised * K
    total_ms_max, particle_steps = job_totals(total_ms, n_avg * K, world, device=dev)
    value = particle_steps / (total_ms_max * 1e-3)
    sel = sum(d1["coll"]) - sum(d0["coll"])  # selected particles over the K steps
    bpp = algorithmic_bytes_per_particle(cfg["scheme"])
    slots = n_avg
    bytes_launch = bpp["per_particle"] * slots + bpp["per_selected"] * sel / K
    if implicit:
        bytes_launch += bpp["predictor_per_particle"] * slots
    peak, peak_kind = measured_peak()
    achieved = bytes_launch / (t_push * 1e-3) / 1e9
    traffic = None
    try:
        tr = json.load(open(PROFILE_TRAFFIC))
        if tr.get("kernel_source_sha") == kernel_source_sha() and tr.get("workload") == wl_name:
            traffic = float(tr["dram_bytes_per_particle"]) * slots
    except Exception:
        traffic = None
    launches_per_step = 2 if implicit else 1
    gpu_launches = launches_per_step * K + len(sort_idx)

    # end to end through the public API with host buffers: every step uploads
    # both species from pinned host memory (pic_set_particles), re-assigns
    # charge and solves (pic_init_field), steps once and reads the diagnostics.
    e2e = run_e2e(sim, args.e2e_steps, dev) if args.e2e_steps > 0 else None
    sim.close()
    return dict(value=value, total_ms=total_ms_max, times=times, t_push=t_push, t_sort=t_sort,
                window_ms=sum(times),
                achieved=achieved, peak=peak, peak_kind=peak_kind, bytes_launch=bytes_launch,
                traffic=traffic, clocks=clk, gpu_launches=gpu_launches, n_avg=n_avg, e2e=e2e,
                wall_s=t_wall, counts=d1["count"], sort_steps=len(sort_idx))


def run_e2e(sim, steps, dev):
    import numpy as np
    import torch

    host = {}
    for sp in ("e", "i"):
        p = sim.get_particles(sp)
        pinned = {}
        for k in ("cell", "off", "vx", "vy", "vz", "id"):
            t = torch.from_numpy(np.ascontiguousarray(p[k])).pin_memory()
            pinned[k] = t.numpy()
        host[sp] = (pinned, p["next_id"])
    h2d = sum(sum(a.nbytes for a in host[sp][0].values()) for sp in host)

    def one_step():
        sim.set_state(host["e"][0], host["i"][0], next_id_e=host["e"][1], next_id_i=host["i"][1])
        sim.init_field(set_abar=False)
        sim.step(1)
        return sim.diag()

    for _ in range(2):  # untimed: first-use costs of the upload path
        one_step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    n_proc = 0
    d2h = 512  # the device state record read by pic_diag
    for _ in range(steps):
        n_proc += sum(one_step()["count"])
    t = time.perf_counter() - t0
    return {"value": n_proc / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h,
            "steps": steps}


def oracle_baseline(cfg, budget_s=12.0, max_steps=40):
    """The FP64 CPU oracle, as it stands, on a bounded sample: the workload
    loaded at full size, then steps until about budget_s of stepping."""
    import oracle
    n = int(cfg["np_init"])
    sim = oracle.Sim(cfg).load(n, n)
    steps, t_used, parts = 0, 0.0, 0
    while steps < max_steps and t_used < budget_s:
        d = sim.diag()
        t0 = time.perf_counter()
        sim.step(1)
        t_used += time.perf_counter() - t0
        parts += sum(d["count"])
        steps += 1
    return {"value": parts / t_used, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%s at full size (%d per species), first %d steps after the load, FP64, one thread"
                      % (cfg["name"], n, steps)}


def energy_drift(steps=2000):
    """Total-energy drift of the collisionless periodic EC plasma (64 cells,
    4096 electrons, dx = 10 Debye lengths, omega_p dt = 0.1): FP32 GPU push
    against the FP64 oracle over the same steps."""
    import numpy as np

    import oracle
    from paper_1310_5284_gb300.sim import Sim
    e, eps0, me = 1.602176634e-19, 8.8541878128e-12, 9.1093837015e-31
    n0, te = 1e15, 2.0
    lam = math.sqrt(eps0 * te / (n0 * e))
    wp = math.sqrt(n0 * e * e / (eps0 * me))
    cfg = workloads.cfg_periodic(n_cells=64, np_e=4096, n0=n0, length=64 * 10 * lam, dt=0.1 / wp, te_ev=te,
                                 seed=11)
    cfg["sort_period"] = 16
    out = {}
    for name, sim in (("gpu_fp32", Sim(cfg)), ("oracle_fp64", oracle.Sim(dict(cfg, quantized=True)).load(4096, 0))):
        sim.step(1)
        e0 = sim.energy()
        dev = 0.0
        for _ in range(steps // 100):
            sim.step(100)
            dev = max(dev, abs(sim.energy() / e0 - 1.0))
        out[name] = dev
        if hasattr(sim, "close"):
            sim.close()
    out["case"] = "periodic 64 cells, 4096 e-, dx=10 lambda_D, omega_p dt=0.1, %d steps, max |dE/E|" % steps
    return out


def _oracle_run_sample(args):
    """One run of the batched sweep in the FP64 oracle: load (untimed), then
    `steps` timed steps.  Runs in a worker process of its own."""
    cfg, steps = args
    import oracle
    n = int(cfg["np_init"])
    sim = oracle.Sim(cfg).load(n, n)
    parts = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        parts += sum(sim.diag()["count"])
        sim.step(1)
    return os.getpid(), parts, time.perf_counter() - t0


def oracle_batched_baseline(cfgs, steps=1):
    """The FP64 oracle over the runs of the batched sweep, one process per
    host core (spawned, so no GPU context is inherited): each run loaded,
    then `steps` steps timed.  Aggregate = all particle-steps / the busiest
    worker's stepping time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    busy, parts = {}, 0
    with ctx.Pool(cores) as pool:
        for pid, p_, t in pool.imap_unordered(_oracle_run_sample, [(c, steps) for c in cfgs]):
            busy[pid] = busy.get(pid, 0.0) + t
            parts += p_
    return {"value": parts / max(busy.values()), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "all %d runs of the batched sweep, %d step(s) each after the load, FP64, one process "
                      "per core" % (len(cfgs), steps)}


def bench_batched(n_runs=256, steps=2000, warmup=3, single_steps=12):
    """Batched persistent launches over the sweep of uneven discharges (cells
    64..1024, 1e4..2e6 particles per species, explicit and implicit) timed
    over `steps` steps (the particles, about 4 GB, are far larger than the
    L2), with the roofline of the launches from each run's algorithmic bytes;
    against the same runs advanced one by one through the single-run path
    (`single_steps` steps each) on the same GPU.  Both forms give
    bit-identical particles (tests/test_gpu_batch.py)."""
    import torch
    from paper_1310_5284_gb300.batch import BatchSim
    from paper_1310_5284_gb300.sim import Sim

    cfgs = workloads.batch_discharges(n_runs)
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    batch = BatchSim(cfgs, device=dev)
    tune = batch.autotune(trial_steps=4)
    batch.step(warmup)
    torch.cuda.synchronize(dev)
    d0 = [batch.diag(r) for r in range(n_runs)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index)
    clocks.start()
    a.record(batch.stream)
    batch.step(steps)
    b.record(batch.stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    t_batch = a.elapsed_time(b) * 1e-3
    d1 = [batch.diag(r) for r in range(n_runs)]
    status = batch.status()
    batch.close()
    del batch
    torch.cuda.empty_cache()
    ps_batch, bytes_total = 0.0, 0.0
    for cfg, x0, x1 in zip(cfgs, d0, d1):
        n_avg = 0.5 * (sum(x0["count"]) + sum(x1["count"]))
        bpp = algorithmic_bytes_per_particle(cfg["scheme"])
        per = bpp["per_particle"] + bpp.get("predictor_per_particle", 0)
        sel = sum(x1["coll"]) - sum(x0["coll"])
        ps_batch += n_avg * steps
        bytes_total += per * n_avg * steps + bpp["per_selected"] * sel
    achieved = bytes_total / t_batch / 1e9
    peak, kind = measured_peak()
    # the single-run form: each run alone, single_steps steps, times summed
    t_single, ps_single = 0.0, 0.0
    for cfg in cfgs:
        sim = Sim(cfg, device=dev)
        sim.step(warmup)
        torch.cuda.synchronize(dev)
        n0_ = sum(sim.diag()["count"])
        a.record(sim.stream)
        sim.step(single_steps)
        b.record(sim.stream)
        torch.cuda.synchronize(dev)
        t_single += a.elapsed_time(b) * 1e-3
        ps_single += 0.5 * (n0_ + sum(sim.diag()["count"])) * single_steps
        sim.close()
    parts = sum(0.5 * (sum(x0["count"]) + sum(x1["count"])) for x0, x1 in zip(d0, d1))
    out = {"n_runs": n_runs, "steps": steps, "window_s": t_batch, "particles": int(parts),
           "value": ps_batch / t_batch, "unit": UNIT, "status": status, "clocks": clk,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "peak_source": kind,
                        "bytes": "per run 24 B (explicit) or 48 B (direct implicit) per particle + 28 B per "
                                 "selected particle"},
           "single_run_value": ps_single / t_single, "single_run_steps": single_steps,
           "speedup_vs_single_runs": (ps_batch / t_batch) / (ps_single / t_single),
           "autotuned": tune, "accuracy": "bit-identical to the single-run form"}
    return out


def bench_adjoint(n_particles=1_000_000, n_cells=256, nsteps=200, checkpoint_every=20):
    """Forward + checkpointed backward of the collisionless EC run (1M
    electrons on a frozen ion background, 256 cells, 200 steps, checkpoint
    every 20) against the plain single-run step of the same configuration,
    and dJ/dV0 of the driven case against a central difference (h = 1e-4 V0)."""
    import numpy as np
    import torch
    from paper_1310_5284_gb300.adjoint import AdjointRun
    from paper_1310_5284_gb300.sim import Sim

    e, eps0, me = 1.602176634e-19, 8.8541878128e-12, 9.1093837015e-31
    n0, te = 1e15, 2.0
    wp = math.sqrt(n0 * e * e / (eps0 * me))
    dt = 0.1 / wp
    length = n_cells * 1.0e-4
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    out = {"n_particles": n_particles, "n_cells": n_cells, "steps": nsteps, "checkpoint_every": checkpoint_every}
    for name, periodic, volt in (("periodic", True, 0.0), ("driven", False, 100.0)):
        spec = dict(periodic=periodic, n_cells=n_cells, n_particles=n_particles, nsteps=nsteps, n0=n0,
                    bg_density=n0, length=length, dt=dt, rf_freq=0.0 if periodic else 1.0 / (nsteps * dt),
                    checkpoint_every=checkpoint_every)
        st = workloads.injected_particles(77, n_particles, n_cells, math.sqrt(e * te / me), sorted_cells=True)
        cell = torch.from_numpy(st["cell"]).to(dev)
        off = torch.from_numpy(st["off"]).to(dev)
        vx = torch.from_numpy(st["vx"]).to(dev)
        run = AdjointRun(spec, device=dev)
        run.forward(volt, cell, off, vx)
        run.backward(1.0, 0.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        pw, fl = run.forward(volt, cell, off, vx)
        t1 = time.perf_counter()
        g_v, _, d_volt = run.backward(1.0, 0.0)
        t2 = time.perf_counter()
        res = {"forward_ms": (t1 - t0) * 1e3, "backward_ms": (t2 - t1) * 1e3, "power": pw, "flux": fl,
               "dP_dV0": d_volt, "grad_v_rms": float(g_v.float().pow(2).mean().sqrt())}
        if not periodic:
            h = 1e-4 * volt
            pp, _ = run.forward(volt + h, cell, off, vx)
            ap = run.final_state()["cell"] >= 0
            pm, _ = run.forward(volt - h, cell, off, vx)
            am = run.final_state()["cell"] >= 0
            res["dP_dV0_central_difference"] = (pp - pm) / (2 * h)
            res["absorption_events_changed_by_h"] = int(np.sum(ap != am))
            res["central_difference_note"] = (
                "not comparable with dP_dV0: the +-h runs absorb different particles, and the adjoint holds "
                "absorption events fixed; the finite-difference check of the gradient is the event-free case "
                "of tests/test_gpu_adjoint.py")
        run.close()
        # the plain single-run form of the same configuration
        cfg = dict(n_cells=n_cells, periodic=periodic, length=length, dt=dt, rf_freq=spec["rf_freq"],
                   rf_volt=volt, n0=n0, bg_density=n0, np_init=n_particles, mcc=False, ions_mobile=False,
                   sort_period=0, capacity=n_particles, births_capacity=16, eedf_bins=8)
        sim = Sim(cfg, device=dev)
        sim.set_particles("e", dict(st, id=np.arange(n_particles, dtype=np.uint32)), next_id=n_particles)
        sim.init_field()
        sim.step(5)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(sim.stream)
        sim.step(nsteps)
        b.record(sim.stream)
        torch.cuda.synchronize(dev)
        res["plain_run_ms"] = a.elapsed_time(b)
        res["forward_plus_backward_over_plain"] = (res["forward_ms"] + res["backward_ms"]) / res["plain_run_ms"]
        sim.close()
        out[name] = res
    return out


def bench_paper_table(steps=200, warmup=20):
    """The paper's Table 1 shape on GB300 (context, not a target): wall time per
    RF period (2469 steps of 1.5e-11 s at 27 MHz) of the paper-shaped
    discharge (4 cm, 200 V, 50 mTorr, 400 macro-particles per cell and
    species) for 800/400/200/64 cells, all four schemes of Sec. 2.
    Steps timed with CUDA events, no L2 flush (the paper's runs are long)."""
    import torch
    from paper_1310_5284_gb300.sim import Sim

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    steps_per_period = round(1.0 / (27.0e6 * 1.5e-11))
    rows = {}
    for n in (800, 400, 200, 64):
        row = {}
        for scheme in ("ec_explicit", "mc_explicit", "ec_implicit", "mc_implicit"):
            cfg = workloads.cfg_paper(n, scheme)
            sim = Sim(cfg, device=dev)
            sim.step(warmup)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(sim.stream)
            sim.step(steps)
            b.record(sim.stream)
            torch.cuda.synchronize(dev)
            ms = a.elapsed_time(b) / steps
            row[scheme] = {"ms_per_step": ms, "s_per_rf_period": ms * 1e-3 * steps_per_period,
                           "particles": sum(sim.diag()["count"])}
            sim.close()
        rows[str(n)] = row
    return {"steps_per_rf_period": steps_per_period, "cells": rows,
            "paper_seconds_per_period_ec_explicit_on_a_pc": {"800": 35.2, "400": 16.7, "200": 8.0, "64": 2.3}}


def bench_self_heating(steps=2000):
    """EC against momentum-conserving gather on the 512-cell grid at dx = 4
    Debye lengths (Sec. 2): a collisionless periodic plasma of the production
    density, 2.05 M electrons on a frozen ion background; relative change of
    the total energy over the run for both schemes."""
    import torch
    from paper_1310_5284_gb300.sim import Sim

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    w = workloads.CFG_WIDE_EXPLICIT
    out = {"steps": steps, "n_cells": w["n_cells"], "electrons": w["np_init"],
           "dx_over_debye": 4.0, "omega_p_dt": 0.44}
    for scheme in ("ec_explicit", "mc_explicit"):
        cfg = workloads.cfg_periodic(n_cells=w["n_cells"], np_e=w["np_init"], n0=w["n0"], length=w["length"],
                                     dt=w["dt"], te_ev=2.0, scheme=scheme, seed=21)
        cfg["sort_period"] = 8
        sim = Sim(cfg, device=dev)
        sim.step(1)
        e0 = sim.energy()
        sim.step(steps)
        torch.cuda.synchronize(dev)
        out[scheme] = {"relative_energy_change": sim.energy() / e0 - 1.0}
        sim.close()
    return out


def bench_implicit(steps=4000, warmup=20, cfg=None, label="ccp_128cells_implicit (omega_p dt = 2)"):
    """The direct-implicit workload (128 cells, 1.02 M per species, omega_p dt
    = 2, 300 V, 50 mTorr): a step is the predictor and corrector launches,
    plus the sort every sort_period steps.  4000 steps timed one by one, the
    L2 flushed between them; the sort is charged to every step at its
    measured cost / sort_period.  Roofline of the launch pair: 48 B per
    particle (predictor reads cell word, offset, vx, abar; corrector reads
    those and writes them) + 28 B per particle whose wait runs out.  `status` says whether the window stayed clean (no dropped
    births or particles)."""
    import torch
    from paper_1310_5284_gb300.sim import Sim

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    cfg = dict(workloads.CFG_IMPLICIT if cfg is None else cfg)
    sim = Sim(cfg, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sim.step(warmup)
    torch.cuda.synchronize(dev)
    d0 = sim.diag()
    step0 = d0["step"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(sim.stream):
        for k in range(steps):
            flush.fill_(float(k))
            evs[k][0].record(sim.stream)
            sim.step(1)
            evs[k][1].record(sim.stream)
    torch.cuda.synchronize(dev)
    d1 = sim.diag()
    status = sim.status()
    sim.close()
    times = [a.elapsed_time(b) for a, b in evs]
    sp = cfg["sort_period"]
    is_sort = [(step0 + k + 1) % sp == 0 for k in range(steps)]
    plain = [t for t, srt in zip(times, is_sort) if not srt]
    sorts = [t for t, srt in zip(times, is_sort) if srt]
    t_pair = sum(plain) / len(plain)
    t_sort = sum(sorts) / len(sorts) - t_pair if sorts else 0.0
    ms = t_pair + t_sort / sp
    n_avg = 0.5 * (sum(d0["count"]) + sum(d1["count"]))
    sel = sum(d1["coll"]) - sum(d0["coll"])
    bpp = algorithmic_bytes_per_particle("ec_implicit")
    bytes_pair = (bpp["per_particle"] + bpp["predictor_per_particle"]) * n_avg + bpp["per_selected"] * sel / steps
    achieved = bytes_pair / (t_pair * 1e-3) / 1e9
    peak, kind = measured_peak()
    return {"workload": label, "ms_per_step": ms, "launch_pair_ms": t_pair,
            "sort_ms": t_sort, "steps": steps, "warmup": warmup, "value": n_avg / (ms * 1e-3), "unit": UNIT,
            "status": status, "counts_start_end": [d0["count"], d1["count"]],
            "births_per_step": (d1["births"] - d0["births"]) / steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": kind,
                         "bytes": "48 B per particle + 28 B per selected, predictor + corrector"}}


def bench_ec3(steps=96, warmup=10):
    """The production explicit workload with the m = 3 scheme (cubic S_3
    assignment, S_2 interpolation; same particles, same MCC): whole steps and
    the fused launch alone (steps without a sort), timed like the headline
    (L2 flushed between steps), with the fused launch's share of the HBM copy
    bandwidth on the same algorithmic bytes as m = 2."""
    return bench_fused_variant(dict(workloads.CFG_WIDE_EXPLICIT, scheme="ec3_explicit"),
                               "ccp_512cells_2048000ppsp_ec3", steps, warmup)


def bench_stretched(steps=96, warmup=10):
    """The production explicit workload on a stretched grid (cells 0.5x the
    uniform width at the electrodes, 1.5x mid-gap; Sec. 4's multi-scale
    grid): the same particles, MCC and algorithmic bytes as the uniform grid
    (the cell widths sit in shared memory), timed like the headline."""
    return bench_fused_variant(workloads.CFG_WIDE_STRETCHED, "ccp_512cells_2048000ppsp_stretched", steps, warmup)


def bench_fused_variant(cfg, label, steps, warmup):
    import torch
    from paper_1310_5284_gb300.sim import Sim

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    sim = Sim(cfg, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sim.step(warmup)
    torch.cuda.synchronize(dev)
    d0 = sim.diag()
    step0 = d0["step"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        evs[k][0].record(sim.stream)
        sim.step(1)
        evs[k][1].record(sim.stream)
    torch.cuda.synchronize(dev)
    d1 = sim.diag()
    status = sim.status()
    sim.close()
    times = [a.elapsed_time(b) for a, b in evs]
    sp = cfg["sort_period"]
    plain = [times[k] for k in range(steps) if (step0 + k + 1) % sp != 0]
    n_avg = 0.5 * (sum(d0["count"]) + sum(d1["count"]))
    sel = sum(d1["coll"]) - sum(d0["coll"])
    bpp = algorithmic_bytes_per_particle(cfg.get("scheme", "ec_explicit"))
    t_push = sum(plain) / len(plain)
    achieved = (bpp["per_particle"] * n_avg + bpp["per_selected"] * sel / steps) / (t_push * 1e-3) / 1e9
    peak, kind = measured_peak()
    ms = sum(times) / steps
    return {"workload": label, "ms_per_step": ms, "launch_ms": t_push,
            "value": n_avg / (ms * 1e-3), "unit": UNIT, "status": status,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": kind}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ccp_512cells_2048000ppsp", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-energy", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the paper table, self-heating and implicit lines")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    wl_name = args.workload
    cfg = dict(WORKLOADS[wl_name])
    config = {"workload": wl_name + "_" + cfg["scheme"], "n_cells": cfg["n_cells"],
              "particles_per_species": cfg["np_init"], "gap_m": cfg["length"], "rf_volt": cfg["rf_volt"],
              "dt_s": cfg["dt"], "pressure_mtorr": cfg["pressure_mtorr"], "sort_period": cfg.get("sort_period"),
              "l2": "flushed (256 MB write) between timed steps", "parallelism": "replicas" if world > 1 else "single"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        base = oracle_baseline(cfg, budget_s=min(20.0, 2.0 * args.steps))
        line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": base, "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                               "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    import __graft_entry__  # noqa: F401  (path setup only; the library must already be built)
    r = run_gpu(args, wl_name, cfg, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "roofline": {"bound": "hbm", "achieved": r["achieved"], "peak": r["peak"], "unit": "GB/s",
                     "frac": r["achieved"] / r["peak"], "traffic": r["traffic"],
                     "kernel": "k_particles (fused gather/push/absorb/MCC/deposit + tail)",
                     "algorithmic_bytes_per_launch": r["bytes_launch"], "launch_ms": r["t_push"],
                     "peak_source": r["peak_kind"]},
        "e2e": r["e2e"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
        "kernels": {"particles_ms": r["t_push"], "sort_ms": r["t_sort"], "sort_steps": r["sort_steps"],
                    "sort_period": cfg.get("sort_period"),
                    "ms_per_step_in_window": r["window_ms"] / args.steps,
                    "ms_per_step": "particle launch + sort_ms / sort_period (a sort every sort_period steps)"},
        "particles_live": r["counts"],
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(cfg)
    if world == 1 and not args.no_energy:
        line["energy_drift"] = energy_drift()
    if world == 1 and not args.no_adjoint:
        line["adjoint"] = bench_adjoint()
    if world == 1 and not args.no_batched:
        line["batched"] = bench_batched()
        if not args.no_cpu_baseline:
            line["batched"]["cpu_baseline"] = oracle_batched_baseline(workloads.batch_discharges(256))
    if world == 1 and not args.no_extras:
        line["implicit"] = bench_implicit()
        line["ec3"] = bench_ec3()
        line["ec3"]["over_m2_value"] = line["ec3"]["value"] / line["value"]
        line["stretched"] = bench_stretched()
        line["stretched"]["over_uniform_value"] = line["stretched"]["value"] / line["value"]
        if not args.no_cpu_baseline:
            line["stretched"]["cpu_baseline"] = oracle_baseline(workloads.CFG_WIDE_STRETCHED, budget_s=8.0,
                                                                max_steps=20)
        # the direct-implicit workload on the stretched grid (cells 0.5x the
        # uniform width at the electrodes, 1.5x mid-gap)
        line["stretched_implicit"] = bench_implicit(1000, 20, workloads.CFG_IMPLICIT_STRETCHED,
                                                    "ccp_128cells_implicit_stretched (omega_p dt = 2)")
        line["stretched_implicit"]["over_uniform_value"] = line["stretched_implicit"]["value"] / line["implicit"]["value"]
        line["self_heating"] = bench_self_heating()
        line["paper_table1"] = bench_paper_table()
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
