"""Benchmark: MLUPS and fraction of the HBM roofline of the capillary-bridge time step on GB300.

Workload (default, tetra4): four free spheres R = 24 in a jittered tetrahedral cluster around a
central drop (liquid 0.05 of the solid volume, 60 degrees) in a 256^3 periodic box, D3Q19, FP32
populations, phase-field kinetics on (the four-particle set-up of Sec. 4.3.2 at R = 24). One step =
the whole hot path: pull streaming + bounce-back, density/psi, Shan-Chen force, Guo-BGK collision,
FP64 body reductions, repulsion, rigid-body update, phase-field advection and kinetics, flags and
refill. Other workloads: spheres2 (two spheres in 128x128x256), plates48, batch64, surrogate.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference] [--precision fp32]

The timed region is exactly K steps (one replay of the step graph each), bracketed by a barrier and a
device synchronisation; it is repeated (at least 5 times, until about two seconds of load have
passed or about 600 steps have run, whichever comes first) and the median repeat is reported.
N > 1 runs under torchrun as independent replicas (one per GPU, no collective: the step does not
shard across GPUs in this build); value = cells x steps summed over ranks / max time.
--impl reference times the FP64 CPU oracle (the slow, plain implementation the CUDA path is
checked against) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic bytes per cell update of the collision kernel: read 19 populations, write 19,
# read the uint16 flag (the density pass and psi are implementation overhead)
POP_BYTES = {"fp64": 8, "fp32": 4, "fp16dev": 2}


def kernels_per_step(nb, mpf, variant):
    """Kernel launches of one step of the library's graph: density + bulk collision (variant 0), the
    fused pass (1), or the edge fix-up + accumulating collision (2); the closing kernel (fluid mass,
    buffer flip); with bodies the tile pass of psi (variants 1 and 2), the collision of the cells
    next to a solid, the force pass, repulsion (two or more bodies), body update, three advection
    sweeps, kinetics (MPF on), flags and refill."""
    k = (1 if variant == 1 else 2) + 1
    if nb:
        k += (1 if variant in (1, 2) else 0) + 1 + 1 + (1 if nb > 1 else 0) + 1 + 3 + (1 if mpf else 0) + 2
    return k


# DRAM bytes per launch of the bulk collision, and per step of the whole step graph, from one-pass
# ncu captures (gpu__time_duration, dram__bytes_read/write only), valid only for the source they were
# taken on (source_hash of the lattice-Boltzmann sources); None otherwise
PROFILED = {
    ("tetra4", "fp32", 19, "e464e6a96e81"): 2722.1e6,      # k_collide<float>, mean of 15 launches
    ("tetra4", "fp16dev", 19, "e464e6a96e81"): 1452.5e6,   # k_collide<__half>, mean of 10 launches
}
PROFILED_STEP = {
    ("tetra4", "fp32", 19, "e464e6a96e81"): 4199.6e6,      # every kernel of one step
}


def source_hash():
    """sha1 prefix of the lattice-Boltzmann kernels' sources (lbm.cu and the shared device headers)."""
    import hashlib

    h = hashlib.sha1()
    for name in ("lbm.cu", "cbl_dev.cuh", "periodic.h", "weights.h"):
        with open(os.path.join(ROOT, "paper_1902_10432_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def profiled_traffic(workload_name, prec, q=19):
    return PROFILED.get((workload_name, prec, q, source_hash()))


def profiled_step_traffic(workload_name, prec, q=19):
    return PROFILED_STEP.get((workload_name, prec, q, source_hash()))


def alg_bytes_per_cell(prec, q=19):
    return 2 * q * POP_BYTES[prec] + 2


HBM_DATASHEET_GBS = 7900.0  # GB300 HBM3e nominal


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def describe(w, q):
    """One-line description of a workload from its own fields."""
    nb = len(w.bodies)
    shapes = sorted({b["shape"] for b in w.bodies})
    radii = sorted({round(b.get("radius", 0.0), 2) for b in w.bodies if b["shape"] == "sphere"})
    held = sum(1 for b in w.bodies if b.get("fixed"))
    body = "no bodies" if nb == 0 else "%d %s%s%s" % (
        nb, "free " if held == 0 else ("held " if held == nb else ""), "/".join(shapes) + ("s" if nb > 1 else ""),
        (" R=" + "/".join("%g" % r for r in radii)) if radii else "")
    extra = []
    if "liquid_fraction_of_solid" in w.meta:
        extra.append("liquid %.3g of solid volume" % w.meta["liquid_fraction_of_solid"])
    if "theta_deg" in w.meta:
        extra.append("%g deg" % w.meta["theta_deg"])
    return "%s %dx%dx%d D3Q%d, %s%s, %s populations, MPF kinetics %s" % (
        w.name, w.nx, w.ny, w.nz, q, body, (", " + ", ".join(extra)) if extra else "", w.params.get("prec", "fp32"),
        "on" if w.params.get("mpf_kinetics") else "off")


def workload(name, prec, q=19, sample=False):
    """The bench workload, or (sample=True) the bounded sample of it that the CPU oracle is timed on:
    tetra4 at half scale (128^3, R = 12, surface gap 4), the others as they are."""
    from paper_1902_10432_gb300 import workloads

    if name == "spheres2":
        w = workloads.spheres2(seed=0, prec=prec)
    elif name == "plates48":
        w = workloads.plates48(prec=prec)
    elif name == "tetra4":
        w = workloads.tetra4(seed=0, prec=prec, n=128, R=12.0, surface_gap=4.0) if sample else \
            workloads.tetra4(seed=0, prec=prec)
    else:
        raise ValueError(name)
    w.params["q"] = q
    return w


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        import statistics

        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_oracle_steps(w, steps, warmup, threads):
    import oracle
    from paper_1902_10432_gb300 import workloads

    kw = {k: v for k, v in w.params.items() if k != "prec"}
    o = oracle.Oracle(w.nx, w.ny, w.nz, nthreads=threads, **kw)
    workloads.build(o, w)
    if warmup:
        o.step(warmup)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        o.step(1)
        times.append(time.perf_counter() - t0)
    return times


def cpu_baseline(w, budget_s=20.0):
    """The oracle, as it stands, on a bounded sample: a lattice of the workload, a few steps."""
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    times = run_oracle_steps(w, 1, 0, threads)
    per = times[0]
    n = max(1, min(20, int((budget_s - (time.perf_counter() - t0)) / max(per, 1e-3))))
    times += run_oracle_steps(w, n, 0, threads) if n > 1 else []
    steps = len(times)
    tot = sum(times)
    one = run_oracle_steps(w, 2, 0, 1)  # the same sample on one core, two steps
    return {"value": w.ncells * steps / tot / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": "%s, %d time steps of the FP64 oracle (set-up excluded)" % (describe(w, w.params["q"]), steps),
            "one_core": {"value": w.ncells * len(one) / sum(one) / 1e6, "unit": "MLUPS", "cores": 1,
                         "sample": "the same lattice, %d time steps" % len(one)}}


def bench_reference(args, rank, world):
    if rank != 0:
        return 0
    w = workload(args.workload, args.precision, args.q, sample=True)
    full = workload(args.workload, args.precision, args.q)
    threads = os.cpu_count() or 1
    times = run_oracle_steps(w, args.steps, args.warmup, threads)
    tot = sum(times)
    value = w.ncells * len(times) / tot / 1e6
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": describe(full, args.q), "cells": full.ncells, "inputs_vs_l2": "CPU run"},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": "%s: %d time steps of the FP64 oracle (arithmetic and storage FP64) "
                                       "after %d warm-up steps" % (describe(w, args.q), args.steps, args.warmup)},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_batch(args, rank, world, local_rank):
    """64 independent two-sphere instances: one batched graph (the bulk lattice-Boltzmann pass of all
    instances in one persistent launch, tile shape from the autotuner) vs the instances run one after
    another.
    On several GPUs each rank runs its share of the instances (no collective on the data path); the
    time is the slowest rank's and the work is the total."""
    import torch

    torch.cuda.set_device(local_rank)
    import __graft_entry__

    if not os.path.exists(os.path.join(ROOT, "paper_1902_10432_gb300", "_lib", "libcbl.so")):
        __graft_entry__.build()
    from paper_1902_10432_gb300 import autotune, cbl, ranks, workloads

    rk = ranks.Ranks("nccl")
    ws_all = workloads.batch64(seed=0, prec=args.precision)
    ws = [ws_all[i] for i in ranks.shard(len(ws_all), rk.rank, rk.world)]
    cells_mine = sum(w.ncells for w in ws)
    sims = []
    choices = {}
    for w in ws:
        s = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
        workloads.build(s, w)
        c, _ = autotune.tune(s, steps=3)
        choices[json.dumps(c, sort_keys=True)] = choices.get(json.dumps(c, sort_keys=True), 0) + 1
        sims.append(s)
    # sequential: each instance alone, one after another
    for s in sims:
        s.step(args.warmup)
    torch.cuda.synchronize()
    rk.barrier()
    t0 = time.perf_counter()
    for s in sims:
        s.step(args.steps)
        torch.cuda.synchronize()
    seq_s = rk.max(time.perf_counter() - t0)
    batch = cbl.Batch(sims)
    tile, tile_ms = autotune.tune_batch(batch, steps=3)
    binfo = batch.info()
    batch.step(args.warmup)
    batch.sync()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.Stream()
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        rk.barrier()
        t1 = time.perf_counter()
        batch.step(args.steps)
        batch.sync()
        bat_s = time.perf_counter() - t1
        rk.barrier()
    bat_s = rk.max(bat_s)
    cells = rk.sum(cells_mine)
    value = cells * args.steps / bat_s / 1e6
    line = {"metric": "aggregate MLUPS (batched)", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * bat_s / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "fp16dev": "f16-storage/f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "batch64: 64 two-sphere instances, boxes U{64..128}^3, R U[10,24], "
                                   "liquid fraction U[0.01,0.2], angle U[30,90] deg, seed 0",
                       "cells": int(cells), "autotune_choices": choices,
                       "batch": {"mode": "persistent" if binfo["mode"] == 1 else "branch per instance",
                                 "tile": autotune.BATCH_TILES.get(binfo["tile"]), "work_items": binfo["items"],
                                 "grid_blocks": binfo["grid"],
                                 "tile_ms_per_step": {str(autotune.BATCH_TILES[k]): round(v, 3)
                                                      for k, v in tile_ms.items()}},
                       "parallelism": "instances sharded over %d GPUs" % world if world > 1 else "single GPU"},
            "sequential_mlups": cells * args.steps / seq_s / 1e6,
            "speedup_vs_sequential": seq_s / bat_s, "clocks": clk.summary(),
            # persistent mode: one launch for the bulk pass of all instances, then each instance's side
            # chain (its step without the density and bulk collision kernels)
            "gpu_launches": args.steps * ((1 + len(ws) * (kernels_per_step(2, 1, False) - 2)) if binfo["mode"] == 1
                                          else sum(n * kernels_per_step(2, 1, 1 if json.loads(c).get("lbm_variant") == 1 else 0)
                                                   for c, n in choices.items()))}
    if rk.root:
        print(json.dumps(line), flush=True)
    batch.close()
    return 0


def bench_surrogate(args, rank, world, local_rank):
    """Learned surrogate: data from batched two-sphere runs, GPU training, then the surrogate-driven
    advance of a 512^3 packing of 200 spheres against plain stepping over the same number of steps."""
    import torch

    torch.cuda.set_device(local_rank)
    import __graft_entry__

    if not os.path.exists(os.path.join(ROOT, "paper_1902_10432_gb300", "_lib", "libcbl.so")):
        __graft_entry__.build()
    from paper_1902_10432_gb300 import cbl, surrogate, workloads

    log = lambda m: print(m, file=sys.stderr, flush=True)
    t0 = time.perf_counter()
    ws = []
    for sd in range(args.sur_seeds):
        ws += workloads.batch64(seed=sd, prec="fp32", gap=(3.0, 7.0), fixed=True)
    X, Y, inst = surrogate.generate(ws, equil=args.sur_equil, hold=args.sur_hold, avg=args.sur_hold // 2,
                                    records=args.sur_records, dgap=args.sur_dgap, log=log)
    gen_s = time.perf_counter() - t0
    if args.sur_save:
        import numpy as np

        np.savez(args.sur_save, X=X, Y=Y, inst=inst)
    sur, tr = surrogate.train(X, Y, inst, iters=args.sur_iters, log=log)
    w, pairs, VL = workloads.packing(seed=0, L=args.sur_box, rho_s=args.sur_rho_s)
    R = [b["radius"] for b in w.bodies]
    dims = (w.nx, w.ny, w.nz)
    theta = w.meta["theta_deg"]
    # both runs start from the same state with the bridges formed (untimed)
    hyb = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(hyb, w)
    hyb.step(args.sur_pack_equil)
    torch.cuda.synchronize()
    res = surrogate.hybrid_run(hyb, sur, R, pairs, VL, theta, dims, windows=args.sur_windows, K=args.sur_k,
                               W=args.sur_w, log=log)
    hyb.close()
    del hyb
    plain = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(plain, w)
    plain.step(args.sur_pack_equil)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    plain.step(res["steps"])
    plain.total_mass()
    plain_s = time.perf_counter() - t1
    line = {"metric": "surrogate vs plain time-to-solution", "value": plain_s / res["wall_seconds"],
            "unit": "x (plain wall / surrogate wall)", "n_gpus": world, "steps": res["steps"], "warmup": 5,
            "higher_is_better": True, "dtype": "f32 populations, bf16 network", "data": "synthetic",
            "config": {"workload": "packing %d^3, %d spheres R U[12,20], %d bridged pairs, liquid 0.1 of solid"
                                   % (w.nx, len(R), len(pairs)),
                       "windows": args.sur_windows, "K_lbm": args.sur_k, "W_surrogate": args.sur_w,
                       "equilibration_steps": args.sur_pack_equil, "sphere_mass_density": args.sur_rho_s,
                       "training": "%d two-sphere instances (gap U[3,7]), fixed spheres moved by %g cells "
                                   "of gap per record, %d-step holds, force mean over the last half, up to %d "
                                   "records of both bodies while the bridge is intact"
                                   % (64 * args.sur_seeds, args.sur_dgap, args.sur_hold, args.sur_records)},
            "surrogate_wall_s": res["wall_seconds"], "plain_wall_s": plain_s,
            "force_rel_err_median": res["force_rel_err_median"], "force_rel_err_p95": res["force_rel_err_p95"],
            "corrected_force_rel_err_median": res.get("corrected_force_rel_err_median"),
            "corrected_force_rel_err_p95": res.get("corrected_force_rel_err_p95"),
            "force_rel_err_bodies": res["n_rel"],
            "force_err_over_2piRsigma_median": res["force_err_over_2piRsigma_median"],
            "force_err_over_2piRsigma_p95": res["force_err_over_2piRsigma_p95"],
            "training": tr, "samples": int(len(X)), "data_generation_s": gen_s}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def bench_cuda(args, rank, world, local_rank):
    import statistics

    import torch

    torch.cuda.set_device(local_rank)
    import __graft_entry__

    if not os.path.exists(os.path.join(ROOT, "paper_1902_10432_gb300", "_lib", "libcbl.so")):
        __graft_entry__.build()
    from paper_1902_10432_gb300 import cbl, ranks, workloads

    rk = ranks.Ranks("nccl")
    w = workload(args.workload, args.precision, args.q)
    prec = args.precision
    barrier = rk.barrier

    sim = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(sim, w)
    if args.lbm_variant is not None:
        sim.set_option("lbm_variant", args.lbm_variant)
    for kv in args.option:
        k, v = kv.split("=")
        sim.set_option(k, float(v))
    variant = int(sim.get_option("lbm_variant"))
    # the bulk collision's live duration, from event nodes inside the replayed step graph
    sim.set_option("kernel_events", 1)
    stream = sim.stream
    sim.step(args.warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed_once():
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        barrier()
        return rk.max(ev0.elapsed_time(ev1)), sim.kernel_times()

    reps, kern = [], []
    with ClockSampler(local_rank) as clk:
        t_ms, kt = timed_once()
        reps.append(t_ms)
        kern += kt
        # every rank takes the same repeat count (from the max over ranks of the first repeat): at
        # least min_repeats, about min_seconds of load, and no more than max_steps_total steps in all
        # (the workloads are dynamic: spheres pulled together by their bridges make contact after
        # some thousand steps, so the bench times the first few hundred steps)
        by_time = -(-args.min_seconds * 1e3 // max(t_ms, 1e-3))
        by_steps = (args.max_steps_total - args.warmup) // args.steps
        n_rep = int(max(args.min_repeats, min(args.max_repeats, by_time, by_steps)))
        for _ in range(n_rep - 1):
            t_ms, kt = timed_once()
            reps.append(t_ms)
            kern += kt
    ms_med = statistics.median(reps)
    value = world * w.ncells * args.steps / (ms_med * 1e-3) / 1e6
    t_kernel_ms = statistics.mean(kern)

    # per-phase durations (CUDA events between the phases, same stream, kernel-by-kernel launch)
    phases = sim.time_phases(max(3, min(args.steps, 20)))
    mass = sim.total_mass()
    err = sim.info()["device_error"]
    sim.close()
    del sim

    # end to end through the C ABI with host buffers: set-up from the host mask, K steps, fields back.
    # The input mask and the output fields live in pinned host memory, allocated before the timed
    # region as a caller that runs many jobs would keep them.
    import dataclasses

    import numpy as np

    pin = lambda n, dt: torch.empty(n, dtype=dt, pin_memory=True).numpy()
    mask_pinned = pin(w.ncells, torch.uint8)
    mask_pinned[:] = np.asarray(w.mask, np.uint8).reshape(-1)
    w_pinned = dataclasses.replace(w, mask=mask_pinned.reshape(np.asarray(w.mask).shape))
    out = (pin(w.ncells, torch.float64), pin(3 * w.ncells, torch.float64), pin(w.ncells, torch.float64))
    # three whole jobs, each timed on its own; the median is reported (the set-up's host work varies
    # from run to run by a few ms)
    e2e_runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        rk.barrier()
        t0 = time.perf_counter()
        s2 = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
        workloads.build(s2, w_pinned)
        if args.lbm_variant is not None:
            s2.set_option("lbm_variant", args.lbm_variant)
        s2.step(args.steps)
        rho, vel, phf = s2.fields(out=out)
        torch.cuda.synchronize()
        e2e_runs.append(rk.max(time.perf_counter() - t0))
        s2.close()
        del s2
    e2e_s = statistics.median(e2e_runs)
    h2d = w.ncells * 1  # the liquid mask uploaded by cbl_init_fluid (expanded to densities on the device)
    d2h = w.ncells * (8 + 24 + 8)

    if rank == 0:
        peak, peak_kind = measured_peaks()
        bpc = alg_bytes_per_cell(prec, args.q)
        achieved = bpc * w.ncells / (t_kernel_ms * 1e-3) / 1e9
        step_achieved = bpc * w.ncells / (ms_med / args.steps * 1e-3) / 1e9
        step_traffic = profiled_step_traffic(w.name, prec, args.q)
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_med / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "fp16dev": "f16-storage/f32"}[prec], "data": "synthetic",
            "config": {"workload": describe(w, args.q), "cells": w.ncells, "seed": w.meta.get("seed"),
                       "inputs_vs_l2": "populations 2 x %.0f MB > 129 MB L2 (no flush needed)"
                                       % (w.ncells * args.q * POP_BYTES[prec] / 1e6),
                       "timing": "median of %d repeats of %d steps (CUDA events on the step stream)"
                                 % (len(reps), args.steps),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "repeats_ms": [round(x, 4) for x in reps],
            "roofline": {"bound": "hbm", "kernel": {0: "bulk collision (k_collide: pull, force, BGK, store)",
                                                    1: "fused pass (k_fused: psi of the plane ahead, collision)",
                                                    2: "accumulating collision (k_collide_acc: collision and "
                                                       "next step's density)"}[variant],
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": profiled_traffic(w.name, prec, args.q), "peak_kind": peak_kind,
                         "peak_datasheet": HBM_DATASHEET_GBS, "alg_bytes_per_cell": bpc,
                         "kernel_ms": t_kernel_ms, "kernel_launches_timed": len(kern),
                         "step": {"achieved": step_achieved, "frac": step_achieved / peak,
                                  "traffic": step_traffic,
                                  "traffic_over_alg": None if step_traffic is None
                                  else step_traffic / (bpc * w.ncells)}},
            "phases_ms": {k: round(v, 5) for k, v in phases.items()},
            "gpu_launches": kernels_per_step(len(w.bodies), w.params.get("mpf_kinetics", 1),
                                             variant) * args.steps * len(reps),
            "clocks": clk.summary(),
            "e2e": {"value": world * w.ncells * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "what": "create + bodies + init from the host mask + K steps + fields to host (pinned host "
                            "buffers), wall clock, median of 3 jobs",
                    "runs_s": [round(x, 5) for x in e2e_runs]},
            "fluid_mass": mass, "device_error": err,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(workload(args.workload, "fp64", args.q, sample=True))
        print(json.dumps(line), flush=True)
    rk.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16dev"])
    ap.add_argument("--q", type=int, default=19, choices=[19, 27], help="velocity set: D3Q19 or D3Q27")
    ap.add_argument("--workload", default="tetra4",
                    choices=["spheres2", "plates48", "tetra4", "batch64", "surrogate"])
    ap.add_argument("--sur-equil", type=int, default=800)
    ap.add_argument("--sur-seeds", type=int, default=2, help="64-instance batches of training runs")
    ap.add_argument("--sur-records", type=int, default=80)
    ap.add_argument("--sur-hold", type=int, default=150)
    ap.add_argument("--sur-dgap", type=float, default=-0.04)
    ap.add_argument("--sur-rho-s", type=float, default=200.0)
    ap.add_argument("--sur-iters", type=int, default=3000)
    ap.add_argument("--sur-box", type=int, default=512)
    ap.add_argument("--sur-windows", type=int, default=4)
    ap.add_argument("--sur-k", type=int, default=100)
    ap.add_argument("--sur-w", type=int, default=200)
    ap.add_argument("--sur-pack-equil", type=int, default=1000)
    ap.add_argument("--sur-save", default="", help="write the training samples to this .npz")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--min-repeats", type=int, default=5)
    ap.add_argument("--max-repeats", type=int, default=200)
    ap.add_argument("--min-seconds", type=float, default=2.0,
                    help="repeat the timed region until about this much load has passed")
    ap.add_argument("--max-steps-total", type=int, default=600,
                    help="cap on warm-up plus timed steps (the workloads evolve with time)")
    ap.add_argument("--option", action="append", default=[],
                    help="execution option key=value for the timed simulation (cbl_set_option), repeatable")
    ap.add_argument("--lbm-variant", type=int, default=None, choices=[0, 1, 2],
                    help="lattice-Boltzmann pass: 0 split density + collision, 1 fused, 2 accumulating "
                         "(default: the library's)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return bench_reference(args, rank, world)
    if args.workload == "batch64":
        return bench_batch(args, rank, world, local_rank)
    if args.workload == "surrogate":
        return bench_surrogate(args, rank, world, local_rank)
    return bench_cuda(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
