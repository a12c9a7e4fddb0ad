"""Project autotuner: picks the execution variant of the lattice kernels for a lattice shape, and the
tile shape of the persistent batch kernel for a batch.

Candidates for one lattice: the split density + collision kernels with 128-thread blocks of x extent
32, 64 or 128, the fused single pass, and the accumulating pass with regions 8 or 16 rows deep. For a batch (tune_batch): the persistent kernel's tile
shapes 32x4x1, 32x4x4, 32x4x8 and 64x2x4 cells. Each candidate is timed on the simulation it will run
(three warm-up steps, then CUDA events around a few steps on the simulation's stream; the state
advances, which does not matter for the choice); the fastest is applied and cached in a JSON file
keyed by lattice shape, precision, whether bodies are present and the GPU name.
"""
from __future__ import annotations

import json
import os
import threading

CACHE = os.environ.get("CBL_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json"))
_lock = threading.Lock()


def candidates(prec):
    c = [dict(lbm_variant=0, lbm_block_x=bx) for bx in (32, 64, 128)]
    c.append(dict(lbm_variant=1, lbm_block_x=32))
    c += [dict(lbm_variant=2, lbm_block_x=32, acc_ty=ty) for ty in (8, 16)]
    return c


def _key(sim):
    import torch

    nx = sim.shape[2]
    ny = sim.shape[1]
    nz = sim.shape[0]
    return "%dx%dx%d/%s/%s/%s" % (nx, ny, nz, sim.params["prec"], "bodies" if sim.nb else "fluid",
                                  torch.cuda.get_device_name())


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def apply(sim, choice):
    for k, v in choice.items():
        sim.set_option(k, v)


def tune(sim, steps=6, use_cache=True):
    """Time the candidates on `sim` and apply the fastest. Returns (choice, {candidate: ms/step})."""
    import torch

    key = _key(sim)
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        apply(sim, cache[key]["choice"])
        return cache[key]["choice"], cache[key]["ms"]
    results = {}
    best, best_ms = None, float("inf")
    s = sim.stream
    for cand in candidates(sim.params["prec"]):
        apply(sim, cand)
        sim.step(3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        sim.step(steps)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        results[json.dumps(cand, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = cand, ms
    apply(sim, best)
    if use_cache:
        with _lock:
            cache = _load()
            cache[key] = {"choice": best, "ms": results}
            tmp = CACHE + ".tmp.%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(tmp, CACHE)
    return best, results


BATCH_TILES = {0: (32, 4, 1), 1: (32, 4, 4), 2: (32, 4, 8), 3: (64, 2, 4)}


def tune_batch(batch, steps=4):
    """Time the persistent kernel's tile shapes on `batch` (its instances advance) and keep the
    fastest. Returns (tile, {tile: ms/step})."""
    import time

    if batch.info()["mode"] != 1:
        return None, {}
    results = {}
    for t in BATCH_TILES:
        batch.set_option("tile", t)
        batch.step(2)
        batch.sync()
        t0 = time.perf_counter()
        batch.step(steps)
        batch.sync()
        results[t] = (time.perf_counter() - t0) * 1e3 / steps
    best = min(results, key=results.get)
    batch.set_option("tile", best)
    return best, results
