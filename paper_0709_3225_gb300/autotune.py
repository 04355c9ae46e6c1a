"""Autotuner for the force kernels' launch choices.

It picks, by timing velocity-Verlet steps on a copy of the state:
  single systems  -- force kernel (warp-per-cell with the velocity-Verlet
                     update separate or fused into it, run kernel with
                     bulk-copy staging, run kernel reading global memory) and the
                     smallest lane-group width of the warp kernel (threads
                     per cell: the group of lanes that owns a cell's
                     particles);
  batches         -- cells per pull from the work counter, lane-group width,
                     graph replay or direct launches.
Choices are cached in a JSON file keyed by (GPU name, kind, N bucket, density
bucket) and re-applied without timing on a cache hit.  The cache lives at
$LJGB_TUNE_CACHE, else ~/.cache/ljgb/autotune.json.

The paper tuned its block size by hand (n_B = 64 in Section 2.1); this does
the equivalent search for the GB300 kernels.  All timed work runs through
the library's entry points on the context's stream.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import lj

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("LJGB_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "ljgb",
                                                             "autotune.json")


def bucket_key(kind: str, n: int, rho: float, gpu: str | None = None) -> str:
    """Cache key: GPU name, kind, log2(N) rounded, density to 0.05."""
    if gpu is None:
        gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    nb = int(round(math.log2(max(n, 1))))
    rb = round(round(rho / 0.05) * 0.05, 2)
    return f"{gpu}|{kind}|N2^{nb}|rho{rb:.2f}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(key: str, value: dict, path: str | None = None) -> None:
    path = path or cache_path()
    with _lock:
        data = load_cache(path)
        data[key] = value
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _time_steps(run, steps: int, warmup: int) -> float:
    """Milliseconds per step of run(k) over `steps`, after `warmup`."""
    run(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run(steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def system_candidates(precision: str) -> list[dict]:
    if precision == "fp64":
        return [{"kernel": 1, "gmin": 0, "grab": 0}, {"kernel": 2, "gmin": 0, "grab": 0}]
    warp = [{"kernel": 3, "gmin": g, "grab": c} for g in (0, 16) for c in (0, 1, 4)]
    return warp + [{"kernel": 3, "gmin": 32, "grab": 0}, {"kernel": 0, "gmin": 0, "grab": 1},
                   {"kernel": 1, "gmin": 0, "grab": 0}, {"kernel": 2, "gmin": 0, "grab": 0}]


def tune_system(system: lj.System, rho: float, steps: int = 10, warmup: int = 3, use_cache: bool = True,
                path: str | None = None) -> dict:
    """Choose and apply the fastest force-kernel setting for ``system``."""
    precision = "fp64" if system.params.precision == lj.LJ_PREC_FP64 else "mixed"
    key = bucket_key(f"system-{precision}", system.n, rho)
    if use_cache:
        hit = load_cache(path).get(key)
        if hit:
            lj.lj_set_tuning(system.ctx, hit["kernel"], hit["gmin"], hit.get("grab", 0))
            return dict(hit, cached=True)
    x, v, f = system.x.clone(), system.v.clone(), system.f.clone()
    lj.lj_forces(system.ctx, x, f)
    results = []
    for cand in system_candidates(precision):
        lj.lj_set_tuning(system.ctx, cand["kernel"], cand["gmin"], cand["grab"])
        ms = _time_steps(lambda k: lj.lj_step(system.ctx, x, v, f, k), steps, warmup)
        results.append(dict(cand, ms_per_step=ms))
    lj.lj_check(system.ctx)
    best = min(results, key=lambda r: r["ms_per_step"])
    lj.lj_set_tuning(system.ctx, best["kernel"], best["gmin"], best["grab"])
    choice = {"kernel": best["kernel"], "gmin": best["gmin"], "grab": best["grab"],
              "ms_per_step": best["ms_per_step"]}
    store_cache(key, choice, path)
    return dict(choice, cached=False, trials=results)


def batch_candidates() -> list[dict]:
    out = [{"cells_per_grab": c, "gmin": g, "graph": True} for c in (1, 2, 4, 8, 16) for g in (0, 16)]
    out.append({"cells_per_grab": 4, "gmin": 0, "graph": False})
    return out


def tune_batch(batch: lj.Batch, rho: float, steps: int = 10, warmup: int = 3, use_cache: bool = True,
               path: str | None = None) -> dict:
    """Choose and apply the fastest batch setting for ``batch``."""
    key = bucket_key(f"batch{batch.nrep}", batch.ntot, rho)
    if use_cache:
        hit = load_cache(path).get(key)
        if hit:
            batch.set_tuning(hit["cells_per_grab"], hit["graph"], hit["gmin"])
            return dict(hit, cached=True)
    saved = (batch.x.clone(), batch.v.clone(), batch.f.clone(), batch._forces_valid)
    results = []
    for cand in batch_candidates():
        batch.set_tuning(cand["cells_per_grab"], cand["graph"], cand["gmin"])
        ms = _time_steps(batch.step, steps, warmup)
        results.append(dict(cand, ms_per_step=ms))
    batch.check()
    batch.x.copy_(saved[0])
    batch.v.copy_(saved[1])
    batch.f.copy_(saved[2])
    batch._forces_valid = saved[3]
    best = min(results, key=lambda r: r["ms_per_step"])
    batch.set_tuning(best["cells_per_grab"], best["graph"], best["gmin"])
    choice = {k: best[k] for k in ("cells_per_grab", "gmin", "graph", "ms_per_step")}
    store_cache(key, choice, path)
    return dict(choice, cached=False, trials=results)
