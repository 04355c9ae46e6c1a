"""Autotuner for the force kernels' launch choices.

It picks, by timing velocity-Verlet steps on a copy of the state:
  single systems  -- cell subdivision k (cell side >= rc / k: 1, the 27-cell
                     stencil, or 2, the 125-cell stencil of half-size cells),
                     force kernel (warp-per-cell over the half stencil
                     with each pair once, warp-per-cell over the 27-cell
                     stencil with the velocity-Verlet
                     update separate or fused into it, run kernel with
                     bulk-copy staging, run kernel reading global memory,
                     the paper's fixed-capacity cell arrays, the warp kernel
                     with bulk-copied stencils, the warp kernel with each
                     step one persistent launch; FP64: the FP64 warp kernel
                     or the run kernels),
                     the lane-group width of the warp kernel (home particles
                     per chunk; 0 = compiled default, -1 = chosen per cell)
                     and the cells per pull
                     from its work counter (0 = static striding);
  batches         -- cell subdivision k (1 or 2, as for single systems, timed
                     on a copy of the state), cells per pull from the work
                     counter, lane-group width, graph replay or direct
                     launches.
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
        # the warp kernel with compacted pair lists, and the two run kernels
        return ([{"subdiv": 1, "kernel": 3, "gw": 0, "grab": c} for c in (1, 4)] +
                [{"subdiv": 1, "kernel": k, "gw": 0, "grab": 0} for k in (1, 2)])
    warp = [{"subdiv": 1, "kernel": 3, "gw": g, "grab": c} for g in (0, -1, 8, 32) for c in (0, 4)]
    n3 = [{"subdiv": 1, "kernel": 7, "gw": 0, "grab": c} for c in (0, 1, 4)]
    return n3 + warp + [{"subdiv": 1, "kernel": 0, "gw": 0, "grab": 4}, {"subdiv": 1, "kernel": 1, "gw": 0, "grab": 0},
                   {"subdiv": 1, "kernel": 2, "gw": 0, "grab": 0}, {"subdiv": 1, "kernel": 4, "gw": 0, "grab": 0},
                   {"subdiv": 1, "kernel": 5, "gw": 0, "grab": 4}, {"subdiv": 1, "kernel": 6, "gw": 0, "grab": 1},
                   {"subdiv": 1, "kernel": 6, "gw": 0, "grab": 4},
                   {"subdiv": 2, "kernel": 3, "gw": 0, "grab": 4}, {"subdiv": 2, "kernel": 3, "gw": 2, "grab": 4}]


def _apply(system: lj.System, choice: dict) -> None:
    lj.lj_set_tuning(system.ctx, choice["kernel"], choice["gw"], choice["grab"])


def _clone_system(system: lj.System, subdiv: int) -> lj.System:
    p = system.params
    prec = "fp64" if p.precision == lj.LJ_PREC_FP64 else "mixed"
    return lj.System(system.x.cpu().numpy(), system.v.cpu().numpy(), p.box, eps=p.eps, sigma=p.sigma, rc=p.rc,
                     dt=p.dt, mass=p.mass, shift_mode=p.shift_mode, precision=prec, flags=p.flags,
                     cell_subdiv=subdiv, device=system.x.device)


def tune_system(system: lj.System, rho: float, steps: int = 10, warmup: int = 3, use_cache: bool = True,
                path: str | None = None) -> dict:
    """Time every candidate setting and apply the fastest one that ``system``
    can take.  A subdivision other than the system's is timed on a temporary
    copy; when it wins, the returned choice names it (``make_system`` then
    builds the system with it) and ``system`` gets the best setting of its own
    subdivision."""
    precision = "fp64" if system.params.precision == lj.LJ_PREC_FP64 else "mixed"
    key = bucket_key(f"system-{precision}", system.n, rho)
    own = system.params.cell_subdiv or 1
    if use_cache:
        hit = load_cache(path).get(key)
        if hit and hit.get("subdiv", 1) == own:
            _apply(system, hit)
            return dict(hit, cached=True)
    results = []
    copies = {own: system}
    try:
        for cand in system_candidates(precision):
            sub = cand["subdiv"]
            if sub not in copies:
                try:
                    copies[sub] = _clone_system(system, sub)
                except lj.LJError:      # box too small for that subdivision
                    copies[sub] = None
            target = copies[sub]
            if target is None:
                continue
            x, v, f = target.x.clone(), target.v.clone(), target.f.clone()
            _apply(target, cand)
            try:
                lj.lj_forces(target.ctx, x, f)
                ms = _time_steps(lambda k: lj.lj_step(target.ctx, x, v, f, k), steps, warmup)
                lj.lj_check(target.ctx)
            except lj.LJError as err:   # e.g. a cell over the fixed AOP capacity
                results.append(dict(cand, ms_per_step=float("inf"), error=str(err)))
                continue
            results.append(dict(cand, ms_per_step=ms))
    finally:
        for sub, t in copies.items():
            if sub != own and t is not None:
                t.close()
    best = min(results, key=lambda r: r["ms_per_step"])
    best_own = min((r for r in results if r["subdiv"] == own), key=lambda r: r["ms_per_step"])
    _apply(system, best_own)
    choice = {k: best[k] for k in ("subdiv", "kernel", "gw", "grab", "ms_per_step")}
    store_cache(key, choice, path)
    return dict(choice, cached=False, trials=results)


def make_system(x, v, box: float, rho: float, *, use_cache: bool = True, path: str | None = None, **kw):
    """A tuned lj.System for (x, v, box): built with the subdivision the
    tuner chose (timing once if the cache has no entry), tuning applied.
    Returns (system, choice)."""
    precision = kw.get("precision", "mixed")
    if use_cache:
        hit = load_cache(path).get(bucket_key(f"system-{precision}", int(len(x)), rho))
        if hit:
            s = lj.System(x, v, box, cell_subdiv=hit.get("subdiv", 1), **kw)
            _apply(s, hit)
            return s, dict(hit, cached=True)
    s = lj.System(x, v, box, **kw)
    choice = tune_system(s, rho, use_cache=False, path=path)
    if choice.get("subdiv", 1) != (s.params.cell_subdiv or 1):
        s.close()
        s = lj.System(x, v, box, cell_subdiv=choice["subdiv"], **kw)
        _apply(s, choice)
    return s, choice


def batch_candidates() -> list[dict]:
    """Batch settings: cell subdivision k (1: 27-cell stencil; 2: half-size
    cells, 125-cell stencil, group width 4 compiled in), force kernel (7:
    each pair once, k = 1 only; 3: the 27-cell code), cells per pull,
    lane-group width, graph replay."""
    out = [{"subdiv": 1, "kernel": 7, "cells_per_grab": c, "gw": 0, "graph": True} for c in (1, 2, 4, 8)]
    out.append({"subdiv": 1, "kernel": 7, "cells_per_grab": 4, "gw": 0, "graph": False})
    out += [{"subdiv": 1, "kernel": 3, "cells_per_grab": c, "gw": g, "graph": True} for c in (1, 2, 4, 8, 16)
            for g in (0, 8, -1)]
    out += [{"subdiv": 2, "kernel": 3, "cells_per_grab": c, "gw": g, "graph": True} for c in (1, 4, 16)
            for g in (0, 2, -1)]
    return out


def _batch_state(batch: lj.Batch):
    x, v = batch.x.cpu().numpy(), batch.v.cpu().numpy()
    o = batch.offsets
    return [x[o[r]:o[r + 1]] for r in range(batch.nrep)], [v[o[r]:o[r + 1]] for r in range(batch.nrep)]


def _clone_batch(batch: lj.Batch, subdiv: int) -> lj.Batch:
    xs, vs = _batch_state(batch)
    p = batch.params
    return lj.Batch(xs, vs, batch.boxes, eps=p.eps, sigma=p.sigma, rc=p.rc, dt=p.dt, mass=p.mass,
                    shift_mode=p.shift_mode, cell_subdiv=subdiv)


def tune_batch(batch: lj.Batch, rho: float, steps: int = 10, warmup: int = 3, use_cache: bool = True,
               path: str | None = None) -> dict:
    """Time every batch setting and apply the fastest one ``batch`` can take.
    A cell subdivision other than the batch's is timed on a temporary copy of
    the state; when it wins, the returned choice names it (``batch_for``
    then builds the batch with it) and ``batch`` gets the best setting of its
    own subdivision."""
    key = bucket_key(f"batch{batch.nrep}", batch.ntot, rho)
    own = batch.cell_subdiv
    if use_cache:
        hit = load_cache(path).get(key)
        if hit and hit.get("subdiv", 1) == own:
            batch.set_kernel(hit.get("kernel", 3))
            batch.set_tuning(hit["cells_per_grab"], hit["graph"], hit["gw"])
            return dict(hit, cached=True)
    results = []
    copies = {own: batch}
    try:
        for cand in batch_candidates():
            sub = cand["subdiv"]
            if sub not in copies:
                try:
                    copies[sub] = _clone_batch(batch, sub)
                    copies[sub].forces()
                except lj.LJError:      # a replica too small for that subdivision
                    copies[sub] = None
            target = copies[sub]
            if target is None:
                continue
            saved = (target.x.clone(), target.v.clone(), target.f.clone(), target._forces_valid)
            target.set_kernel(cand.get("kernel", 3))
            target.set_tuning(cand["cells_per_grab"], cand["graph"], cand["gw"])
            ms = _time_steps(target.step, steps, warmup)
            target.check()
            target.x.copy_(saved[0])
            target.v.copy_(saved[1])
            target.f.copy_(saved[2])
            target._forces_valid = saved[3]
            results.append(dict(cand, ms_per_step=ms))
    finally:
        for sub, t in copies.items():
            if sub != own and t is not None:
                t.close()
    best = min(results, key=lambda r: r["ms_per_step"])
    best_own = min((r for r in results if r["subdiv"] == own), key=lambda r: r["ms_per_step"])
    batch.set_kernel(best_own.get("kernel", 3))
    batch.set_tuning(best_own["cells_per_grab"], best_own["graph"], best_own["gw"])
    choice = {k: best[k] for k in ("subdiv", "kernel", "cells_per_grab", "gw", "graph", "ms_per_step")}
    store_cache(key, choice, path)
    return dict(choice, cached=False, trials=results)


def batch_for(batch: lj.Batch, choice: dict) -> lj.Batch:
    """``batch`` if the choice has its cell subdivision, else a new batch of the
    same state with the chosen subdivision and setting (``batch`` is closed)."""
    if choice.get("subdiv", 1) == batch.cell_subdiv:
        return batch
    nb = _clone_batch(batch, choice["subdiv"])
    batch.close()
    nb.set_kernel(choice.get("kernel", 3) if choice["subdiv"] == 1 else 3)
    nb.set_tuning(choice["cells_per_grab"], choice["graph"], choice["gw"])
    nb.forces()
    return nb
