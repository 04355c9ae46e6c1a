"""Benchmark: velocity-Verlet MD steps/s of the 4,000,000-particle LJ fluid.

One step = the whole hot path: kick + drift + wrap + cell binning (count,
scan, scatter) + cell-list LJ forces + closing kick, FP32-mixed precision.
Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the path needs no exchange between replicas); value = all ranks'
steps / max-over-ranks time.  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LJ steps/s & pair-interactions/s at N=4M, FP32-mixed vs FP64, % FP32 peak"
WORKLOAD = "fluid-4m"
FLOPS_PER_PAIR = 20          # flop convention per in-range pair evaluation
FP32_LANES, SM_MAX_MHZ = 128, 2070.0   # for the derived cross-check beside the measured peak


def measure_peaks() -> dict:
    """FP32 and FP64 FMA peaks measured on this device at its current clocks
    (lj_measure_peak: chains of FMAs on every SM), with the SM count queried
    from the device and the datasheet-style derivation beside them as a
    cross-check."""
    from paper_0709_3225_gb300 import lj
    fp32, ms32, nsm = lj.lj_measure_peak(lj.PEAK_FP32)
    fp32x2, ms32x2, _ = lj.lj_measure_peak(lj.PEAK_FP32X2)
    fp64, ms64, _ = lj.lj_measure_peak(lj.PEAK_FP64)
    return {"fp32_tflops": max(fp32, fp32x2) / 1e12, "fp32_scalar_tflops": fp32 / 1e12,
            "fp32_packed_tflops": fp32x2 / 1e12, "fp64_tflops": fp64 / 1e12, "sms": nsm,
            "launch_ms": {"fp32": ms32, "fp32x2": ms32x2, "fp64": ms64},
            "derived_fp32_tflops": nsm * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12,
            "how": "lj_measure_peak: 8 independent FMA chains per thread, 8 CTAs x 256 threads per SM, "
                   "launch lengthened to >= 20 ms, fastest of 3 (CUDA events); FP32 = max(scalar fmaf, "
                   "packed __ffma2_rn)"}


def unique_pairs(n: int, rho: float, rc: float) -> float:
    """Expected unique pairs within rc of a homogeneous fluid: N (2/3) pi rc^3 rho."""
    return n * (2.0 / 3.0) * math.pi * rc ** 3 * rho


CANDIDATE_FLOPS = 7          # flop convention per candidate distance test


def stencil_candidates(ctx) -> float:
    """Candidate pairs the full (2k+1)^3 stencil presents in one force
    evaluation, sum_c n_c * sum_{c' in stencil(c)} n_c', from the cell counts
    of the context's last binning (both directions, self pairs included)."""
    import torch
    from paper_0709_3225_gb300 import lj
    nc = ctx.nc
    count = torch.empty(nc ** 3, dtype=torch.int32, device="cuda")
    lj.lj_get_cells(ctx, count=count)
    return candidate_pairs(count.double().view(nc, nc, nc), ctx.params.cell_subdiv or 1)


def half_stencil_candidates(ctx) -> float:
    """Candidate pairs the half stencil presents when each pair is taken
    once: sum_c n_c (n_c - 1) / 2 + sum_c n_c * sum_{13 forward c'} n_c',
    from the cell counts of the context's last binning."""
    import torch
    from paper_0709_3225_gb300 import lj
    nc = ctx.nc
    count = torch.empty(nc ** 3, dtype=torch.int32, device="cuda")
    lj.lj_get_cells(ctx, count=count)
    g = count.double().view(nc, nc, nc)
    nb = torch.zeros_like(g)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) > (0, 0, 0):
                    nb += torch.roll(g, shifts=(-dz, -dy, -dx), dims=(0, 1, 2))
    return float((g * (g - 1) / 2).sum() + (g * nb).sum())


def candidate_pairs(g, k: int) -> float:
    """sum_c g[c] * sum_{|d|_inf <= k} g[c + d] over a periodic grid of counts."""
    import torch
    nb = torch.zeros_like(g)
    for dz in range(-k, k + 1):
        for dy in range(-k, k + 1):
            for dx in range(-k, k + 1):
                nb += torch.roll(g, shifts=(dz, dy, dx), dims=(0, 1, 2))
    return float((g * nb).sum())


def pinned_link_gbs(nbytes: int = 256 << 20) -> dict:
    """Host-device bandwidth of one pinned copy each way (best of 5, CUDA
    events): the rate the end-to-end figure's copies run at."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, dst, src in (("h2d", d, h), ("d2h", h, d)):
        best = float("inf")
        for _ in range(5):
            torch.cuda.synchronize()
            ev0.record()
            dst.copy_(src, non_blocking=True)
            ev1.record()
            torch.cuda.synchronize()
            best = min(best, ev0.elapsed_time(ev1))
        out[name] = nbytes / (best * 1e-3) / 1e9
    return out


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [q.strip() for q in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        mx = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] > 0.5 * mx] or rows
        reasons = set()
        for r in rows:
            for name, flag in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                  r[2:]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    """The largest value over the ranks (NCCL on GPUs, gloo on the CPU)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank: float, seconds_this_rank: float) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time.  Returns (rate, max seconds)."""
    t = max_over_ranks(world, seconds_this_rank)
    return world * units_per_rank / t, t


def run_ensemble(args, stream, world):
    """The batched workload: 256 replicas, N_r uniform in [500, 50000], rho_r
    in [0.7, 0.9], T_r in [0.7, 1.5]; 50 capped steepest-descent steps and
    autotuning (untimed), then steps timed with CUDA events, one cooperative
    launch per step (graph-replayed)."""
    import torch
    from paper_0709_3225_gb300 import autotune, inputs, lj
    e = inputs.ensemble()
    xs, vs = inputs.ensemble_state(e)
    b = lj.Batch(xs, vs, e.box)
    b.relax(50, 1e-3, 0.05)
    b.forces()
    tuning = autotune.tune_batch(b, float(np.mean(e.rho)))
    trials = tuning.pop("trials", None) or []
    b = autotune.batch_for(b, tuning)
    # the cell-size dimension of the tuning: the fastest setting per subdivision
    by_k = {}
    for t in trials:
        if t["subdiv"] not in by_k or t["ms_per_step"] < by_k[t["subdiv"]]["ms_per_step"]:
            by_k[t["subdiv"]] = t
    tuning["best_per_subdiv"] = {str(k): v for k, v in sorted(by_k.items())}
    b.step(args.warmup)
    b.check()
    k = max(10, min(args.steps, 200))
    n0, _ = b.launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    ev0.record(stream)
    b.step(k)
    ev1.record(stream)
    torch.cuda.synchronize()
    b.check()
    n1, graph = b.launches()
    ms = max_over_ranks(world, ev0.elapsed_time(ev1)) / k
    pairs = float(sum(unique_pairs(int(n), float(r), 2.5) for n, r in zip(e.n, e.rho)))
    info = b.info()
    b.close()
    return {"workload": "ensemble-256", "replicas": int(b.nrep), "n_total": int(info["ntot"]),
            "cells_total": int(info["ncell"]), "steps": k, "ms_per_step": ms,
            "value": world * 1e3 / ms, "unit": "ensemble steps/s",
            "replica_steps_per_s": world * b.nrep * 1e3 / ms,
            "pair_interactions_per_s": world * pairs * 1e3 / ms,
            "launches_per_step": (n1 - n0 - 1) / k, "graph": graph, "tuning": tuning}


def run_n2_breakeven(stream):
    """All-pairs (lj_forces_n2) against cell-list (lj_forces) force time,
    FP32-mixed, liquid-density lattice gases of growing N: where the cell
    list overtakes the paper's N^2 algorithm on this GPU."""
    import torch
    from paper_0709_3225_gb300 import inputs, lj
    out = []
    for n in (500, 2048, 8788, 32000, 131072):
        x, L = inputs.lattice_gas(n, 0.8442, 5)
        s = lj.System(x, None, L)
        row = {"n": n}
        for name, fn in (("cells_ms", lj.lj_forces), ("n2_ms", lj.lj_forces_n2)):
            reps = 3 if (name == "n2_ms" and n > 30000) else 20
            fn(s.ctx, s.x, s.f)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn(s.ctx, s.x, s.f)
            e1.record(stream)
            torch.cuda.synchronize()
            row[name] = e0.elapsed_time(e1) / reps
        s.check()
        s.close()
        out.append(row)
    return out


def run_rand48(stream, hbm_gbs):
    """Section 4's generator: the first R S numbers of the lrand48 series from
    S parallel streams (device-resident output, as the paper stored it),
    against the measured HBM copy bandwidth (4 bytes written per number)."""
    import torch
    from paper_0709_3225_gb300 import lj
    S, R = 152 * 4096, 512
    st = torch.empty(S, dtype=torch.int64, device="cuda")
    out = torch.empty(S * R, dtype=torch.int32, device="cuda")
    outd = torch.empty(S * R, dtype=torch.float64, device="cuda")
    lj.lj_rand48_seed(st, lj.lj_srand48_state(12345))
    lj.lj_rand48_lrand(st, R, out)
    res = {"streams": S, "per_stream": R, "numbers": S * R}
    for name, fn, buf, nb in (("lrand48", lj.lj_rand48_lrand, out, 4), ("drand48", lj.lj_rand48_drand, outd, 8)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            fn(st, R, buf)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        gbs = S * R * nb / ms / 1e6
        res[name] = {"ms": ms, "numbers_per_s": S * R / ms * 1e3, "GB_per_s": gbs,
                     "frac_of_hbm": gbs / hbm_gbs if hbm_gbs else None}
    del out, outd
    return res


def run_langevin(x, v, L, w, stream):
    """The Langevin-thermostatted step (BAOAB, rand48 normals) on the 4M
    workload: ms per step beside the plain velocity-Verlet step."""
    import torch
    from paper_0709_3225_gb300 import lj
    s = lj.System(x, v, L, precision="mixed", dt=w.dt, rc=w.rc)
    s.forces()
    lj.lj_langevin_seed(s.ctx, 7)
    lj.lj_langevin_step(s.ctx, s.x, s.v, s.f, 3, 1.0, w.temperature)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = 20
    e0.record(stream)
    lj.lj_langevin_step(s.ctx, s.x, s.v, s.f, k, 1.0, w.temperature)
    e1.record(stream)
    torch.cuda.synchronize()
    s.check()
    s.close()
    return {"ms_per_step": e0.elapsed_time(e1) / k, "steps": k, "gamma": 1.0, "kT": w.temperature,
            "scheme": "BAOAB, Box-Muller normals from the rand48 series (one stream per particle)"}


def run_aop_density(stream):
    """The paper's density study (Section 3.2): force time at fixed N =
    131,072 over densities 0.2 .. 1.0 for the fixed-capacity cell arrays
    (kernel 4, the paper's layout: work per cell fixed, so time follows the
    number of cells) and the default CSR warp kernel (time follows the pair
    count)."""
    import torch
    from paper_0709_3225_gb300 import inputs, lj
    out = []
    for rho in (0.2, 0.4, 0.6, 0.8, 1.0):
        x, L = inputs.lattice_gas(131072, rho, 17)
        s = lj.System(x, None, L)
        row = {"rho": rho, "cells": s.ctx.nc ** 3, "mean_per_cell": 131072 / s.ctx.nc ** 3}
        for name, kern in (("csr_ms", 3), ("aop_ms", 4)):
            lj.lj_set_tuning(s.ctx, kern)
            s.forces()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(20):
                s.forces()
            e1.record(stream)
            torch.cuda.synchronize()
            row[name] = e0.elapsed_time(e1) / 20
        s.check()
        s.close()
        out.append(row)
    return out


def run_graph_small(stream, steps=200):
    """Small systems, where launches rather than the GPU bound a step: ms per
    step with direct launches, with graph replay of the middle steps
    (lj_set_graph), and with each step one persistent cooperative launch
    (lj_set_tuning kernel 6), for the 2,048- and 131,072-particle fluids."""
    import torch
    from paper_0709_3225_gb300 import inputs, lj
    out = []
    for name in ("fluid-2k", "fluid-131k"):
        x, v, L, w = inputs.workload_state(name)
        row = {"workload": name, "n": w.n}
        for label, graph, kernel in (("direct", False, 3), ("graph", True, 3), ("persistent", True, 6)):
            s = lj.System(x, v, L, dt=w.dt, rc=w.rc)
            lj.lj_set_graph(s.ctx, graph)
            lj.lj_set_tuning(s.ctx, kernel, 0, 1 if kernel == 6 else 4)
            s.forces()
            s.step(10)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            s.check()
            s.close()
            row[f"{label}_ms_per_step"] = e0.elapsed_time(e1) / steps
        out.append(row)
    return out


def run_accuracy_131k(with_oracle: bool, max_oracle_s: float = 60.0):
    """The 131,072-particle fluid (FCC 4*32^3 start, T = 0.728): the force
    error of both GPU paths against the FP64 oracle at the start, and the
    total-energy drift per particle over 1000 velocity-Verlet steps of the
    FP32-mixed and FP64 GPU paths and, with with_oracle, of the oracle itself
    (on the host cores, stopped early and scaled if it would pass
    max_oracle_s)."""
    import torch
    from paper_0709_3225_gb300 import inputs, lj
    x, v, L, w = inputs.workload_state("fluid-131k")
    n = w.n
    out = {"workload": "fluid-131k", "n": n, "steps": w.steps}
    xj, Lj = inputs.jittered_fcc(32, w.rho, 0.1, 7)   # a non-lattice state for the force error
    fo = None
    if with_oracle:
        import oracle
        fo = oracle.forces_cells(xj, Lj, rc=w.rc, mode=1)[0]
    for precision in ("mixed", "fp64"):
        row = {}
        if fo is not None:
            s = lj.System(xj, None, Lj, precision=precision, rc=w.rc)
            s.forces()
            fg = s.f.double().cpu().numpy()[:, :3]
            s.check()
            s.close()
            row["force_rel_rms_vs_oracle"] = float(np.sqrt(((fg - fo) ** 2).sum() / (fo ** 2).sum()))
        s = lj.System(x, v, L, precision=precision, dt=w.dt, rc=w.rc)
        o0 = s.observables()
        s.step(w.steps)
        o1 = s.observables()
        s.check()
        s.close()
        torch.cuda.synchronize()
        e0, e1 = o0["e_tot"], o1["e_tot"]
        row["energy_drift_per_particle"] = (e1 - e0) / n
        row["e_total_start_per_particle"] = e0 / n
        row["T_start"], row["T_end"] = o0["T"], o1["T"]
        row["P_start"], row["P_end"] = o0["P"], o1["P"]
        out[precision] = row
    if with_oracle:
        import oracle
        xo, vo = x.copy(), v.copy()
        f, _, ep0, _ = oracle.forces_cells(xo, L, rc=w.rc, mode=1)
        e0 = ep0 + oracle.ekin(vo)
        t0 = time.perf_counter()
        done = 0
        while done < w.steps and time.perf_counter() - t0 < max_oracle_s:
            k = min(100, w.steps - done)
            ep, _ = oracle.vv(xo, vo, f, L, k, dt=w.dt, rc=w.rc, mode=1)
            done += k
        e1 = ep + oracle.ekin(vo)
        out["oracle"] = {"steps": done, "energy_drift_per_particle": (e1 - e0) / n,
                         "energy_drift_per_particle_per_1000_steps": (e1 - e0) / n * 1000.0 / done,
                         "seconds": time.perf_counter() - t0}
    return out


def run_accuracy_2k():
    """The fluid-2k workload as stated (N = 2,048 FCC start, rho 0.8442,
    T 0.728, 100 FP64 velocity-Verlet steps): the GPU's FP64 trajectory
    against the oracle's trajectory with all-pairs forces (Section 2, no
    cells), and both total-energy drifts, with the temperature and pressure
    at the end."""
    import oracle
    from paper_0709_3225_gb300 import inputs, lj
    x, v, L, w = inputs.workload_state("fluid-2k")
    xo, vo = x.copy(), v.copy()
    fo, _, ep0, _ = oracle.forces_brute(xo, L, rc=w.rc)
    e0 = ep0 + oracle.ekin(vo)
    ep1, _ = oracle.vv(xo, vo, fo, L, w.steps, dt=w.dt, rc=w.rc, k=0)
    e1 = ep1 + oracle.ekin(vo)
    ob = oracle.observables(xo, vo, L, rc=w.rc)
    s = lj.System(x, v, L, precision="fp64", dt=w.dt, rc=w.rc)
    g0 = s.observables()
    s.step(w.steps)
    g1 = s.observables()
    s.check()
    d = s.x.cpu().numpy() - xo
    d -= L * np.round(d / L)
    s.close()
    return {"workload": "fluid-2k", "n": w.n, "steps": w.steps, "precision": "fp64",
            "oracle_forces": "all pairs (Section 2), no cells",
            "max_abs_dx_vs_oracle": float(np.abs(d).max()),
            "gpu": {"energy_drift_per_particle": (g1["e_tot"] - g0["e_tot"]) / w.n, "T_end": g1["T"],
                    "P_end": g1["P"]},
            "oracle": {"energy_drift_per_particle": (e1 - e0) / w.n, "T_end": ob["T"], "P_end": ob["P"]}}


def run_skin(x, v, L, w, stream, steps=60):
    """Cell lists with a skin on the 4M workload: ms per step and rebuilds
    for a few skins, beside the per-step rebuild (skin 0)."""
    import torch
    from paper_0709_3225_gb300 import lj
    out = []
    for skin in (0.0, 0.3, 0.6):
        s = lj.System(x, v, L, precision="mixed", dt=w.dt, rc=w.rc)
        if skin > 0:
            lj.lj_set_skin(s.ctx, skin)
        s.forces()
        s.step(5)
        torch.cuda.synchronize()
        r0, n0 = lj.lj_skin_stats(s.ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        r1, n1 = lj.lj_skin_stats(s.ctx)
        s.check()
        out.append({"skin": skin, "cells_per_axis": s.ctx.nc, "ms_per_step": e0.elapsed_time(e1) / steps,
                    "rebuilds": (r1 - r0) if skin > 0 else steps, "steps": steps})
        s.close()
    return out


def run_adjoint(x4m, L4m, stream):
    """The adjoint workload: the force-matching gradient (loss = mean |F -
    F_target|^2 + mean |x(50) - x_target(50)|^2, theta = (0.9, 1.05)) of the
    32,000-particle jittered lattice, forward + checkpointed backward through
    50 force-shifted steps, FP32-mixed; plus one VJP launch at N = 4M.
    Targets come from the same library at theta = (1, 1) (this times the
    path; parity is established in the tests)."""
    import torch
    from paper_0709_3225_gb300 import autograd, inputs, lj
    w = inputs.WORKLOADS["fm-32k"]
    x0, L = inputs.jittered_fcc(w.n_fcc, w.rho, 0.1, w.seed)
    v0 = inputs.velocities(w.n, w.temperature, w.seed)
    s = lj.System(x0, v0, L, shift_mode=2)
    with torch.no_grad():
        star = torch.tensor([1.0, 1.0], dtype=torch.float64, device="cuda")
        f_t = autograd.forces(s.x, star, s.ctx).clone()
        x_t, _ = autograd.trajectory(s.x, s.v, star, s.ctx, 50, 10)
    n = w.n

    def grad():
        theta = torch.tensor([0.9, 1.05], dtype=torch.float64, device="cuda", requires_grad=True)
        F = autograd.forces(s.x, theta, s.ctx)
        xT, _ = autograd.trajectory(s.x, s.v, theta, s.ctx, 50, 10)
        d = xT - x_t
        d = d - L * torch.round(d / L)
        loss = ((F - f_t) ** 2).sum() / n + (d ** 2).sum() / n
        loss.backward()
        return theta.grad

    grad()
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        g = grad()
    torch.cuda.synchronize()
    t_grad = (time.perf_counter() - t0) / reps
    s.close()
    # one VJP of the 4M system (binning, cotangent gather and the VJP kernel),
    # FP32-mixed and FP64
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vjp_ms = {}
    for precision in ("mixed", "fp64"):
        s4 = lj.System(x4m, None, L4m, precision=precision)
        g4 = torch.randn((s4.n, 3), dtype=torch.float64, device="cuda")
        dx = torch.zeros_like(s4.x)
        dp = torch.zeros(2, dtype=torch.float64, device="cuda")
        lj.lj_forces_vjp(s4.ctx, s4.x, g4, 1.0, dx, dp)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(3):
            lj.lj_forces_vjp(s4.ctx, s4.x, g4, 1.0, dx, dp)
        ev1.record(stream)
        torch.cuda.synchronize()
        s4.check()
        vjp_ms[precision] = ev0.elapsed_time(ev1) / 3
        s4.close()
    pairs4m = unique_pairs(4_000_000, 0.8442, 2.5)
    return {"workload": "fm-32k force matching, 50 steps, checkpoints every 10", "n": n,
            "gradient_s": t_grad, "gradients_per_s": 1.0 / t_grad,
            "dL_dtheta": [float(g[0]), float(g[1])],
            "vjp_4m_ms": vjp_ms["mixed"], "vjp_4m_pairs_per_s": pairs4m / (vjp_ms["mixed"] / 1e3),
            "vjp_4m_fp64_ms": vjp_ms["fp64"], "vjp_4m_fp64_pairs_per_s": pairs4m / (vjp_ms["fp64"] / 1e3)}


def cpu_baseline(x, v, L, w, max_seconds: float = 20.0, max_steps: int = 3, one_core: bool = True):
    """The FP64 oracle as it stands, on this host's cores: full velocity-Verlet
    steps of the same workload until ~max_seconds of work, scaled to steps/s."""
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    used = oracle.set_threads(cores)
    xo, vo = x.copy(), v.copy()
    t0 = time.perf_counter()
    fo = oracle.forces_cells(xo, L, rc=w.rc, mode=1)[0]
    t_force = time.perf_counter() - t0
    steps = 0
    t0 = time.perf_counter()
    while steps < max_steps:
        oracle.vv(xo, vo, fo, L, 1, dt=w.dt, rc=w.rc, mode=1)
        steps += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    out = {"value": steps / dt, "unit": "steps/s", "cores": used, "kind": "oracle",
           "sample": f"{steps} full FP64 velocity-Verlet step(s) of the {w.n}-particle workload "
                     f"(plus one initial force evaluation, {t_force:.1f} s, untimed)",
           "pair_interactions_per_s": unique_pairs(w.n, w.rho, w.rc) * steps / dt}
    if one_core:
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.vv(xo, vo, fo, L, 1, dt=w.dt, rc=w.rc, mode=1)
        dt1 = time.perf_counter() - t0
        oracle.set_threads(used)
        out["one_core"] = {"value": 1.0 / dt1, "unit": "steps/s", "cores": 1,
                           "sample": "1 full FP64 velocity-Verlet step, one thread"}
    return out


def run_reference(args):
    """--impl reference: the oracle on the host cores, same metric and workload."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_0709_3225_gb300 import inputs
    x, v, L, w = inputs.workload_state(WORKLOAD)
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    used = oracle.set_threads(cores)
    xo, vo = x.copy(), v.copy()
    fo = oracle.forces_cells(xo, L, rc=w.rc, mode=1)[0]
    # bounded: W warm-up steps (at most 5; the first one sizes the sample)
    # and as many timed steps as fit ~90 s
    n_warm = max(1, min(args.warmup, 5))
    t0 = time.perf_counter()
    oracle.vv(xo, vo, fo, L, 1, dt=w.dt, rc=w.rc, mode=1)
    t_step = time.perf_counter() - t0
    if n_warm > 1:
        oracle.vv(xo, vo, fo, L, n_warm - 1, dt=w.dt, rc=w.rc, mode=1)
    k = max(1, min(args.steps, int(90.0 / max(t_step, 1e-3))))
    t0 = time.perf_counter()
    oracle.vv(xo, vo, fo, L, k, dt=w.dt, rc=w.rc, mode=1)
    T = time.perf_counter() - t0
    value = k / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": k, "warmup": n_warm, "ms_per_step": 1e3 * T / k, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": w.n, "rho": w.rho, "T": w.temperature, "rc": w.rc, "dt": w.dt,
                   "start": "fcc", "requested_steps": args.steps, "requested_warmup": args.warmup},
        "pair_interactions_per_s": unique_pairs(w.n, w.rho, w.rc) * value,
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": used, "kind": "oracle",
                         "sample": f"{k} of {args.steps} requested steps timed (bounded to ~90 s), {n_warm} warm-up"},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    from paper_0709_3225_gb300 import inputs, lj

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    x, v, L, w = inputs.workload_state(WORKLOAD)
    n = w.n
    pairs = unique_pairs(n, w.rho, w.rc)
    mpk = measure_peaks()
    FP32_PEAK_TFLOPS, FP64_PEAK_TFLOPS = mpk["fp32_tflops"], mpk["fp64_tflops"]

    # ---- FP32-mixed, device-resident (the headline `value`) --------------
    from paper_0709_3225_gb300 import autotune
    s, tuning = autotune.make_system(x, v, L, w.rho, precision="mixed", dt=w.dt, rc=w.rc)
    s.forces()
    tuning.pop("trials", None)
    s.step(args.warmup)
    s.check()
    lj.lj_set_timing(s.ctx, True)
    _, _, k0 = lj.lj_read_timing(s.ctx)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        lj.lj_step(s.ctx, s.x, s.v, s.f, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms_total = ev0.elapsed_time(ev1)
    s.check()
    force_ms, force_n, k1 = lj.lj_read_timing(s.ctx)
    lj.lj_set_timing(s.ctx, False)
    launches = k1 - k0
    value, t_max = job_rate(world, args.steps, ms_total / 1e3)
    ms_total = t_max * 1e3
    ms_step = ms_total / args.steps
    force_avg_ms = force_ms / max(force_n, 1)
    achieved_tflops = FLOPS_PER_PAIR * pairs / (force_avg_ms / 1e3) / 1e12
    clocks = clk.summary()

    # HBM view of the non-force kernels: algorithmic bytes per particle per step
    # (kick-drift-bin 124 B, scatter 56 B, force in/out 32 B).
    other_ms = ms_step - force_avg_ms
    candidates = stencil_candidates(s.ctx)
    pair_once = tuning.get("kernel") == 7
    if pair_once:   # each pair once over the half stencil
        half = half_stencil_candidates(s.ctx)
        issued_flops = CANDIDATE_FLOPS * half + FLOPS_PER_PAIR * pairs
    else:
        half = None
        issued_flops = CANDIDATE_FLOPS * candidates + FLOPS_PER_PAIR * 2 * pairs
    issued_tflops = issued_flops / (force_avg_ms / 1e3) / 1e12

    # ---- the same system as an equilibrated fluid ---------------------------
    # The lattice start melts within ~100 steps; 1000 steps after it the cell
    # occupancies have the fluid's spread.  Timed the same way.
    eq_total = 1000
    s.step(max(0, eq_total - args.warmup - args.steps))
    s.check()
    lj.lj_set_timing(s.ctx, True)
    barrier(world)
    torch.cuda.synchronize()
    ev0.record(stream)
    lj.lj_step(s.ctx, s.x, s.v, s.f, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    s.check()
    fl_force_ms, fl_force_n, _ = lj.lj_read_timing(s.ctx)
    lj.lj_set_timing(s.ctx, False)
    fl_value, fl_t = job_rate(world, args.steps, ev0.elapsed_time(ev1) / 1e3)
    fluid = {"start": f"the lattice start after {max(eq_total, args.warmup + args.steps)} FP32-mixed steps",
             "value": fl_value, "unit": "steps/s", "ms_per_step": fl_t * 1e3 / args.steps,
             "force_ms_per_launch": fl_force_ms / max(fl_force_n, 1),
             "pair_interactions_per_s": pairs * fl_value,
             "stencil_candidates_per_launch": stencil_candidates(s.ctx)}

    # ---- end to end through the host-buffer entry point ------------------
    e2e_steps = max(3, min(20, args.steps))
    xh = torch.from_numpy(s.x.cpu().numpy()).pin_memory()
    vh = torch.from_numpy(s.v.cpu().numpy()).pin_memory()
    fh = torch.from_numpy(s.f.cpu().numpy()).pin_memory()
    lj.lj_step_host(s.ctx, xh, vh, fh, 1)           # warm the staging buffers
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lj.lj_step_host(s.ctx, xh, vh, fh, 1)
    e2e_value, t_e2e = job_rate(world, e2e_steps, time.perf_counter() - t0)
    bytes_h2d = n * (3 * 8 + 3 * 8 + 4 * 4)
    link = pinned_link_gbs()
    s.close()
    del s
    torch.cuda.empty_cache()

    # ---- plain FP64 GPU path on the same workload --------------------------
    s64 = lj.System(x, v, L, precision="fp64", dt=w.dt, rc=w.rc)
    s64.forces()
    s64.step(2)
    k64 = max(3, min(10, args.steps))
    lj.lj_set_timing(s64.ctx, True)
    torch.cuda.synchronize()
    ev0.record(stream)
    lj.lj_step(s64.ctx, s64.x, s64.v, s64.f, k64)
    ev1.record(stream)
    torch.cuda.synchronize()
    s64.check()
    ms64 = ev0.elapsed_time(ev1) / k64
    f64_ms, f64_n, _ = lj.lj_read_timing(s64.ctx)
    s64.close()
    del s64

    ensemble = None if args.no_ensemble else run_ensemble(args, stream, world)
    adjoint = None if (args.no_ensemble or rank != 0) else run_adjoint(x, L, stream)
    n2 = None if (args.no_ensemble or rank != 0) else run_n2_breakeven(stream)
    rng = None if (args.no_ensemble or rank != 0) else run_rand48(stream, (read_peaks() or {}).get("hbm_gbs"))
    langevin = None if (args.no_ensemble or rank != 0) else run_langevin(x, v, L, w, stream)
    skin = None if (args.no_ensemble or rank != 0) else run_skin(x, v, L, w, stream)
    aop = None if (args.no_ensemble or rank != 0) else run_aop_density(stream)
    small = None if (args.no_ensemble or rank != 0) else run_graph_small(stream)
    accuracy = None if (args.no_ensemble or rank != 0) else run_accuracy_131k(world == 1 and not args.no_cpu_baseline)
    accuracy_2k = None if (args.no_ensemble or rank != 0) else run_accuracy_2k()

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    peaks = read_peaks()
    # the committed ncu figures describe the default kernel; report them only
    # when the tuner kept it
    default_kernel = (tuning.get("kernel"), tuning.get("gw"), tuning.get("subdiv", 1)) == (7, 0, 1)
    traffic = force_traffic() if default_kernel else None

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "rho": w.rho, "T": w.temperature, "rc": w.rc, "dt": w.dt,
                   "start": "fcc lattice", "precision": "mixed (FP32 pairs, FP64 x/v/energy)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (x, v 96 MB each, forces and sorted positions 64 MB each)"},
        "pair_interactions_per_s": pairs * value,
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tflops / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": ("k_force_n3 (each pair once, half stencil)" if pair_once else
                                "k_force_warp (27-cell stencil)") + f", tuning kernel {tuning.get('kernel')}",
                     "force_ms_per_launch": force_avg_ms,
                     "flops_per_launch": FLOPS_PER_PAIR * pairs,
                     "stencil_candidates_per_launch": candidates,
                     "half_stencil_candidates_per_launch": half,
                     "issued_flops_per_launch": issued_flops,
                     "issued_frac": issued_tflops / FP32_PEAK_TFLOPS,
                     "issued_convention": ("7 flop per half-stencil candidate + 20 per pair, once" if pair_once else
                                           "7 flop per full-stencil candidate + 20 per pair, both directions"),
                     "peak_source": "measured (lj_measure_peak, FP32 FMA chains; see measured_fp_peaks)",
                     "frac_of_derived": achieved_tflops / mpk["derived_fp32_tflops"],
                     "fp32_pipe_busy": force_traffic("fp32_pipe_busy") if default_kernel else None,
                     "fp32_pipe_busy_source": "ncu sm__pipe_fmaheavy_cycles_active of the default force "
                                              "kernel at this size (profiles/k_force_n3_traffic_fluid-4m.md)"},
        "other_kernels_ms_per_step": other_ms,
        "tuning": tuning,
        "ensemble": ensemble,
        "adjoint": adjoint,
        "n2_vs_cells": n2,
        "rand48": rng,
        "langevin": langevin,
        "skin": skin,
        "aop_vs_csr_density": aop,
        "small_systems_graph": small,
        "fluid_start": fluid,
        "accuracy_131k": accuracy,
        "accuracy_2k": accuracy_2k,
        "fp64": {"value": 1e3 / ms64, "unit": "steps/s", "ms_per_step": ms64, "steps": k64,
                 "force_ms_per_launch": f64_ms / max(f64_n, 1),
                 "pair_interactions_per_s": pairs * 1e3 / ms64,
                 "kernel": "k_force_w64 (compacted in-range pair lists, each pair once)",
                 "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                              "achieved": FLOPS_PER_PAIR * pairs / (f64_ms / max(f64_n, 1) / 1e3) / 1e12,
                              "frac": FLOPS_PER_PAIR * pairs / (f64_ms / max(f64_n, 1) / 1e3) / 1e12
                              / FP64_PEAK_TFLOPS,
                              "peak_source": "measured (lj_measure_peak, FP64 FMA chains)"}},
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": bytes_h2d,
                "d2h_bytes_per_step": bytes_h2d, "steps": e2e_steps,
                "api": "lj_step_host, pinned host x, v, f; 1 step per call",
                "pinned_link_gbs": link,
                "copy_ms_per_step_at_link_rate": (bytes_h2d / link["h2d"] + bytes_h2d / link["d2h"]) / 1e6},
        "clocks": clocks,
        "measured_peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")} if peaks else None,
        "measured_fp_peaks": mpk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(x, v, L, w)
        # the paper's speed-up form, T_CPU / T_GPU, for the FP32-mixed and FP64
        # GPU paths against the oracle on all host cores and on one
        ref = {"all_cores": cpu["value"], "one_core": cpu.get("one_core", {}).get("value")}
        cpu["gpu_speedup"] = {f"{path}_vs_{k}": (val / r if r else None)
                              for path, val in (("mixed", value), ("fp64", 1e3 / ms64)) for k, r in ref.items()}
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


FORCE_SOURCES = [os.path.join(ROOT, "paper_0709_3225_gb300", "csrc", f)
                 for f in ("lj_force_n3.cu", "lj_force_n3.cuh", "lj_force_cell.cuh", "lj_internal.cuh", "lj_pair.cuh")]
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_force_n3_traffic_fluid-4m.md")


def force_traffic(field="dram_bytes_per_launch"):
    """A figure of the committed ncu summary of the force kernel (DRAM bytes
    per launch, or the FP32-pipe activity), or None when the summary is
    missing or was taken on a different kernel source."""
    import hashlib
    try:
        h = hashlib.sha1()
        for path in FORCE_SOURCES:
            with open(path, "rb") as fh:
                h.update(fh.read())
        sha = h.hexdigest()
        fields = {}
        with open(TRAFFIC_SUMMARY) as fh:
            for line in fh:
                if ":" in line and line.strip().startswith(("kernel_source_sha1", "dram_bytes_per_launch",
                                                            "fp32_pipe_busy")):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
    except OSError:
        return None
    if fields.get("kernel_source_sha1") != sha:
        return None
    try:
        return float(fields[field])
    except (KeyError, ValueError):
        return None


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=180)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble and adjoint measurements")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    from __graft_entry__ import build
    build()
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
