"""Run one library operation on a synthetic LJ liquid, for profilers.

  python -m paper_0709_3225_gb300.profile_run --op force --n-fcc 80 --reps 3

Builds a jittered FCC liquid of 4 n^3 particles at rho = 0.8442 (or the
lattice itself, ``--lattice``), then runs
``--reps`` force evaluations (``--op force``), velocity-Verlet steps
(``--op step``) or force VJPs with a seeded Gaussian cotangent (``--op
vjp``) through the C ABI after one untimed warm-up, and prints the
CUDA-event time per call.  ``--op batch`` instead steps the 256-replica
ensemble (one cooperative launch per step, direct launches, ``--grab``
cells per pull, the batch kernel ``--kernel`` if given: 3 the 27-cell
code, 7 each pair once) after its 50 relaxation steps.  It reports no
benchmark figures; use bench.py for those.
"""
from __future__ import annotations

import argparse

import torch

from . import inputs, lj


def run_batch(reps: int, kernel: int | None = None, grab: int = 1) -> int:
    e = inputs.ensemble()
    xs, vs = inputs.ensemble_state(e)
    b = lj.Batch(xs, vs, e.box)
    b.relax(50, 1e-3, 0.05)
    if kernel is not None:
        b.set_kernel(kernel)
    b.set_tuning(grab, False, 0)
    b.forces()
    b.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.step(1)
    e1.record()
    torch.cuda.synchronize()
    b.check()
    print(f"batch n={b.ntot} replicas={b.nrep} {e0.elapsed_time(e1) / reps:.3f} ms per step")
    b.close()
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["force", "step", "vjp", "batch"], default="force")
    ap.add_argument("--n-fcc", type=int, default=80)
    ap.add_argument("--rho", type=float, default=0.8442)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--flags", type=int, default=0)
    ap.add_argument("--subdiv", type=int, default=1, help="cell subdivision k (1 or 2)")
    ap.add_argument("--group-width", type=int, default=None, help="warp-kernel lane-group width (0 = per cell)")
    ap.add_argument("--kernel", type=int, default=None, help="lj_set_tuning force kernel (default: the context's)")
    ap.add_argument("--lattice", action="store_true", help="the FCC lattice itself instead of a jittered one")
    ap.add_argument("--grab", type=int, default=1, help="cells per work pull of the batched step (--op batch)")
    args = ap.parse_args(argv)
    if args.op == "batch":
        return run_batch(args.reps, args.kernel, args.grab)
    if args.lattice:
        x, L = inputs.fcc(args.n_fcc, args.rho)
    else:
        x, L = inputs.jittered_fcc(args.n_fcc, args.rho, 0.1, 1)
    v = inputs.velocities(x.shape[0], 1.0, 1)
    s = lj.System(x, v, L, precision=args.precision, flags=args.flags, cell_subdiv=args.subdiv)
    if args.group_width is not None or args.kernel is not None:
        lj.lj_set_tuning(s.ctx, 3 if args.kernel is None else args.kernel, args.group_width or 0, 4)
    s.forces()
    g = dx = dp = None
    if args.op == "vjp":
        gen = torch.Generator(device="cuda").manual_seed(1)
        g = torch.randn((s.n, 3), dtype=torch.float64, device="cuda", generator=gen)
        dx = torch.zeros_like(s.x)
        dp = torch.zeros(2, dtype=torch.float64, device="cuda")
        lj.lj_forces_vjp(s.ctx, s.x, g, 1.0, dx, dp)
    if args.op == "step":
        s.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        if args.op == "force":
            s.forces()
        elif args.op == "vjp":
            lj.lj_forces_vjp(s.ctx, s.x, g, 1.0, dx, dp)
        else:
            s.step(1)
    e1.record()
    torch.cuda.synchronize()
    s.check()
    print(f"{args.op} n={s.n} nc={s.ctx.nc} {e0.elapsed_time(e1) / args.reps:.3f} ms per call")
    s.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
