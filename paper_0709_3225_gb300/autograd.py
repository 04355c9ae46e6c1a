"""torch.autograd wrappers over the library's forces and their adjoint.

``forces(x, theta, ctx)``  -> F (n, 3) float64; backward gives dL/dx and
                              dL/dtheta, theta = (eps, sigma).
``trajectory(x0, v0, theta, ctx, nsteps, every)`` -> (x_T, v_T) after nsteps
                              velocity-Verlet steps; backward runs the adjoint
                              with checkpoints every ``every`` steps.

The paper has no adjoint; these differentiate its force (Eq. n2_force with the
Section 2 pair force, rc held fixed) and its velocity-Verlet integration.
The cell list is piecewise constant and contributes no derivative.  Every
arithmetic step runs in the library's kernels (lj_forces, lj_step,
lj_forces_vjp, lj_vv_adjoint_step); this module only sequences the calls and
keeps checkpoints.  Use the force-shifted potential (shift_mode 2) when the
trajectory derivative must match finite differences: with the energy shift
the force jumps at rc and the trajectory is not differentiable there.
"""
from __future__ import annotations

import torch

from . import lj


def _set(ctx: lj.Context, theta: torch.Tensor) -> None:
    t = theta.detach().to("cpu", torch.float64)
    lj.lj_set_params(ctx, float(t[0]), float(t[1]))


class _Forces(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x, theta, ctx):
        _set(ctx, theta)
        f = torch.empty((ctx.n, 4), dtype=ctx.force_dtype, device=x.device)
        lj.lj_forces(ctx, x.detach().contiguous(), f)
        fctx.ctx = ctx
        fctx.save_for_backward(x.detach(), theta.detach())
        return f[:, :3].to(torch.float64)

    @staticmethod
    def backward(fctx, g):
        x, theta = fctx.saved_tensors
        ctx = fctx.ctx
        _set(ctx, theta)
        dx = torch.zeros_like(x)
        dp = torch.zeros(2, dtype=torch.float64, device=x.device)
        lj.lj_forces_vjp(ctx, x, g.to(torch.float64).contiguous(), 1.0, dx, dp)
        return dx, dp.to(theta.device, theta.dtype), None


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x0, v0, theta, ctx, nsteps, every):
        _set(ctx, theta)
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        f = torch.empty((ctx.n, 4), dtype=ctx.force_dtype, device=x.device)
        lj.lj_forces(ctx, x, f)
        ckpts = []
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            ckpts.append((x.clone(), v.clone(), k))
            lj.lj_step(ctx, x, v, f, k)
            done += k
        fctx.ctx = ctx
        fctx.ckpts = ckpts
        fctx.save_for_backward(theta.detach())
        return x, v

    @staticmethod
    def backward(fctx, gx, gv):
        (theta,) = fctx.saved_tensors
        ctx = fctx.ctx
        _set(ctx, theta)
        ref = fctx.ckpts[0][0]
        lam_x = torch.zeros_like(ref) if gx is None else gx.to(torch.float64).clone().contiguous()
        lam_v = torch.zeros_like(ref) if gv is None else gv.to(torch.float64).clone().contiguous()
        dp = torch.zeros(2, dtype=torch.float64, device=ref.device)
        f = torch.empty((ctx.n, 4), dtype=ctx.force_dtype, device=ref.device)
        for xs, vs, k in reversed(fctx.ckpts):
            # recompute the segment's states from its checkpoint
            x = xs.clone()
            v = vs.clone()
            lj.lj_forces(ctx, x, f)
            states = [x.clone()]
            for _ in range(k):
                lj.lj_step(ctx, x, v, f, 1)
                states.append(x.clone())
            for s in range(k - 1, -1, -1):
                lj.lj_vv_adjoint_step(ctx, states[s], states[s + 1], lam_x, lam_v, dp)
        fctx.ckpts = None
        return lam_x, lam_v, dp.to(theta.device, theta.dtype), None, None, None


def forces(x: torch.Tensor, theta: torch.Tensor, ctx: lj.Context) -> torch.Tensor:
    """Differentiable forces F(x; eps, sigma) (n, 3) float64."""
    return _Forces.apply(x, theta, ctx)


def trajectory(x0: torch.Tensor, v0: torch.Tensor, theta: torch.Tensor, ctx: lj.Context, nsteps: int,
               every: int = 10):
    """Differentiable (x_T, v_T) after nsteps velocity-Verlet steps from
    (x0, v0); the backward pass recomputes each segment of ``every`` steps
    from its checkpoint."""
    return _Trajectory.apply(x0, v0, theta, ctx, int(nsteps), int(every))
