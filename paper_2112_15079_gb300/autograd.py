"""``torch.autograd`` wrapper over the library's adjoint (``nbody_grad``).

``VerletTrajectory.apply(r0, v0, m, n_steps, G, dt, precision, ckpt_every)``
runs ``n_steps`` velocity-Verlet steps (Eqs. 1, 3, 4) from (r0, v0) on the
GPU and returns (r_T, v_T).  Its backward pass calls ``nbody_grad``: the
discrete adjoint of exactly that recurrence, with (r, v) checkpoints every
``ckpt_every`` steps and recomputation between them, giving dL/dr0, dL/dv0
and dL/dm.  All arithmetic runs in the library's CUDA kernels; this module
only moves tensors.
"""
from __future__ import annotations

import torch

from . import nbody as _nb


class VerletTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r0, v0, m, n_steps: int, G: float, dt: float, precision: str = "fp64",
                ckpt_every: int = 0):
        sim = _nb.NBody(r0.detach(), v0.detach(), m.detach(), G=G, dt=dt, precision=precision,
                        ckpt_every=ckpt_every, device=r0.device)
        sim.step(int(n_steps))
        sim.sync()
        ctx.sim = sim
        ctx.n_steps = int(n_steps)
        return sim.r.clone(), sim.v.clone()

    @staticmethod
    def backward(ctx, grad_r, grad_v):
        sim = ctx.sim
        gr = grad_r if grad_r is not None else torch.zeros_like(sim.r)
        dr, dv, dm = sim.grad(ctx.n_steps, gr, grad_v)
        sim.close()
        ctx.sim = None
        return dr, dv, dm, None, None, None, None, None


def trajectory(r0, v0, m, n_steps: int, G: float, dt: float, precision: str = "fp64", ckpt_every: int = 0):
    """Differentiable (r_T, v_T) after n_steps Verlet steps."""
    return VerletTrajectory.apply(r0, v0, m, n_steps, G, dt, precision, ckpt_every)
