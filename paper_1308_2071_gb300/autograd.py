"""The hot-wall mean Nusselt number (Eq. 38) after a fixed number of steps,
as a differentiable function of a per-cell porosity field.

forward runs the time stepping from the initial state with the given field
(lbm_set_porous_field, lbm_step, lbm_nusselt); backward calls the discrete
adjoint (lbm_adjoint_step), which repeats the forward sweep keeping a
checkpoint every ckpt_every steps, recomputes each segment from its checkpoint
and runs the reverse steps over it.  Its repeated forward sweep must land on
the same J as the forward pass: the step is deterministic, so a mismatch
means the cavity was changed in between, and backward raises.
"""
from __future__ import annotations

import torch

from .lbm import Cavity


class HotWallNusselt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi: torch.Tensor, cavity: Cavity, nsteps: int, ckpt_every: int):
        if phi.shape != (cavity.ny, cavity.nx):
            raise ValueError(f"phi has shape {tuple(phi.shape)}, the cavity is {(cavity.ny, cavity.nx)}")
        cavity.set_porous_field(phi)  # resets the cavity to t = 0
        cavity.step(int(nsteps))
        J = cavity.nusselt()[0]
        ctx.cavity, ctx.nsteps, ctx.ckpt_every, ctx.J = cavity, int(nsteps), int(ckpt_every), J
        ctx.save_for_backward(phi)
        return torch.tensor(J, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (phi,) = ctx.saved_tensors
        cav = ctx.cavity
        cav.set_porous_field(phi)
        J, g = cav.adjoint(ctx.nsteps, ctx.ckpt_every)
        if J != ctx.J:
            raise RuntimeError(f"the adjoint's forward sweep gave J = {J!r}, the forward pass {ctx.J!r}: "
                               "the cavity changed between forward and backward")
        return (grad_out.to(phi.dtype) * g.to(phi.dtype)), None, None, None


def hot_wall_nusselt(phi: torch.Tensor, cavity: Cavity, nsteps: int, ckpt_every: int = 100) -> torch.Tensor:
    """J(phi) = mean Nu of the hot wall after nsteps steps from the initial
    state (0-d FP64 tensor), differentiable with respect to phi (ny, nx).
    cavity must have been created with a porosity field (use_phi_field = 1)
    in FP64 or FP32."""
    return HotWallNusselt.apply(phi, cavity, nsteps, ckpt_every)
