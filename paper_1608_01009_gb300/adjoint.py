"""torch.autograd.Function around the library's hand-written adjoint.

forward runs the differentiable FP64 path (pic_tape_forward: the whole PIC
step -- cloud-in-cell gather, Boris push, Villasenor-Buneman deposit, Yee FDTD
-- with a checkpoint every `ckpt_every` steps) from the given initial fields
and the simulation's current particles, and returns the final electron
kinetic energy W_K.  backward calls pic_tape_backward, which replays each
checkpoint segment and runs the adjoint kernels in reverse, and returns
dW_K/dE0 and dW_K/dB0.  Gradients with respect to anything the initial fields
are built from (a laser amplitude a0, say) follow by ordinary autograd.
"""
from __future__ import annotations

import torch


class KineticEnergyAfter(torch.autograd.Function):
    """W_K after `nsteps` steps as a differentiable function of (E0, B0)."""

    @staticmethod
    def forward(ctx, E0, B0, sim, nsteps, ckpt_every):
        sim.set_fields(E0.detach().contiguous(), B0.detach().contiguous())
        sim.stream.synchronize()
        wk = sim.tape_forward(nsteps, ckpt_every)
        ctx.sim = sim
        return torch.tensor(wk, dtype=torch.float64, device=E0.device)

    @staticmethod
    def backward(ctx, grad):
        dE0, dB0 = ctx.sim.tape_backward(1.0)
        return grad * dE0, grad * dB0, None, None, None


def kinetic_energy_after(E0, B0, sim, nsteps, ckpt_every):
    return KineticEnergyAfter.apply(E0, B0, sim, nsteps, ckpt_every)
