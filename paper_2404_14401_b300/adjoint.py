"""torch.autograd interface to the adjoint split step (lattice-depth control).

J(v) = E(psi_T) + |<phi|psi_T>|^2, with psi_T the state after nsteps
real-time steps under the lattice depth v(t) given by control values v at
the context's control times, is a differentiable function of v: its forward
is one gpe_adjoint_lattice call (forward steps, then the reverse sweep of the
hand-written adjoint passes over states from checkpoints or, with
reverse=True, from steps backward in time), which also returns dJ/dv;
backward scales that gradient.  Nothing here computes physics: it only marshals.
"""
from __future__ import annotations

import numpy as np
import torch


class LatticeControlObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, sim, params, psi0, phi, nsteps, dt, t0, reverse):
        p = dict(params, ctrl_v=v.detach().cpu().numpy().astype(np.float64))
        sim.set_potential(p)
        sim.set_psi(psi0)
        sim.t = t0
        J, grad = sim.adjoint_lattice(phi, nsteps, dt, reverse)
        ctx.save_for_backward(torch.tensor(grad, dtype=v.dtype, device=v.device))
        return v.new_tensor(J)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None, None, None, None, None, None, None, None


def lattice_control_objective(v: torch.Tensor, sim, params: dict, psi0, phi, nsteps: int, dt: float,
                              t0: float = 0.0, reverse: bool = False) -> torch.Tensor:
    """Differentiable J(v) on the Simulation `sim` (see module docstring).
    params: the potential dict (ctrl_target = lattice, ctrl_t set); psi0:
    initial state (numpy or cuda tensor); phi: target state."""
    return LatticeControlObjective.apply(v, sim, params, psi0, phi, nsteps, dt, t0, reverse)
