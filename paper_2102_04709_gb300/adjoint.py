"""torch.autograd.Function around the C-ABI adjoint (lbm3_adjoint_centroid).

J(angles, u_in) = x-centroid of fluid 0 after `nsteps` timesteps from the rest state `rho0`;
`angles` are the wall-angle triples (theta_01, theta_20, theta_12) of every solid boundary node
(degrees, [n_wall, 3], the order of Lbm3.wall_nodes()), `u_in` the Zou-He inflow velocity.  The
forward call runs the checkpointed forward pass and the adjoint kernels on the GPU and keeps the
gradient for backward.  The simulation keeps the adjoint's device memory and its recorded sweep
between calls of the same size (an optimisation loop's steady state); Lbm3.adjoint_release()
frees them.
"""
from __future__ import annotations

import torch

from . import lbm3


class CentroidObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, angles, u_in, sim, rho0, nsteps, checkpoint_every):
        u_t = torch.as_tensor(u_in)
        sim.set_wall_angles(angles.detach().cpu().double().numpy())
        if sim.bc_x == 2:
            sim.set_inflow(float(u_t))
        sim.set_fields(rho0)
        J, dang, du = sim.adjoint_centroid(nsteps, checkpoint_every)
        # the gradients live where the inputs do, in their dtype
        ctx.save_for_backward(torch.as_tensor(dang, dtype=angles.dtype, device=angles.device),
                              torch.tensor(du, dtype=u_t.dtype, device=u_t.device))
        return torch.tensor(J, dtype=torch.float64, device=angles.device)

    @staticmethod
    def backward(ctx, gJ):
        dang, du = ctx.saved_tensors
        return (gJ.to(dang.device, dang.dtype) * dang, gJ.to(du.device, du.dtype) * du, None, None,
                None, None)


def centroid(sim: "lbm3.Lbm3", angles: torch.Tensor, u_in: torch.Tensor, rho0, nsteps: int,
             checkpoint_every: int = 100) -> torch.Tensor:
    """Differentiable x-centroid of fluid 0 after nsteps steps (see module docstring)."""
    return CentroidObjective.apply(angles, u_in, sim, rho0, nsteps, checkpoint_every)
