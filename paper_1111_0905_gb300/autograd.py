"""PyTorch autograd binding of the time-averaged Nusselt objective and its discrete adjoint.

J = (1/N_t) sum_{n=1..N_t} Nu_mean(n), Nu of Eq. (4), over N_t steps of the thermal lattice
Boltzmann scheme started from the equilibrium of (rho, T0). The forward pass is `lb_init` + the
forward sweep of `lb_adjoint_step` (steps with checkpoints every K and the Nu samples); the
gradient dJ/d(T_d, T_u, G, T0) comes from the same call's reverse sweep and `backward` scales it
by the incoming gradient. Without any input that requires a gradient the forward pass is
`lb_init` + `lb_step` with a Nu sample every step. Argument marshalling only: every step runs in
the library's kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .lb import Lattice, Params

__all__ = ["NusseltObjective", "nusselt_objective"]


def _scalar(x) -> float:
    return float(x.detach().cpu()) if torch.is_tensor(x) else float(x)


class NusseltObjective(torch.autograd.Function):
    """J(T_d, T_u, G, T0); rho (initial density, no gradient), params, nsteps and the checkpoint
    interval are constants."""

    @staticmethod
    def forward(ctx, T_d, T_u, G, T0, rho, params: Params, nsteps: int, checkpoint_every: int):
        need = ctx.needs_input_grad[:4]
        p = dataclasses.replace(params, T_d=_scalar(T_d), T_u=_scalar(T_u), G=_scalar(G),
                                nu_every=0 if any(need) else 1)
        T0_arg = T0.detach().to(torch.float64).contiguous()
        rho_arg = torch.as_tensor(rho, dtype=torch.float64).to(T0_arg.device).contiguous()
        lat = Lattice(p, rho_arg, T0_arg)
        try:
            if any(need):
                r = lat.adjoint(int(nsteps), int(checkpoint_every), grad_T0=bool(need[3]))
                J = r["J"]
                grads = [torch.tensor(r["T_d"], dtype=torch.float64),
                         torch.tensor(r["T_u"], dtype=torch.float64),
                         torch.tensor(r["G"], dtype=torch.float64)]
                dT0 = (torch.from_numpy(np.ascontiguousarray(r["T0"])).to(T0.device)
                       if need[3] else torch.zeros(0, dtype=torch.float64))
                ctx.save_for_backward(*grads, dT0)
            else:
                lat.step(int(nsteps))
                J = lat.nusselt()[2]
        finally:
            lat.close()
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dTd, dTu, dG, dT0 = ctx.saved_tensors
        need = ctx.needs_input_grad
        out_T0 = gJ.to(dT0.device) * dT0 if need[3] else None
        return (gJ * dTd if need[0] else None, gJ * dTu if need[1] else None,
                gJ * dG if need[2] else None, out_T0, None, None, None, None)


def nusselt_objective(T_d, T_u, G, T0, rho, params: Params, nsteps: int,
                      checkpoint_every: int = 50) -> torch.Tensor:
    """J = time-averaged Nu over nsteps steps from (rho, T0), differentiable in T_d, T_u, G
    (scalar tensors) and T0 ([nz, ny, nx] float64 tensor, host or CUDA)."""
    return NusseltObjective.apply(T_d, T_u, G, T0, rho, params, nsteps, checkpoint_every)
