"""Shared test helpers: map the binding's parameters onto the oracle's, run the oracle."""
from __future__ import annotations

import numpy as np
import torch

from oracle import lbm
from paper_1111_0905_gb300 import lb


def oracle_params(p: lb.Params) -> lbm.Params:
    return lbm.Params(p.nx, p.ny, p.nz, p.tau_nu, p.tau_kappa, p.G, p.kappa, p.c_v, p.g_z,
                      p.T_d, p.T_u,
                      forcing="guo" if p.forcing == lb.LB_FORCE_GUO else "shift",
                      psi_kind="vdw" if p.psi_kind == lb.LB_PSI_VDW else "exp",
                      vdw_a=p.vdw_a, vdw_b=p.vdw_b, vdw_T=p.vdw_T)


def oracle_run(p: lb.Params, rho, T, steps: int, nu_every: int = 0):
    """Oracle state after `steps` steps and the list of Nu_mean sampled every nu_every steps."""
    op = oracle_params(p)
    f, g = lbm.init_state(torch.from_numpy(np.asarray(rho)), torch.from_numpy(np.asarray(T)), op)
    samples = []
    for n in range(1, steps + 1):
        f, g = lbm.step(f, g, op)
        if nu_every and n % nu_every == 0:
            samples.append(lbm.nusselt(f, g, op)[0].item())
    return f, g, op, samples


def rel_err(a, b) -> float:
    """max |a - b| / max |b| (field-scale relative error)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.abs(b).max()
    return float(np.abs(a - b).max() / (scale if scale > 0 else 1.0))
