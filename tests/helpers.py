"""Shared test helpers: map the binding's parameters onto the oracle's, run the oracle."""
from __future__ import annotations

import dataclasses

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


# Dependency radius (Chebyshev, in nodes). A step's collision at y needs the force at y (psi one
# node out) and, for g, div(u) at y (u one node out, whose force reaches psi two nodes out);
# streaming adds one. So a step reaches at most 3 nodes; the moments rho, u, T after k steps from
# the equilibrium start reach exactly 2 k + 1 (measured tight for k = 1, 2, 3 and pinned in
# test_oracle_cutout.py). The cut-outs below use the bound, 3 k + 1.
STEP_RADIUS = 3


def oracle_cutout_moments(p: lb.Params, rho, T, steps: int, nodes):
    """Oracle (rho, ux, uy, uz, T) after `steps` steps at each (x, y, z) of `nodes`, each from a
    cut-out of the initial fields (arrays [nz, ny, nx]) of half-width R = 3 steps + 1 around the
    node: periodic wrap in x and y, clipped at the real walls in z. The cut-out's own edges (its
    wrap and its artificial walls) reach at most 2 steps + 1 nodes inward, so the centre is exact.
    Returns an array [len(nodes), 5]."""
    rho = np.asarray(rho)
    T = np.asarray(T)
    R = STEP_RADIUS * steps + 1
    out = np.empty((len(nodes), 5))
    for k, (x, y, z) in enumerate(nodes):
        out[k] = _cutout_centre(p, rho, T, steps, x, y, z, R)
    return out


def _cutout_centre(p, rho, T, steps, x, y, z, R):
    xs = np.arange(x - R, x + R + 1) % p.nx
    ys = np.arange(y - R, y + R + 1) % p.ny
    z_lo, z_hi = max(0, z - R), min(p.nz - 1, z + R)
    sub_r = np.ascontiguousarray(rho[z_lo:z_hi + 1][:, ys][:, :, xs])
    sub_t = np.ascontiguousarray(T[z_lo:z_hi + 1][:, ys][:, :, xs])
    q = dataclasses.replace(p, nx=2 * R + 1, ny=2 * R + 1, nz=z_hi - z_lo + 1)
    f, g, op, _ = oracle_run(q, sub_r, sub_t, steps)
    r_o, u_o, T_o = lbm.moments_out(f, g, op)
    c = (z - z_lo, R, R)
    return [float(r_o[c]), float(u_o[0][c]), float(u_o[1][c]), float(u_o[2][c]), float(T_o[c])]
