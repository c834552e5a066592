"""Statistics of a state, written plainly (FP64): per-plane profiles, the T-rho joint histogram
and horizontal structure functions (the paper's single-point analysis of Fig. 2, Eq. (5)'s
P div(u) term, and the two-point analysis of Eq. (10) / Fig. 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import lbm


def profiles(f, g, p: lbm.Params):
    """Per-plane means of rho, T and P div(u), P = rho T + (G/2) psi^2 (bulk pressure: with the
    paper's psi (G/2) e^{-2/rho}, with the van der Waals psi rho^2 (b T_v/(1 - b rho) - a))."""
    rho, u, T = lbm.moments_out(f, g, p)
    D = lbm.divergence(u, p)
    if p.psi_kind == "vdw":
        P = rho * T + rho * rho * (p.vdw_b * p.vdw_T / (1.0 - p.vdw_b * rho) - p.vdw_a)
    else:
        P = rho * T + 0.5 * p.G * torch.exp(-2.0 / rho)
    return rho.mean(dim=(1, 2)), T.mean(dim=(1, 2)), (P * D).mean(dim=(1, 2))


def histogram_T_rho(rho, T, z_lo, z_hi, nT, T_range, nr, r_range):
    """counts[iT, ir] of the nodes in planes [z_lo, z_hi) with lo <= v < hi in both variables,
    bin = floor((v - lo)/(hi - lo) n)."""
    rho = np.asarray(rho)[z_lo:z_hi].ravel()
    T = np.asarray(T)[z_lo:z_hi].ravel()
    counts = np.zeros((nT, nr), dtype=np.uint64)
    for t, r in zip(T, rho):
        if T_range[0] <= t < T_range[1] and r_range[0] <= r < r_range[1]:
            it = min(int(math.floor((t - T_range[0]) / (T_range[1] - T_range[0]) * nT)), nT - 1)
            ir = min(int(math.floor((r - r_range[0]) / (r_range[1] - r_range[0]) * nr)), nr - 1)
            counts[it, ir] += 1
    return counts


def structure_functions(uz, T, rmax, z_lo, z_hi):
    """S^(p)(r) = <(q(x + r e) - q(x))^p> over e = e_x, e_y (periodic) and the planes [z_lo, z_hi),
    for q = u_z, T and p = 2, 4; r = 1..rmax."""
    uz = torch.as_tensor(np.asarray(uz))[z_lo:z_hi]
    T = torch.as_tensor(np.asarray(T))[z_lo:z_hi]
    out = {k: np.zeros(rmax) for k in ("S2_uz", "S4_uz", "S2_T", "S4_T")}
    for r in range(1, rmax + 1):
        for name, q in (("uz", uz), ("T", T)):
            dx = torch.roll(q, shifts=-r, dims=2) - q
            dy = torch.roll(q, shifts=-r, dims=1) - q
            d = torch.cat([dx.reshape(-1), dy.reshape(-1)])
            out[f"S2_{name}"][r - 1] = (d ** 2).mean().item()
            out[f"S4_{name}"][r - 1] = (d ** 4).mean().item()
    return out


def heat_flux_pdf(f, g, p: lbm.Params, z_lo, z_hi, nbins, q_range):
    """Local convective heat flux q = rho U u_z (the bulk part of Nu, Eq. (4) and Fig. 2 inset)
    over the planes [z_lo, z_hi): counts of lo <= q < hi with bin = floor((q - lo)/(hi - lo) n),
    and (number of nodes, mean, variance) of q over every node of the planes."""
    rho, j, T, F, u_eq, u = lbm.macroscopic(f, g, p)
    U = lbm.internal_energy(rho, T, p)
    q = (rho * U * u[2])[z_lo:z_hi].reshape(-1).numpy()
    counts = np.zeros(nbins, dtype=np.uint64)
    lo, hi = q_range
    for v in q:
        if lo <= v < hi:
            counts[min(int(math.floor((v - lo) / (hi - lo) * nbins)), nbins - 1)] += 1
    n = q.size
    mean = float(np.sum(q) / n)
    var = float(np.sum((q - mean) ** 2) / n)
    return counts, (float(n), mean, var)

