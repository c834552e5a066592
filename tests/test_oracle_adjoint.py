"""Pins of the objective of the adjoint (time-averaged Nu) and of the oracle's exact discrete
gradient (PyTorch autograd through the plain steps) against central finite differences."""
import math

import numpy as np
import pytest
import torch

from oracle import lbm
from paper_1111_0905_gb300 import config

DT = torch.float64


def _setup(n=6, nz=6):
    w = config.boiling_cell(n, nz=nz)
    pp = w.params
    rho, T = w.fields()
    p = lbm.Params(pp.nx, pp.ny, pp.nz, pp.tau_nu, pp.tau_kappa, pp.G, pp.kappa, pp.c_v, pp.g_z,
                   pp.T_d, pp.T_u)
    return p, torch.from_numpy(rho), torch.from_numpy(T)


def test_mean_nusselt_is_one_plus_convective_flux():
    """Sum_z of the central dT/dz with the wall ghosts telescopes to T_u - T_d per column, so
    Nu_mean = 1 + sum_z <rho U u_z> / (kappa (T_d - T_u)) exactly."""
    p, rho, T = _setup(6, 7)
    f, g = lbm.init_state(rho, T, p)
    f, g = lbm.run(f, g, p, 5)
    nu_mean, _ = lbm.nusselt(f, g, p)
    r, u, TT = lbm.moments_out(f, g, p)
    conv = (r * lbm.internal_energy(r, TT, p) * u[2]).mean(dim=(1, 2)).sum()
    assert abs(nu_mean.item() - (1 + conv.item() / (p.kappa * (p.T_d - p.T_u)))) < 1e-12


def test_oracle_gradient_matches_central_differences():
    """dJ/d(T_d, T_u, G) and dJ/dT0 (two directions) from autograd vs central differences."""
    p, rho, T = _setup(5, 5)
    N = 6
    Td = torch.tensor(p.T_d, dtype=DT, requires_grad=True)
    Tu = torch.tensor(p.T_u, dtype=DT, requires_grad=True)
    G = torch.tensor(p.G, dtype=DT, requires_grad=True)
    T0 = T.clone().requires_grad_(True)
    q = lbm.Params(p.nx, p.ny, p.nz, p.tau_nu, p.tau_kappa, G, p.kappa, p.c_v, p.g_z, Td, Tu)
    J = lbm.time_averaged_nusselt(rho, T0, q, N)
    J.backward()
    grads = {"T_d": Td.grad.item(), "T_u": Tu.grad.item(), "G": G.grad.item()}

    def J_of(**kw):
        pq = lbm.Params(p.nx, p.ny, p.nz, p.tau_nu, p.tau_kappa, kw.get("G", p.G), p.kappa, p.c_v,
                        p.g_z, kw.get("T_d", p.T_d), kw.get("T_u", p.T_u))
        return lbm.time_averaged_nusselt(rho, kw.get("T0", T), pq, N).item()

    h = 1e-6
    for name, base in [("T_d", p.T_d), ("T_u", p.T_u), ("G", p.G)]:
        fd = (J_of(**{name: base + h}) - J_of(**{name: base - h})) / (2 * h)
        assert abs(fd - grads[name]) <= 1e-6 * max(1.0, abs(fd)), (name, fd, grads[name])
    gen = torch.Generator().manual_seed(3)
    for _ in range(2):
        v = torch.randn(T.shape, generator=gen, dtype=DT)
        fd = (J_of(T0=T + h * v) - J_of(T0=T - h * v)) / (2 * h)
        ad = (T0.grad * v).sum().item()
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(fd)), (fd, ad)


def test_forward_mode_agrees_with_reverse_mode():
    """Forward-mode (dual-number) JVP of J through the oracle equals the reverse-mode gradient
    contracted with the same direction of T0."""
    from torch.func import jvp
    p, rho, T = _setup(5, 4)
    N = 5
    v = torch.randn(T.shape, generator=torch.Generator().manual_seed(11), dtype=DT)
    _, tangent = jvp(lambda t0: lbm.time_averaged_nusselt(rho, t0, p, N), (T,), (v,))
    T0 = T.clone().requires_grad_(True)
    lbm.time_averaged_nusselt(rho, T0, p, N).backward()
    assert abs(tangent.item() - (T0.grad * v).sum().item()) <= 1e-10 * max(1.0, abs(tangent.item()))
