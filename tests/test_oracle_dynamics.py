"""Pins of the oracle's time step against conservation laws, closed forms and continuum limits.

Each test checks a property the paper or the mathematics fixes independently of the oracle's
own code: exact mass conservation with halfway walls, momentum conservation of the pair force
(Eq. (9)) in a periodic box, the gradient limit of Eq. (9), the shear viscosity of Eq. (6),
the adiabatic sound speed produced by the counter term (Eq. (3), second line), the linear
conduction profile with the wall temperatures and Nu = 1, the conducted energy flux (the
magnitude of kappa and the c_v factor), and a fixed point at rest.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lbm
from paper_1111_0905_gb300 import synthetic

DT = torch.float64
G0 = -math.e ** 2 * 10.0 / 27.0
TM = 1.0 / 3.0


def test_rest_state_is_a_fixed_point():
    """Uniform rho, T with T_d = T_u = T and no gravity: steps return f^eq, g^eq (to rounding)."""
    p = lbm.Params(6, 5, 4, 0.8, 0.9, G0, 0.1, T_d=TM, T_u=TM)
    rho = torch.full((4, 5, 6), 1.7, dtype=DT)
    T = torch.full((4, 5, 6), TM, dtype=DT)
    f0, g0 = lbm.init_state(rho, T, p)
    f, g = lbm.run(f0, g0, p, 3)
    assert torch.allclose(f, f0, rtol=1e-14, atol=0)
    assert torch.allclose(g, g0, rtol=1e-14, atol=0)


def test_mass_is_conserved_with_walls():
    """Halfway bounce-back and BGK conserve sum(rho) exactly (to rounding)."""
    p = lbm.Params(8, 8, 8, 1.0, 1.0, G0, 0.05, g_z=-1e-5, T_d=1.05 * TM, T_u=0.95 * TM)
    rho, T = synthetic.boiling_fields(8, 8, 8, 1.30, p.T_d, p.T_u)
    f, g = lbm.init_state(rho, T, p)
    m0 = f.sum().item()
    f, g = lbm.run(f, g, p, 60)
    assert abs(f.sum().item() - m0) / m0 < 1e-13


def test_momentum_is_conserved_periodic():
    """Fully periodic, no gravity: the pair force of Eq. (9) is antisymmetric, so sum(j) is
    conserved: post-collision momentum is j + F and sum(F) = 0."""
    p = lbm.Params(6, 7, 5, 0.9, 1.0, G0, 0.05, T_d=TM, T_u=TM, periodic_z=True)
    rho, T = synthetic.boiling_fields(6, 7, 5, 1.30, TM, TM)
    f, g = lbm.init_state(rho, torch.full_like(torch.as_tensor(T), TM), p)
    F = lbm.force(lbm.density_momentum(f)[0], p)
    assert F.abs().max() > 1e-3
    assert F.sum(dim=(1, 2, 3)).abs().max() < 1e-15 * 210
    j0 = lbm.density_momentum(f)[1].sum(dim=(1, 2, 3))
    f, g = lbm.run(f, g, p, 40)
    j1 = lbm.density_momentum(f)[1].sum(dim=(1, 2, 3))
    assert (j1 - j0).abs().max() < 1e-13


def _force_gradient_error(L):
    """Max |F + G psi grad psi| for rho = 1.2 + 0.3 sin(2 pi x/L) sin(2 pi y/L)."""
    p = lbm.Params(L, L, 2, 1.0, 1.0, G0, 0.05, periodic_z=True)
    x = torch.arange(L, dtype=DT)
    k = 2 * math.pi / L
    sx, cx = torch.sin(k * x), torch.cos(k * x)
    rho = (1.2 + 0.3 * sx[None, :] * sx[:, None]).expand(2, L, L).clone()
    F = lbm.force(rho, p)
    ps = torch.exp(-1.0 / rho)
    drho_dx = (0.3 * k * cx[None, :] * sx[:, None]).expand(2, L, L)
    drho_dy = (0.3 * k * sx[None, :] * cx[:, None]).expand(2, L, L)
    dpsi = ps / rho ** 2
    ex = (F[0] + G0 * ps * dpsi * drho_dx).abs().max().item()
    ey = (F[1] + G0 * ps * dpsi * drho_dy).abs().max().item()
    assert F[2].abs().max() < 1e-16
    return max(ex, ey), (G0 * ps * dpsi * drho_dx).abs().max().item()


def test_force_tends_to_minus_G_psi_grad_psi():
    """Eq. (9) with W = (1/6, 1/12): F = -G psi grad(psi) + O(h^2); the error drops ~4x per
    halving of the grid spacing (relative to the gradient). Pins the force weights, signs and the G normalisation."""
    e16, s16 = _force_gradient_error(16)
    e32, s32 = _force_gradient_error(32)
    r16, r32 = e16 / s16, e32 / s32
    assert r16 < 0.06
    assert 3.5 < r16 / r32 < 4.5


def test_shear_wave_viscosity():
    """Eq. (6): a transverse wave decays at nu k^2 with nu = T (tau_nu - 1/2) (T = c_s^2 = 1/3)."""
    L, tau = 32, 0.8
    p = lbm.Params(1, L, 2, tau, 1.0, 0.0, 0.05, T_d=TM, T_u=TM, periodic_z=True)
    y = torch.arange(L, dtype=DT)
    k = 2 * math.pi / L
    rho = torch.ones((2, L, 1), dtype=DT)
    T = torch.full((2, L, 1), TM, dtype=DT)
    u = torch.zeros((3, 2, L, 1), dtype=DT)
    u[2] = 1e-4 * torch.sin(k * y)[None, :, None]
    f, g = lbm.equilibrium_f(rho, u, T), lbm.equilibrium_g(rho, T, u, p.lam)
    amp = []
    for n in range(301):
        if n in (100, 300):
            _, uu, _ = lbm.moments_out(f, g, p)
            amp.append((uu[2][0, :, 0] * torch.sin(k * y)).sum().item() * 2 / L)
        f, g = lbm.step(f, g, p)
    nu = -math.log(amp[1] / amp[0]) / 200 / k ** 2
    assert abs(nu / (TM * (tau - 0.5)) - 1) < 0.01


@pytest.mark.parametrize("c_v", [1.0, 2.0])
def test_adiabatic_sound_speed_from_counter_term(c_v):
    """With the counter term, Eq. (3) line 2 makes sound adiabatic: c^2 = (1 + 1/c_v) T for
    P0 = rho T. Without it (or with the wrong sign) c^2 would be T (or (1 - 1/c_v) T)."""
    L = 64
    p = lbm.Params(L, 1, 1, 1.0, 1.0, 0.0, 1e-4, c_v=c_v, T_d=TM, T_u=TM, periodic_z=True)
    x = torch.arange(L, dtype=DT)
    k = 2 * math.pi / L
    eps = 1e-4
    rho = (1 + eps * torch.cos(k * x))[None, None, :].clone()
    T = (TM * (1 + eps / c_v * torch.cos(k * x)))[None, None, :].clone()
    f, g = lbm.init_state(rho, T, p)
    A = []
    for n in range(60):
        r, _, _ = lbm.moments_out(f, g, p)
        A.append(((r[0, 0] - 1) * torch.cos(k * x)).sum().item() * 2 / L)
        f, g = lbm.step(f, g, p)
    A = np.array(A)
    i = int(np.where(np.sign(A[:-1]) != np.sign(A[1:]))[0][0])
    t_quarter = i + A[i] / (A[i] - A[i + 1])
    c2 = ((math.pi / 2) / t_quarter / k) ** 2
    assert abs(c2 / ((1 + 1 / c_v) * TM) - 1) < 0.03


def test_conduction_profile_and_unit_nusselt():
    """No gravity, ideal fluid: the steady state is at rest with T linear between T_d at z=-1/2
    and T_u at z=nz-1/2 (constant kappa), and Nu(z) = 1 at every z (Eq. (4) normalisation)."""
    nz = 8
    Td, Tu = 1.05 * TM, 0.95 * TM
    p = lbm.Params(2, 2, nz, 1.0, 1.0, 0.0, 0.1, c_v=1.0, g_z=0.0, T_d=Td, T_u=Tu)
    z = (torch.arange(nz, dtype=DT) + 0.5) / nz
    Tlin = Td + (Tu - Td) * z
    T = Tlin[:, None, None].expand(nz, 2, 2).clone()
    rho = (TM / T)                               # uniform pressure rho T
    f, g = lbm.init_state(rho, T, p)
    f, g = lbm.run(f, g, p, 1500)
    r, u, TT = lbm.moments_out(f, g, p)
    assert (TT[:, 0, 0] - Tlin).abs().max() < 1e-9
    assert u.abs().max() < 1e-9
    nu_mean, nu_z = lbm.nusselt(f, g, p)
    assert (nu_z - 1).abs().max() < 1e-6


def test_nusselt_of_an_exact_conduction_state_is_one():
    """Nu(z) of a state at rest with the linear wall-to-wall profile is 1 to rounding."""
    nz = 10
    Td, Tu = 0.36, 0.30
    p = lbm.Params(3, 2, nz, 1.0, 1.0, 0.0, 0.07, g_z=0.0, T_d=Td, T_u=Tu)
    z = (torch.arange(nz, dtype=DT) + 0.5) / nz
    T = (Td + (Tu - Td) * z)[:, None, None].expand(nz, 2, 3).clone()
    rho = torch.ones_like(T)
    f, g = lbm.init_state(rho, T, p)
    nu_mean, nu_z = lbm.nusselt(f, g, p)
    assert (nu_z - 1).abs().max() < 1e-12


@pytest.mark.parametrize("c_v,kappa,tau_k", [(1.0, 0.1, 1.0), (2.0, 0.1, 1.0), (1.0, 0.05, 1.0),
                                             (1.0, 0.1, 1.5)])
def test_conducted_energy_flux_is_kappa_over_cv_times_the_gradient(c_v, kappa, tau_k):
    """The magnitude of the conductivity (which the linear profile and Nu = 1 above do not fix):
    in the steady conduction state the energy rho T that streaming carries across each interior
    plane per step, sum of g*_l(z) over c_lz = +1 minus sum of g*_l(z+1) over c_lz = -1, equals
    kappa (T_d - T_u)/L, the conduction flux of Eq. (3), divided by c_v (the g lattice carries
    rho T, not rho c_v T), with L = nz between the halfway walls."""
    nz = 8
    Td, Tu = 1.05 * TM, 0.95 * TM
    p = lbm.Params(2, 2, nz, 1.0, tau_k, 0.0, kappa, c_v=c_v, g_z=0.0, T_d=Td, T_u=Tu)
    z = (torch.arange(nz, dtype=DT) + 0.5) / nz
    T = (Td + (Tu - Td) * z)[:, None, None].expand(nz, 2, 2).clone()
    rho = TM / T
    f, g = lbm.init_state(rho, T, p)
    f, g = lbm.run(f, g, p, 2000)
    _, gs, _ = lbm.collide(f, g, p)
    up = [l for l in range(lbm.Q) if lbm.C[l][2] == 1]
    down = [l for l in range(lbm.Q) if lbm.C[l][2] == -1]
    want = kappa / c_v * (Td - Tu) / nz
    for k in range(nz - 1):
        q = sum(gs[l, k].mean() for l in up) - sum(gs[l, k + 1].mean() for l in down)
        assert abs(float(q) / want - 1) < 1e-7, (k, float(q), want)
