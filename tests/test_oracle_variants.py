"""Pins of the oracle's two scheme variants (comparisons, not the paper's scheme):

- Guo forcing: the source term's moments (zeroth 0, first F, second uF + Fu), the momentum it
  adds (exactly F per node and step, as the velocity shift), and f^eq taken at the physical
  velocity;
- the van der Waals-type pseudopotential: psi^2 G/2 equals the non-ideal van der Waals pressure
  at T_v, the Eq. (9) force tends to minus its gradient, the internal energy is its integral,
  and the van der Waals thermodynamics (critical point, chemical potential, Maxwell rule);
- the psi-rule coexistence used for the flat-interface checks reduces to Maxwell's rule for the
  paper's psi.
"""
import math

import numpy as np
import pytest
import torch

from oracle import eos, lbm
from paper_1111_0905_gb300 import synthetic

DT = torch.float64
G0 = -math.e ** 2 * 10.0 / 27.0
TM = 1.0 / 3.0
A, B = 5.0 / 42.0, 2.0 / 21.0


def _rand(shape, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.rand(shape, generator=g, dtype=DT) * 2.0 - 1.0


def test_guo_source_moments():
    """sum_l S_l = 0, sum_l c_l S_l = F, sum_l c_l c_l S_l = u F + F u, for random u and F."""
    u = 0.1 * _rand((3, 4, 3, 2), 1)
    F = 0.01 * _rand((3, 4, 3, 2), 2)
    S = lbm.guo_source(u, F)
    assert S.sum(dim=0).abs().max() < 1e-17
    for a in range(3):
        m1 = sum(lbm.C[l][a] * S[l] for l in range(lbm.Q))
        assert (m1 - F[a]).abs().max() < 1e-17
        for b in range(3):
            m2 = sum(lbm.C[l][a] * lbm.C[l][b] * S[l] for l in range(lbm.Q))
            assert (m2 - (u[a] * F[b] + F[a] * u[b])).abs().max() < 1e-17


@pytest.mark.parametrize("forcing", ["shift", "guo"])
def test_uniform_force_adds_exactly_F_per_step(forcing):
    """Uniform density in a periodic box with gravity only: every step adds rho g_z to each
    node's z momentum and leaves the mass unchanged, for either forcing."""
    p = lbm.Params(3, 4, 5, 0.8, 1.0, 0.0, 0.05, g_z=-1e-3, T_d=TM, T_u=TM, periodic_z=True,
                   forcing=forcing)
    rho = torch.full((5, 4, 3), 1.7, dtype=DT)
    f, g = lbm.init_state(rho, torch.full_like(rho, TM), p)
    for n in range(1, 6):
        f, g = lbm.step(f, g, p)
        r, j = lbm.density_momentum(f)
        assert (r - 1.7).abs().max() < 1e-14
        assert (j[2] - n * 1.7 * -1e-3).abs().max() < 1e-15
        assert j[0].abs().max() < 1e-16 and j[1].abs().max() < 1e-16


def test_guo_collision_relaxes_to_the_physical_velocity():
    """With Guo forcing f^eq is taken at u = (j + F/2)/rho and the source adds (1 - 1/(2 tau)) S:
    the post-collision momentum is j + F and its second moment follows the Guo relation
    Pi* = Pi - (Pi - Pi^eq(u))/tau + (1 - 1/(2 tau))(u F + F u)."""
    p = lbm.Params(4, 5, 6, 0.9, 1.0, G0, 0.05, g_z=-2e-3, T_d=TM, T_u=TM, periodic_z=True,
                   forcing="guo")
    rho, T = synthetic.boiling_fields(4, 5, 6, 1.30, TM, TM)
    f, g = lbm.init_state(rho, T, p)
    f, g = lbm.step(f, g, p)          # a state away from equilibrium
    rho, j, T, F, u_eq, u = lbm.macroscopic(f, g, p)
    assert torch.equal(u_eq, u)
    fs, _, _ = lbm.collide(f, g, p)
    _, js = lbm.density_momentum(fs)
    assert (js - (j + F)).abs().max() < 1e-15
    feq = lbm.equilibrium_f(rho, u, T)
    for a in range(3):
        for b in range(3):
            m = lambda h: sum(lbm.C[l][a] * lbm.C[l][b] * h[l] for l in range(lbm.Q))
            want = m(f) - (m(f) - m(feq)) / p.tau_nu + (1 - 0.5 / p.tau_nu) * (u[a] * F[b] + F[a] * u[b])
            assert (m(fs) - want).abs().max() < 1e-14


def test_vdw_psi_closed_forms():
    """(G/2) psi^2 = rho^2 (b T_v/(1 - b rho) - a), so P = rho T + (G/2) psi^2 is the van der
    Waals pressure at T = T_v; U_NI' = P_NI/rho^2; mu' = P'/rho; critical point 1/(3b), 8a/(27b)."""
    p = lbm.Params(2, 2, 2, 1.0, 1.0, -1.0, 0.05, psi_kind="vdw", vdw_a=A, vdw_b=B, vdw_T=TM)
    rho = torch.linspace(0.3, 7.0, 50, dtype=DT)
    psi = lbm.psi_of(rho, p)
    pni = rho * rho * (B * TM / (1 - B * rho) - A)
    assert ((0.5 * p.G * psi * psi - pni).abs() / pni.abs()).max() < 1e-14
    vdw = rho * TM / (1 - B * rho) - A * rho * rho
    assert (eos.pressure_vdw(rho, TM, A, B, TM) - vdw).abs().max() < 1e-14
    h = 1e-6
    U = lambda r: lbm.internal_energy(r, torch.zeros_like(r), p)
    dU = (U(rho + h) - U(rho - h)) / (2 * h)
    assert (dU - pni / rho ** 2).abs().max() < 1e-8
    r = rho.numpy()
    dmu = (eos.chemical_potential_vdw(r + h, 0.3, A, B, TM) - eos.chemical_potential_vdw(r - h, 0.3, A, B, TM)) / (2 * h)
    assert np.abs(dmu - eos.dP_drho_vdw(r, 0.3, A, B, TM) / r).max() < 1e-7
    dP = (eos.pressure_vdw(r + h, 0.3, A, B, TM) - eos.pressure_vdw(r - h, 0.3, A, B, TM)) / (2 * h)
    assert np.abs(dP - eos.dP_drho_vdw(r, 0.3, A, B, TM)).max() < 1e-7
    rc, Tc, Pc = eos.critical_point_vdw(A, B)
    assert abs(Tc - 10.0 / 27.0) < 1e-15 and abs(rc - 3.5) < 1e-14
    assert abs(eos.dP_drho_vdw(rc, Tc, A, B, Tc)) < 1e-13
    d2 = (eos.dP_drho_vdw(rc + 1e-5, Tc, A, B, Tc) - eos.dP_drho_vdw(rc - 1e-5, Tc, A, B, Tc)) / 2e-5
    assert abs(d2) < 1e-8
    assert abs(eos.pressure_vdw(rc, Tc, A, B, Tc) - Pc) < 1e-14


def test_vdw_maxwell_construction_is_consistent():
    """The Maxwell construction of the van der Waals variant: equal P and mu, the liquid inside
    the range where psi is real, and Clausius-Clapeyron dP/dT = Delta s/Delta v with T = T_v."""
    Tc = 10.0 / 27.0
    T = 0.9 * Tc
    rg, rl = eos.coexistence_vdw(T, A, B, T)
    assert abs(eos.pressure_vdw(rg, T, A, B, T) - eos.pressure_vdw(rl, T, A, B, T)) < 1e-12
    assert abs(eos.chemical_potential_vdw(rg, T, A, B, T) - eos.chemical_potential_vdw(rl, T, A, B, T)) < 1e-11
    assert rl < (1 - B * T / A) / B
    # along the saturation curve of the full van der Waals fluid (T_v = T)
    h = 1e-4
    Psat = lambda t: eos.pressure_vdw(eos.coexistence_vdw(t, A, B, t)[0], t, A, B, t)
    dPdT = (Psat(T + h) - Psat(T - h)) / (2 * h)
    # entropy jump of the full vdW fluid: s = -ln(1/rho - b) + ..., Delta s = ln((1/rg - b)/(1/rl - b))
    ds = math.log((1 / rg - B) / (1 / rl - B))
    assert abs(dPdT / (ds / (1 / rg - 1 / rl)) - 1) < 1e-6


def _force_error(L, p):
    x = torch.arange(L, dtype=DT)
    k = 2 * math.pi / L
    sx, cx = torch.sin(k * x), torch.cos(k * x)
    rho = (4.0 + 0.8 * sx[None, :] * sx[:, None]).expand(2, L, L).clone()
    F = lbm.force(rho, p)
    drho_dx = (0.8 * k * cx[None, :] * sx[:, None]).expand(2, L, L)
    # minus the gradient of P_NI(rho) = rho^2 (b T_v/(1 - b rho) - a)
    dpni = 2 * rho * (B * TM / (1 - B * rho) - A) + rho * rho * B * B * TM / (1 - B * rho) ** 2
    ex = (F[0] + dpni * drho_dx).abs().max().item()
    return ex / (dpni * drho_dx).abs().max().item()


def test_vdw_force_tends_to_minus_grad_of_the_nonideal_pressure():
    """Eq. (9) with the van der Waals psi: F = -(G/2) grad psi^2 + O(h^2) = -grad P_NI."""
    p = lbm.Params(16, 16, 2, 1.0, 1.0, -1.0, 0.05, periodic_z=True, psi_kind="vdw",
                   vdw_a=A, vdw_b=B, vdw_T=TM)
    e16 = _force_error(16, p)
    p.nx = p.ny = 32
    e32 = _force_error(32, p)
    assert e16 < 0.06 and 3.5 < e16 / e32 < 4.5


@pytest.mark.parametrize("t", [0.8, 0.9, 0.95])
def test_psi_rule_reduces_to_maxwell_for_the_papers_psi(t):
    """With psi = exp(-1/rho), psi'/psi = 1/rho^2: the eps = 0 psi-rule is Maxwell's equal area in
    the specific volume, so both constructions give the same densities."""
    T = t * 10.0 / 27.0
    rg, rl = eos.coexistence(T, G0)
    lo, hi = eos.spinodal(T, G0)
    r0 = eos.coexistence_psi_rule(lambda r: eos.pressure(r, T, G0), lambda r: math.exp(-1 / r),
                                  lambda r: math.exp(-1 / r) / r ** 2, lo, hi, 0.0, [rg, rl])
    assert abs(r0[0] / rg - 1) < 1e-9 and abs(r0[1] / rl - 1) < 1e-9
