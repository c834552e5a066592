"""Workload definitions: the synthetic cells the tests and the benchmark run.

Parameters follow the paper's setting (Table 1, Fig. 1 caption, the text around Eq. (4)):
D3Q19, periodic x/y, no-slip walls with fixed T_d (bottom) and T_u (top), psi = exp(-1/rho).
With the force weights W = w/c_s^2 the bulk pressure is P = rho T + (G/2) e^{-2/rho}, so the
critical point is rho_c = 1, T_c = -G e^{-2}. G is chosen so that T_c = 10/27 and the mean
temperature T_m = 0.9 T_c = 1/3 equals the lattice c_s^2. T_d/T_u sit 5 % above/below T_m.

Derived quantities (Table 1 caption): beta = 1/(dP/drho)_T, c_p = c_v + T beta,
chi = kappa/(rho c_p), Pr = nu/chi, Ra = g beta L^4 (dT/L - gamma_ad)/(chi nu) with the
adiabatic gradient gamma_ad = beta T g / c_p, viscosity nu = T_m (tau_nu - 1/2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import synthetic
from .lb import LB_FP64, Params

T_C = 10.0 / 27.0
G_DEFAULT = -math.exp(2.0) * T_C
T_M = 0.9 * T_C
T_D = 1.05 * T_M
T_U = 0.95 * T_M


def dP_drho(rho: float, T: float, G: float = G_DEFAULT) -> float:
    """Isothermal slope of P = rho T + (G/2) e^{-2/rho}."""
    return T + G * math.exp(-2.0 / rho) / (rho * rho)


def beta_cp(rho: float, T: float, G: float = G_DEFAULT, c_v: float = 1.0):
    b = 1.0 / dP_drho(rho, T, G)
    return b, c_v + T * b


def kappa_from_prandtl(Pr: float, nu: float, rho: float, T: float, G: float = G_DEFAULT, c_v=1.0):
    """kappa such that nu / (kappa/(rho c_p)) = Pr."""
    _, cp = beta_cp(rho, T, G, c_v)
    return nu / Pr * rho * cp


def gravity_from_rayleigh(Ra: float, L: float, dT: float, kappa: float, nu: float, rho: float,
                          T: float, G: float = G_DEFAULT, c_v=1.0) -> float:
    """Smaller positive root g of Ra = g beta L^4 (dT/L - beta T g/c_p)/(chi nu); returns -g
    (downward). Raises if Ra exceeds the largest value the adiabatic gradient allows."""
    b, cp = beta_cp(rho, T, G, c_v)
    chi = kappa / (rho * cp)
    a2 = b * b * T * L ** 4 / cp
    a1 = b * L ** 4 * dT / L
    a0 = Ra * chi * nu
    disc = a1 * a1 - 4.0 * a2 * a0
    if disc < 0:
        raise ValueError(f"Ra={Ra:g} is above the maximum {a1 * a1 / (4 * a2) / (chi * nu):.3g} for L={L}")
    return -(a1 - math.sqrt(disc)) / (2.0 * a2)


@dataclass
class Workload:
    name: str
    params: Params
    rho_mean: float
    kind: str          # "boiling" (density noise) or "single_phase" (temperature noise)
    steps: int

    def fields(self, seed: int = synthetic.SEED):
        p = self.params
        if self.kind == "boiling":
            return synthetic.boiling_fields(p.nx, p.ny, p.nz, self.rho_mean, p.T_d, p.T_u, 0.01, seed)
        return synthetic.single_phase_fields(p.nx, p.ny, p.nz, self.rho_mean, p.T_d, p.T_u, 0.01, seed)


def boiling_cell(n: int = 32, nz: int | None = None, precision: int = LB_FP64, steps: int = 200,
                 ny: int | None = None, kappa: float = 0.05, tau_nu: float = 1.0) -> Workload:
    """Plain boiling cell: rho = 1.30 (1 + 0.01 xi) inside the spinodal at T_m, T linear in z,
    tau_nu = tau_kappa = 1, kappa = 0.05, g_z = -1e-5 (the 200-step parity cell). The spinodal
    decomposition at tau_nu = 1 breaks down after ~500 steps; long runs use tau_nu >= 1.25 with
    lambda = kappa/(tau_kappa - 1/2) inside the g^eq positivity window rho_l/9 .. 5 rho_g/9."""
    p = Params(nx=n, ny=n if ny is None else ny, nz=n if nz is None else nz, tau_nu=tau_nu,
               tau_kappa=1.0, G=G_DEFAULT, kappa=kappa, c_v=1.0, g_z=-1e-5, T_d=T_D, T_u=T_U,
               precision=precision)
    return Workload(f"boiling_{p.nx}x{p.ny}x{p.nz}", p, 1.30, "boiling", steps)


def max_rayleigh(L: float, dT: float, kappa: float, nu: float, rho: float, T: float,
                 G: float = G_DEFAULT, c_v=1.0) -> float:
    """Largest Ra reachable at height L once the adiabatic gradient is subtracted."""
    b, cp = beta_cp(rho, T, G, c_v)
    chi = kappa / (rho * cp)
    a2 = b * b * T * L ** 4 / cp
    a1 = b * L ** 4 * dT / L
    return a1 * a1 / (4.0 * a2) / (chi * nu)


# Relaxation times of the synthetic cells. With the temperature of g in the f equilibrium the
# uniform state is linearly unstable for small tau_nu (checkerboard modes; the paper's
# nu = 0.0165, tau_nu = 0.5495, has spectral radius > 1.7), and long runs need more: at
# tau_nu = 1 the single-phase cell (measured) and the phase-separating cells break down within
# ~1000 steps. The single-phase cell runs at tau_nu = 1.25, tau_kappa = 1 (Pr = 9, lambda = 0.49
# inside the g^eq positivity window [rho/9, 5 rho/9]; bounded over 10,000 steps, measured).
TAU_NU = 1.25
TAU_KAPPA = 1.0
# Boiling cells at the paper's geometry: tau_nu = 1.25, tau_kappa = 1.5 (Pr = 9, lambda = 0.36);
# bounded over 10,000 steps at 64^3 with T inside [T_u, T_d] (measured; tau_kappa = 1.75 drifted).
TAU_NU_BOILING = 1.25
TAU_KAPPA_BOILING = 1.5


def single_phase_cell(n: int = 128, precision: int = LB_FP64, steps: int = 2000,
                      ra_fraction: float = 0.5) -> Workload:
    """Single-phase convection: compressed liquid rho = 2.30 (above the liquid branch at every T
    of the cell), T linear with 1 % seeded noise, Pr = 9 at the cell centre, gravity from
    Ra = ra_fraction * (largest Ra reachable at L = n)."""
    nu = T_M * (TAU_NU - 0.5)
    kappa = kappa_from_prandtl(9.0, nu, 2.30, T_M)
    Ra = ra_fraction * max_rayleigh(n, T_D - T_U, kappa, nu, 2.30, T_M)
    gz = gravity_from_rayleigh(Ra, n, T_D - T_U, kappa, nu, 2.30, T_M)
    p = Params(nx=n, ny=n, nz=n, tau_nu=TAU_NU, tau_kappa=TAU_KAPPA, G=G_DEFAULT, kappa=kappa,
               c_v=1.0, g_z=gz, T_d=T_D, T_u=T_U, precision=precision)
    return Workload(f"single_phase_{n}^3", p, 2.30, "single_phase", steps)


def paper_scale_cell(n: int = 512, precision: int = LB_FP64, steps: int = 1000,
                     ra_fraction: float = 0.5) -> Workload:
    """Boiling cell at the paper's geometry (L = 512, Table 1): rho = 1.50 (1 + 0.01 xi) inside
    coexistence (T_d above the local saturation temperature), tau_nu = 1.25, tau_kappa = 1.5,
    Pr = 9 at the liquid density of T_m, gravity from Ra = ra_fraction * (largest Ra reachable
    at L = n)."""
    rho_l = 1.788830  # liquid coexistence density at T_m = 0.9 T_c for this EOS
    nu = T_M * (TAU_NU_BOILING - 0.5)
    kappa = kappa_from_prandtl(9.0, nu, rho_l, T_M)
    Ra = ra_fraction * max_rayleigh(n, T_D - T_U, kappa, nu, rho_l, T_M)
    gz = gravity_from_rayleigh(Ra, n, T_D - T_U, kappa, nu, rho_l, T_M)
    p = Params(nx=n, ny=n, nz=n, tau_nu=TAU_NU_BOILING, tau_kappa=TAU_KAPPA_BOILING, G=G_DEFAULT, kappa=kappa,
               c_v=1.0, g_z=gz, T_d=T_D, T_u=T_U, precision=precision)
    return Workload(f"boiling_{n}^3", p, 1.50, "boiling", steps)
