"""Equation of state of the pseudopotential fluid and its thermodynamics (FP64, scipy).

TEST INFRASTRUCTURE ONLY: used by the oracle's tests to pin the lattice against the
thermodynamics the paper states; the product path never imports it.

With psi = exp(-1/rho) and the force weights of Eq. (9) normalised as W = w/c_s^2, the bulk
pressure is P = rho T + (G/2) exp(-2/rho) (ideal part rho T, non-ideal part after Eq. (1)).
Reduced units: rho_c = 1, T_c = -G exp(-2), P_c = T_c / 2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq, fsolve


def pressure(rho, T, G):
    """P(rho, T) = rho T + (G/2) exp(-2/rho)."""
    return rho * T + 0.5 * G * np.exp(-2.0 / rho)


def dP_drho(rho, T, G):
    """(dP/drho)_T = T + G rho^-2 exp(-2/rho)."""
    return T + G * np.exp(-2.0 / rho) / (rho * rho)


def chemical_potential(rho, T, G):
    """mu(rho, T) with dmu = dP/rho at fixed T: T ln rho + (G/4)(2/rho + 1) exp(-2/rho)."""
    return T * np.log(rho) + 0.25 * G * (2.0 / rho + 1.0) * np.exp(-2.0 / rho)


def critical_point(G):
    """(rho_c, T_c, P_c) = (1, -G e^-2, -G e^-2 / 2): where dP/drho = d2P/drho2 = 0."""
    Tc = -G * math.exp(-2.0)
    return 1.0, Tc, 0.5 * Tc


def spinodal(T, G):
    """Densities where (dP/drho)_T = 0 (below T_c), bracketing the unstable branch."""
    f = lambda r: dP_drho(r, T, G)
    lo = brentq(f, 0.2, 1.0)
    hi = brentq(f, 1.0, 20.0)
    return lo, hi


def coexistence(T, G):
    """Maxwell construction: (rho_g, rho_l) with equal pressure and chemical potential."""
    s_lo, s_hi = spinodal(T, G)

    def eqs(x):
        rg, rl = x
        return [pressure(rg, T, G) - pressure(rl, T, G),
                chemical_potential(rg, T, G) - chemical_potential(rl, T, G)]

    guess = [0.5 * s_lo, 1.5 * s_hi]
    rg, rl = fsolve(eqs, guess, xtol=1e-12)
    if not (rg < s_lo < s_hi < rl):
        raise ValueError("Maxwell construction did not converge to a two-phase solution")
    return float(rg), float(rl)


def saturation_pressure(T, G):
    rg, rl = coexistence(T, G)
    return float(pressure(rg, T, G))


def entropy_jump(rho_g, rho_l):
    """s_g - s_l = ln(rho_l / rho_g): with P = rho T + P_NI(rho), (ds/dv)_T = (dP/dT)_v = rho."""
    return math.log(rho_l / rho_g)


def beta(rho, T, G):
    """Isobaric expansion coefficient -(d rho/dT)_P / rho = 1/(dP/drho)_T for this EOS."""
    return 1.0 / dP_drho(rho, T, G)


def c_p(rho, T, G, c_v=1.0):
    """c_p = c_v + T (dP/dT)_rho^2 / (rho^2 (dP/drho)_T) = c_v + T beta."""
    return c_v + T * beta(rho, T, G)


def rayleigh(g, rho, T, G, L, dT, kappa, nu, c_v=1.0):
    """Ra = g beta L^4 (dT/L - gamma_ad) / (chi nu), chi = kappa/(rho c_p), gamma_ad = beta T g / c_p (Table 1)."""
    b = beta(rho, T, G)
    cp = c_p(rho, T, G, c_v)
    chi = kappa / (rho * cp)
    return g * b * L ** 4 * (dT / L - b * T * g / cp) / (chi * nu)
