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


# ---------------------------------------------------------------------------------------
# Van der Waals-type pseudopotential variant (a comparison, not the paper's psi):
# psi^2 = 2 (P_vdW(rho, T_v) - rho T_v) / G, so the bulk pressure of the lattice fluid is
# P = rho T + rho^2 (b T_v / (1 - b rho) - a): at T = T_v exactly the van der Waals pressure
# rho T/(1 - b rho) - a rho^2, whose critical point is rho_c = 1/(3b), T_c = 8a/(27b).
# ---------------------------------------------------------------------------------------

def pressure_vdw(rho, T, a, b, Tv):
    """P(rho, T) = rho T + rho^2 (b T_v/(1 - b rho) - a)."""
    return rho * T + rho * rho * (b * Tv / (1.0 - b * rho) - a)


def dP_drho_vdw(rho, T, a, b, Tv):
    """(dP/drho)_T = T + 2 rho b T_v/(1 - b rho) + rho^2 b^2 T_v/(1 - b rho)^2 - 2 a rho."""
    x = 1.0 - b * rho
    return T + 2.0 * rho * b * Tv / x + rho * rho * b * b * Tv / (x * x) - 2.0 * a * rho


def chemical_potential_vdw(rho, T, a, b, Tv):
    """mu with dmu = dP/rho at fixed T: T ln rho - T_v ln(1 - b rho) + T_v/(1 - b rho) - 2 a rho."""
    x = 1.0 - b * rho
    return T * np.log(rho) - Tv * np.log(x) + Tv / x - 2.0 * a * rho


def critical_point_vdw(a, b):
    """(rho_c, T_c, P_c) = (1/(3b), 8a/(27b), a/(27 b^2)) of the van der Waals pressure (T = T_v)."""
    return 1.0 / (3.0 * b), 8.0 * a / (27.0 * b), a / (27.0 * b * b)


def coexistence_vdw(T, a, b, Tv):
    """Maxwell construction of pressure_vdw at temperature T: (rho_g, rho_l)."""
    rc = 1.0 / (3.0 * b)
    f = lambda r: dP_drho_vdw(r, T, a, b, Tv)
    s_lo = brentq(f, 1e-6 * rc, rc)
    s_hi = brentq(f, rc, 0.999 / b)

    def eqs(x):
        rg, rl = x
        return [pressure_vdw(rg, T, a, b, Tv) - pressure_vdw(rl, T, a, b, Tv),
                chemical_potential_vdw(rg, T, a, b, Tv) - chemical_potential_vdw(rl, T, a, b, Tv)]

    rg, rl = fsolve(eqs, [0.5 * s_lo, min(1.3 * s_hi, 0.5 * (s_hi + 1.0 / b))], xtol=1e-12)
    if not (rg < s_lo < s_hi < rl):
        raise ValueError("Maxwell construction did not converge to a two-phase solution")
    return float(rg), float(rl)


def coexistence_psi_rule(P, psi, dpsi, s_lo, s_hi, eps, guess):
    """Flat-interface coexistence of a pseudopotential fluid with bulk pressure P(rho) and
    pseudopotential psi(rho): P(rho_g) = P(rho_l) = P0 and
    int_{rho_g}^{rho_l} (P0 - P(rho)) psi'(rho)/psi(rho)^(1+eps) drho = 0.
    eps = 0 is the equal-area rule in ln(psi) (Maxwell's rule when psi = exp(-c/rho));
    eps = 1 is the equal-area rule in 1/psi, the mechanical balance T rho' = -G psi (psi' +
    psi'''/6) of the Eq. (9) force expanded to third derivatives with an isotropic ideal part."""
    from scipy.integrate import quad

    def eqs(x):
        rg, rl = x
        P0 = P(rg)
        integ = quad(lambda r: (P0 - P(r)) * dpsi(r) / psi(r) ** (1.0 + eps), rg, rl,
                     epsabs=1e-14, epsrel=1e-12, limit=200)[0]
        return [P(rl) - P0, integ]

    rg, rl = fsolve(eqs, guess, xtol=1e-12)
    if not (rg < s_lo < s_hi < rl):
        raise ValueError("psi-rule construction did not converge to a two-phase solution")
    return float(rg), float(rl)
