"""Physics validation of the CUDA path at GPU scale (the paper's Fig. 1 checks and the
classical limits), each with its oracle counterpart at small size in the CPU tests.

- Flat liquid slabs at T/T_c = 0.80 ... 0.95: bulk densities vs the Maxwell construction of
  P = rho T + (G/2) e^{-2/rho}, and the Clausius-Clapeyron relation dP/dT = Delta s / Delta v
  along the simulated coexistence curve (Fig. 1).
- Static 3-D bubbles: Laplace law Delta P = 2 sigma / R (linear in 1/R).
- Conduction below onset: linear T between the walls and Nu = 1.
- Scheme variants: with Guo forcing the flat-interface densities do not depend on tau_nu and
  sit on the Maxwell construction (the velocity shift's tau bias disappears); with the van der
  Waals psi they follow the psi-rule of the pseudopotential (equal area in ln psi).
- Rayleigh-Benard rolls (quasi-2-D, aspect 2.016 = the rigid-rigid critical wavelength): a roll
  perturbation decays at half the nominal onset Rayleigh number 1708 and grows into steady
  convection (Nu > 1.3) at twice it, with FP32 and FP64 agreeing on Nu; in the stationary rolls
  Nu(z) obeys the integral constraint of Eq. (5) with the P div(u) profile.
- Onset: over one and a half thermal diffusion times the roll decays at Ra = 1707.76 (the
  rigid-rigid critical value of the Oberbeck-Boussinesq limit) and grows at 1.05 times it
  (alpha dT = 0.46); at half the temperature difference (alpha dT = 0.23, L = 128, from the relaxed
  base state) it decays at 1.00 and grows at 1.02 times it: the critical Rayleigh number of the
  compressible cell approaches the classical one as alpha dT falls.
"""
import math

import numpy as np
import pytest
import torch

from oracle import eos
from paper_1111_0905_gb300 import config, lb

pytestmark = pytest.mark.gpu
G0 = config.G_DEFAULT
TC = config.T_C


def _run(p, rho, T, steps, precision=lb.LB_FP64):
    q = lb.Params(**{**p.__dict__, "precision": precision})
    lat = lb.Lattice(q, rho, T)
    lat.step(steps)
    r, u, TT = lat.moments()
    lat.close()
    return r, u, TT


def _slab(t, nz=96, steps=30000):
    T0 = t * TC
    rg, rl = eos.coexistence(T0, G0)
    p = lb.Params(nx=4, ny=4, nz=nz, tau_nu=1.0, tau_kappa=1.0, G=G0, kappa=0.24, g_z=0.0,
                  T_d=T0, T_u=T0)
    z = np.arange(nz) + 0.5
    prof = 0.5 * (np.tanh((z - nz / 4) / 2.5) - np.tanh((z - 3 * nz / 4) / 2.5))
    rho = np.broadcast_to((rg + (rl - rg) * prof)[:, None, None], (nz, 4, 4)).copy()
    T = np.full_like(rho, T0)
    r, u, TT = _run(p, rho, T, steps)
    return r[nz // 2].mean(), r[1].mean(), rl, rg, float(np.abs(TT / T0 - 1).max())


def test_flat_interfaces_maxwell_and_clausius_clapeyron():
    ts = [0.80, 0.85, 0.90, 0.95]
    res = {t: _slab(t) for t in ts}
    for t, (rl_m, rg_m, rl, rg, dT) in res.items():
        print(f"T/Tc={t}: rho_l {rl_m:.5f} (Maxwell {rl:.5f}, {100*(rl_m/rl-1):+.2f} %), "
              f"rho_g {rg_m:.5f} (Maxwell {rg:.5f}, {100*(rg_m/rg-1):+.2f} %), max |dT/T| {dT:.1e}")
        assert abs(rl_m / rl - 1) < 0.02 and abs(rg_m / rg - 1) < 0.06 and dT < 1e-2
    # Clausius-Clapeyron on the simulated coexistence curve: P_sat(T) from the bulk EOS at the
    # measured liquid density; dP/dT by central differences vs Delta s / Delta v at the centre
    for i in (1, 2):
        tm, t0, tp = ts[i - 1], ts[i], ts[i + 1]
        P = lambda t: eos.pressure(res[t][0], t * TC, G0)
        dPdT = (P(tp) - P(tm)) / ((tp - tm) * TC)
        rl_m, rg_m = res[t0][0], res[t0][1]
        ds_dv = math.log(rl_m / rg_m) / (1 / rg_m - 1 / rl_m)
        print(f"T/Tc={t0}: dP/dT {dPdT:.5f} vs Delta s/Delta v {ds_dv:.5f} ({100*(dPdT/ds_dv-1):+.2f} %)")
        # at tau_nu = 1 the velocity-shift forcing biases the coexistence densities (largest in
        # the vapour at low T), which the relation inherits; the paper's tau_nu = 0.55 would
        # reduce the bias ~100x but is linearly unstable under these readings
        assert abs(dPdT / ds_dv - 1) < 0.10


def test_laplace_law_for_static_droplets():
    """Liquid droplets of radius R in vapour at T = 0.9 T_c, far from the walls: the pressure
    jump from the bulk EOS is linear in 1/R with an intercept near zero. The droplets start from
    the lattice's own flat-interface densities at this T (measured above: 0.5815, 1.8047)."""
    T0 = 0.9 * TC
    rg, rl = 0.5815, 1.8047
    n = 80
    p = lb.Params(nx=n, ny=n, nz=n, tau_nu=1.0, tau_kappa=1.0, G=G0, kappa=0.24, g_z=0.0,
                  T_d=T0, T_u=T0)
    c = (np.arange(n) + 0.5 - n / 2)
    r3 = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    inv_R, dP = [], []
    for R in (10.0, 14.0, 18.0):
        rho = rg + (rl - rg) * 0.5 * (1 - np.tanh((r3 - R) / 2.5))
        T = np.full_like(rho, T0)
        r, u, TT = _run(p, rho, T, 12000, precision=lb.LB_FP32)
        P = eos.pressure(r, TT, G0)
        P_in = P[n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1].mean()
        P_out = P[n // 2, n // 2, 2:6].mean()
        # equimolar radius from the excess mass over the vapour, with the measured bulk densities
        rho_in = r[n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1].mean()
        rho_out = r[n // 2, n // 2, 2:6].mean()
        vol = float(np.sum(r - rho_out) / (rho_in - rho_out))
        R_eq = (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
        assert R_eq > 4, f"droplet of initial radius {R} did not survive (R = {R_eq})"
        inv_R.append(1.0 / R_eq)
        dP.append(P_in - P_out)
        print(f"R0={R}: R={R_eq:.2f}, dP={P_in - P_out:.5e}, max|u|={np.abs(np.stack(u)).max():.2e}")
    A = np.vstack([inv_R, np.ones(3)]).T
    (slope, icpt), res, *_ = np.linalg.lstsq(A, np.array(dP), rcond=None)
    pred = A @ np.array([slope, icpt])
    r2 = 1 - np.sum((np.array(dP) - pred) ** 2) / np.sum((np.array(dP) - np.mean(dP)) ** 2)
    print(f"Laplace: 2 sigma = {slope:.5e}, intercept {icpt:.2e}, R^2 = {r2:.5f}")
    assert slope > 0 and r2 > 0.995 and abs(icpt) < 0.1 * abs(slope) * max(inv_R)


def test_conduction_profile_and_nusselt_one():
    """No gravity, single phase: steady T linear between T_d (z=-1/2) and T_u (z=nz-1/2),
    fluid at rest, Nu(z) = 1."""
    nz = 32
    Td, Tu = config.T_D, config.T_U
    p = lb.Params(nx=16, ny=16, nz=nz, tau_nu=1.0, tau_kappa=1.0, G=0.0, kappa=0.3, g_z=0.0,
                  T_d=Td, T_u=Tu)
    z = (np.arange(nz) + 0.5) / nz
    Tlin = Td + (Tu - Td) * z
    T = np.broadcast_to(Tlin[:, None, None], (nz, 16, 16)).copy()
    rho = (1.0 / 3.0) / T
    lat = lb.Lattice(p, rho, T)
    lat.step(20000)
    r, u, TT = lat.moments()
    nu_mean, nu_z, _ = lat.nusselt()
    lat.close()
    assert np.abs(TT[:, 0, 0] - Tlin).max() < 1e-8
    assert np.abs(np.stack(u)).max() < 1e-8
    assert np.abs(nu_z - 1).max() < 1e-6


def _rolls(ratio, precision, L=64):
    """Compressed liquid rho = 2.6 between T_d = 1.1 T_m and T_u = 0.9 T_m, Pr = 9, gravity from
    Ra = ratio * 1707.76 (Table 1 definition with the adiabatic gradient); T perturbed by
    1e-3 dT sin(k x) sin(pi z / L) with k the critical wavenumber of the box 2.016 L x 1 x L."""
    Tm = config.T_M
    Td, Tu = 1.1 * Tm, 0.9 * Tm
    nu = Tm * (1.25 - 0.5)
    kappa = config.kappa_from_prandtl(9.0, nu, 2.6, Tm)
    gz = config.gravity_from_rayleigh(ratio * 1707.76, L, Td - Tu, kappa, nu, 2.6, Tm)
    nx = 2 * round(2.016 * L / 2)
    p = lb.Params(nx=nx, ny=1, nz=L, tau_nu=1.25, tau_kappa=1.0, G=G0, kappa=kappa, g_z=gz,
                  T_d=Td, T_u=Tu, precision=precision, tile_y=4)
    k = 2 * math.pi / nx
    zc = (np.arange(L) + 0.5) / L
    x = np.arange(nx)
    T = (Td + (Tu - Td) * zc)[:, None, None] + 1e-3 * (Td - Tu) * (
        np.sin(math.pi * zc)[:, None, None] * np.sin(k * x)[None, None, :])
    rho = np.full((L, 1, nx), 2.6)
    return p, rho, np.ascontiguousarray(T), np.exp(-1j * k * x)


def _roll_amplitude(lat, e):
    _, u, _ = lat.moments()
    return float(np.abs((u[2][:, 0, :] * e[None, :]).sum()))


def test_rayleigh_benard_rolls_decay_below_and_convect_above_onset():
    """Measured on this cell (alpha dT = 0.46, far from the Oberbeck-Boussinesq limit): Nu = 1.54
    at 2 x 1708 and 1.67 at 3 x 1708 after 120,000 steps; the onset itself is bracketed by the
    next test."""
    p, rho, T, e = _rolls(0.5, lb.LB_FP32)
    lat = lb.Lattice(p, rho, T)
    lat.step(4000)
    a0 = _roll_amplitude(lat, e)
    lat.step(116000)
    a1 = _roll_amplitude(lat, e)
    nu_below = lat.nusselt()[0]
    lat.close()
    assert a1 < 0.2 * a0 and abs(nu_below - 1.0) < 1e-3, (a0, a1, nu_below)
    nus = {}
    for prec in (lb.LB_FP32, lb.LB_FP64):
        p, rho, T, e = _rolls(2.0, prec)
        lat = lb.Lattice(p, rho, T)
        lat.step(4000)
        a0 = _roll_amplitude(lat, e)
        lat.step(116000)
        a1 = _roll_amplitude(lat, e)
        nus[prec], nu_z, _ = lat.nusselt()
        _, _, pdivu_z = lat.profiles()
        d = lat.diagnostics()
        lat.close()
        assert a1 > 100 * a0 and d["nonfinite"] == 0, (prec, a0, a1)
    assert nus[lb.LB_FP32] > 1.3 and nus[lb.LB_FP64] > 1.3, nus
    assert abs(nus[lb.LB_FP32] - nus[lb.LB_FP64]) < 2e-3 * nus[lb.LB_FP64], nus
    # Eq. (5), the integral constraint of the stationary heat balance Eq. (4):
    # Nu(z) - Nu(0) = -int_0^z <P div u> dz' / (kappa (T_d - T_u)/L). In these compressible rolls
    # Nu(z) varies by 0.27 across the cell; the integral of P div u (trapezoidal, unit spacing)
    # reproduces it to 0.0032 (measured).
    lhs = nu_z - nu_z[0]
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (pdivu_z[1:] + pdivu_z[:-1]))])
    rhs = -cum / (p.kappa * (p.T_d - p.T_u) / p.nz)
    assert np.abs(lhs).max() > 0.1, lhs
    assert np.abs(lhs - rhs).max() < 0.03 * np.abs(lhs).max(), (lhs, rhs)


def test_onset_of_the_rolls_within_five_percent_of_the_classical_critical_rayleigh_number():
    """Linear growth of the roll mode on the L = 64 cell (alpha dT = 0.46) over 1.5 thermal
    diffusion times L^2 / chi (chi = kappa / (rho c_p)): at r = Ra / 1707.76 = 1.00 the mode
    decays, at r = 1.05 it grows. Measured amplitude ratios over this window: 0.54 and 2.4
    (and 0.55 / 2.2 at alpha dT = 0.23, L = 128, not run here); the sign change of the growth
    rate, with r = 0.95 decaying and r = 1.1 growing at both sizes, lies in 1.00 < r < 1.05."""
    ratios = {}
    for r in (1.0, 1.05):
        p, rho, T, e = _rolls(r, lb.LB_FP32)
        chi = p.kappa / (2.6 * config.beta_cp(2.6, config.T_M)[1])
        t_th = p.nz * p.nz / chi
        first = int(0.05 * t_th)
        lat = lb.Lattice(p, rho, T)
        lat.step(first)
        a0 = _roll_amplitude(lat, e)
        lat.step(int(1.5 * t_th) - first)
        a1 = _roll_amplitude(lat, e)
        bad = lat.diagnostics()["nonfinite"]
        lat.close()
        assert bad == 0, r
        ratios[r] = a1 / a0
    assert ratios[1.0] < 0.8 and ratios[1.05] > 1.5, ratios


def test_onset_within_two_percent_at_half_the_temperature_difference():
    """The same roll at L = 128 with T_d/u = (1 +- 0.05) T_m (alpha dT = 0.23), started from the
    relaxed base state: a 32-wide column of the unperturbed cell runs half a thermal time
    (hydrostatic and conductive profiles; the uniform start otherwise launches sound waves that
    swamp the roll's early amplitude), then the full cell starts from its rho(z), T(z) plus the roll.
    The roll's temperature amplitude, projected on sin(pi z / L), after 1.5 thermal times against
    its value at 0.075: measured 0.79 at r = 1.00 and 2.26 at r = 1.02, so 1.00 < r_c < 1.02."""
    L, Tm = 128, config.T_M
    zc = (np.arange(L) + 0.5) / L
    ratios = {}
    for r in (1.0, 1.02):
        Td, Tu = 1.05 * Tm, 0.95 * Tm
        nu = Tm * (1.25 - 0.5)
        kappa = config.kappa_from_prandtl(9.0, nu, 2.6, Tm)
        gz = config.gravity_from_rayleigh(r * 1707.76, L, Td - Tu, kappa, nu, 2.6, Tm)
        chi = kappa / (2.6 * config.beta_cp(2.6, Tm)[1])
        t_th = L * L / chi
        col = lb.Params(nx=32, ny=1, nz=L, tau_nu=1.25, tau_kappa=1.0, G=G0, kappa=kappa, g_z=gz,
                        T_d=Td, T_u=Tu, precision=lb.LB_FP32, tile_y=4)
        Tlin = np.ascontiguousarray(np.broadcast_to((Td + (Tu - Td) * zc)[:, None, None], (L, 1, 32)))
        lat = lb.Lattice(col, np.full((L, 1, 32), 2.6), Tlin)
        lat.step(int(0.5 * t_th))
        rho_c, _, T_c = lat.moments()
        lat.close()
        nx = 2 * round(2.016 * L / 2)
        k = 2 * math.pi / nx
        x = np.arange(nx)
        p = lb.Params(**{**col.__dict__, "nx": nx})
        rho = np.ascontiguousarray(np.broadcast_to(rho_c.mean(axis=(1, 2))[:, None, None], (L, 1, nx)))
        T = T_c.mean(axis=(1, 2))[:, None, None] + 1e-3 * (Td - Tu) * (
            np.sin(math.pi * zc)[:, None, None] * np.sin(k * x)[None, None, :])
        e, sz = np.exp(-1j * k * x), np.sin(math.pi * zc)

        def amp(lat):
            Tn = lat.moments()[2][:, 0, :]
            dT = Tn - Tn.mean(axis=1, keepdims=True)
            return float(np.abs(((dT * e[None, :]).sum(axis=1) * sz).sum()))

        lat = lb.Lattice(p, rho, np.ascontiguousarray(T))
        chunk = int(3.0 * t_th) // 40
        lat.step(chunk)
        a0 = amp(lat)
        lat.step(19 * chunk)
        a1 = amp(lat)
        bad = lat.diagnostics()["nonfinite"]
        lat.close()
        assert bad == 0, r
        ratios[r] = a1 / a0
    assert ratios[1.0] < 0.9 and ratios[1.02] > 1.5, ratios


def _slab_variant(t, psi, forcing, tau, nz=96, steps=30000, kappa=0.24, with_T=False):
    """Flat liquid slab at T = t T_c (isothermal walls), the paper's psi (G of the default cell)
    or the van der Waals psi (a = 5/42, b = 2/21, T_v = T, G = -1); returns (rho_l, rho_g), and
    with with_T also the temperatures (T_l, T_g) at the two sampling planes."""
    T0 = t * TC
    A, B = 5.0 / 42.0, 2.0 / 21.0
    if psi == lb.LB_PSI_EXP:
        rg, rl = eos.coexistence(T0, G0)
        G = G0
    else:
        rg, rl = eos.coexistence_vdw(T0, A, B, T0)
        G = -1.0
    p = lb.Params(nx=4, ny=4, nz=nz, tau_nu=tau, tau_kappa=1.0, G=G, kappa=kappa, g_z=0.0,
                  T_d=T0, T_u=T0, forcing=forcing, psi_kind=psi, vdw_a=A, vdw_b=B, vdw_T=T0)
    z = np.arange(nz) + 0.5
    prof = 0.5 * (np.tanh((z - nz / 4) / 2.5) - np.tanh((z - 3 * nz / 4) / 2.5))
    rho = np.broadcast_to((rg + (rl - rg) * prof)[:, None, None], (nz, 4, 4)).copy()
    r, u, TT = _run(p, rho, np.full_like(rho, T0), steps)
    if with_T:
        return float(r[nz // 2].mean()), float(r[1].mean()), float(TT[nz // 2].mean()), float(TT[1].mean())
    return float(r[nz // 2].mean()), float(r[1].mean())


def test_guo_forcing_removes_the_tau_bias_of_the_coexistence_densities():
    """Paper's psi at T = 0.85 T_c. Guo forcing: rho_l, rho_g at tau_nu = 1, 1.5, 2 agree to
    1e-3 and lie within 0.5 % of the Maxwell construction (measured 2.0729 / 0.49359 vs 2.0772 /
    0.49266). Velocity shift: +1.1 % / +3.8 % at tau_nu = 1 growing to +6.0 % / +21 % at 2."""
    rg, rl = eos.coexistence(0.85 * TC, G0)
    guo = [_slab_variant(0.85, lb.LB_PSI_EXP, lb.LB_FORCE_GUO, tau) for tau in (1.0, 1.5, 2.0)]
    for rl_m, rg_m in guo:
        assert abs(rl_m / guo[0][0] - 1) < 1e-3 and abs(rg_m / guo[0][1] - 1) < 1e-3, guo
        assert abs(rl_m / rl - 1) < 5e-3 and abs(rg_m / rg - 1) < 5e-3, (guo, rl, rg)
    shift = [_slab_variant(0.85, lb.LB_PSI_EXP, lb.LB_FORCE_SHIFT, tau) for tau in (1.0, 2.0)]
    assert shift[0][0] / rl - 1 > 0.005 and shift[1][0] / rl - 1 > 2 * (shift[0][0] / rl - 1), shift
    assert shift[1][1] / rg - 1 > 0.1, shift


def test_vdw_psi_coexistence_follows_the_psi_rule():
    """Van der Waals psi at T = 0.85 T_c with Guo forcing: tau-independent (tau_nu = 1.5, 2) and
    closer to the psi-rule (equal area in ln psi: rho_g 1.0301, rho_l 6.2998) than to Maxwell's
    rule of the same pressure (1.1191, 6.3250); measured 1.0634 / 6.2750."""
    T0 = 0.85 * TC
    A, B = 5.0 / 42.0, 2.0 / 21.0
    res = [_slab_variant(0.85, lb.LB_PSI_VDW, lb.LB_FORCE_GUO, tau) for tau in (1.5, 2.0)]
    assert abs(res[0][0] / res[1][0] - 1) < 1e-3 and abs(res[0][1] / res[1][1] - 1) < 1e-3, res
    rl_m, rg_m = res[1]
    P = lambda r: eos.pressure_vdw(r, T0, A, B, T0)
    psi = lambda r: r * math.sqrt(2.0 * (A - B * T0 / (1 - B * r)))
    dpsi = lambda r: (psi(r + 1e-6) - psi(r - 1e-6)) / 2e-6
    mg, ml = eos.coexistence_vdw(T0, A, B, T0)
    from scipy.optimize import brentq
    lo = brentq(lambda r: eos.dP_drho_vdw(r, T0, A, B, T0), 0.05, 3.5)
    hi = brentq(lambda r: eos.dP_drho_vdw(r, T0, A, B, T0), 3.5, 0.999 / B)
    eg, el = eos.coexistence_psi_rule(P, psi, dpsi, lo, hi, 0.0, [mg, ml])
    assert abs(rg_m / eg - 1) < 0.05 and abs(rl_m / el - 1) < 0.01, (res, eg, el)
    assert abs(rg_m / eg - 1) < abs(rg_m / mg - 1), (rg_m, eg, mg)


def test_clausius_clapeyron_with_guo_forcing_at_four_temperatures():
    """Fig. 1's Clausius-Clapeyron relation on the simulated coexistence curve, with the
    tau-independent Guo forcing (no velocity-shift bias), at T/T_c = 0.80, 0.85, 0.90, 0.95
    (tau_nu = 1.5, kappa = 0.12, 60,000 steps: stable at all four temperatures, measured; at
    tau_nu = 1 the slab at 0.80 T_c breaks down with kappa = 0.24 and the ones at 0.90 and 0.95 T_c
    with kappa = 0.12):
    - each slab's bulk densities lie within 1 % of the Maxwell construction of
      P = rho T + (G/2) e^{-2/rho} (measured within 0.6 %), and its two bulk phases have equal EOS
      pressure at their own temperatures within 0.3 % (mechanical equilibrium; at the nominal T
      the liquid's P, a difference of terms ~6 times larger than itself, is off by a 1e-3
      temperature nonuniformity left by the slow conduction at kappa = 0.12);
    - P_sat(T) from the bulk EOS; dP/dT from the cubic through the four (T, P_sat) points (on the
      Maxwell values this derivative is within 2e-4 of the exact one) equals the latent-heat
      ratio Delta s / Delta v = ln(rho_l/rho_g) / (1/rho_g - 1/rho_l) of the simulated densities
      within 1 % at every temperature, and the oracle's Maxwell-construction Delta s / Delta v
      within 1 %."""
    ts = np.array([0.80, 0.85, 0.90, 0.95])
    runs = [_slab_variant(t, lb.LB_PSI_EXP, lb.LB_FORCE_GUO, 1.5, kappa=0.12, with_T=True, steps=60000)
            for t in ts]
    sim = [(r[0], r[1]) for r in runs]
    Psat = []
    for t, (rl_m, rg_m, Tl, Tg) in zip(ts, runs):
        rg, rl = eos.coexistence(t * TC, G0)
        Pl, Pg = eos.pressure(rl_m, Tl, G0), eos.pressure(rg_m, Tg, G0)
        print(f"T/Tc={t}: rho_l {rl_m:.5f} ({100 * (rl_m / rl - 1):+.3f} %), rho_g {rg_m:.5f} "
              f"({100 * (rg_m / rg - 1):+.3f} %), T_l/T {Tl / (t * TC):.6f}, T_g/T {Tg / (t * TC):.6f}, "
              f"P_l {Pl:.6f} P_g {Pg:.6f}")
        assert abs(rl_m / rl - 1) < 1e-2 and abs(rg_m / rg - 1) < 1e-2
        assert abs(Pl / Pg - 1) < 3e-3
        Psat.append(eos.pressure(rg_m, t * TC, G0))   # the vapour's: ~5 times less sensitive to T
    T = ts * TC
    c = np.polyfit(T, np.array(Psat), 3)
    dPdT = np.polyval(np.polyder(c), T)
    for k, t in enumerate(ts):
        rl_m, rg_m = sim[k]
        ds_dv = math.log(rl_m / rg_m) / (1 / rg_m - 1 / rl_m)
        rg, rl = eos.coexistence(t * TC, G0)
        ds_dv_max = math.log(rl / rg) / (1 / rg - 1 / rl)
        print(f"T/Tc={t}: dP/dT {dPdT[k]:.5f}, Delta s/Delta v {ds_dv:.5f} ({100 * (dPdT[k] / ds_dv - 1):+.3f} %), "
              f"Maxwell {ds_dv_max:.5f} ({100 * (dPdT[k] / ds_dv_max - 1):+.3f} %)")
        assert abs(dPdT[k] / ds_dv - 1) < 0.01
        assert abs(dPdT[k] / ds_dv_max - 1) < 0.01


def test_laplace_law_up_to_radius_30():
    """Static liquid droplets of radius 16 ... 30 in vapour at T = 0.9 T_c in a 128^3 box (Guo
    forcing, tau_nu = 1.5, kappa = 0.12, FP32; with kappa = 0.24 the 128^3 droplets break down
    within 2000 steps, measured): the pressure jump from the bulk EOS between the droplet centre
    and the far vapour is linear in the inverse equimolar radius, Delta P = 2 sigma / R, with
    R^2 > 0.999 and an intercept below 5 % of the largest jump. (A droplet of R = 12, about four
    interface widths, sits visibly off the line: with it the data need a 1/R^2 term, the
    finite-interface correction, measured R^2 0.99878 linear against 0.999996 with that term.)"""
    T0 = 0.9 * TC
    rg, rl = eos.coexistence(T0, G0)
    n = 128
    p = lb.Params(nx=n, ny=n, nz=n, tau_nu=1.5, tau_kappa=1.0, G=G0, kappa=0.12, g_z=0.0,
                  T_d=T0, T_u=T0, forcing=lb.LB_FORCE_GUO)
    c = (np.arange(n) + 0.5 - n / 2)
    r3 = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    inv_R, dP = [], []
    for R in (16.0, 20.0, 25.0, 30.0):
        rho = rg + (rl - rg) * 0.5 * (1 - np.tanh((r3 - R) / 2.5))
        T = np.full_like(rho, T0)
        r, u, TT = _run(p, rho, T, 15000, precision=lb.LB_FP32)
        P = eos.pressure(r, TT, G0)
        m = n // 2
        P_in = P[m - 2:m + 2, m - 2:m + 2, m - 2:m + 2].mean()
        rho_in = r[m - 2:m + 2, m - 2:m + 2, m - 2:m + 2].mean()
        # far vapour: the box corners (farthest from the droplet)
        far = r3 > 0.5 * n * 0.95 * math.sqrt(3)
        P_out = P[far].mean()
        rho_out = r[far].mean()
        vol = float(np.sum(r - rho_out) / (rho_in - rho_out))
        R_eq = (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
        assert R_eq > 0.8 * R, f"droplet of initial radius {R} shrank to {R_eq}"
        inv_R.append(1.0 / R_eq)
        dP.append(P_in - P_out)
        print(f"R0={R}: R={R_eq:.3f}, dP={P_in - P_out:.6e}, max|u|={np.abs(np.stack(u)).max():.2e}")
    A = np.vstack([inv_R, np.ones(len(inv_R))]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, np.array(dP), rcond=None)
    pred = A @ np.array([slope, icpt])
    r2 = 1 - np.sum((np.array(dP) - pred) ** 2) / np.sum((np.array(dP) - np.mean(dP)) ** 2)
    print(f"Laplace: 2 sigma = {slope:.5e}, intercept {icpt:.2e}, R^2 = {r2:.6f}")
    assert slope > 0 and r2 > 0.999 and abs(icpt) < 0.05 * max(dP)
