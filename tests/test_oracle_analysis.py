"""Pins of the oracle's statistics against closed forms: structure functions and flatness of
sinusoidal fields (S2 = A^2 (1 - cos kr), flatness 3/2) and of Gaussian noise (flatness 3), the
histogram's bin arithmetic and totals, and the profiles of a state at rest."""
import math

import numpy as np
import pytest
import torch

from oracle import analysis, lbm

DT = torch.float64


def test_structure_functions_of_a_sinusoid():
    L, A = 32, 0.3
    k = 2 * math.pi / L
    x = np.arange(L)
    q = A * (np.sin(k * x)[None, None, :] + np.sin(k * x)[None, :, None]) * np.ones((3, L, L))
    out = analysis.structure_functions(q, q, 10, 0, 3)
    r = np.arange(1, 11)
    assert np.allclose(out["S2_uz"], A ** 2 * (1 - np.cos(k * r)), rtol=1e-12, atol=0)
    assert np.allclose(out["S4_uz"] / out["S2_uz"] ** 2, 1.5, rtol=1e-10, atol=0)
    assert np.allclose(out["S2_T"], out["S2_uz"], rtol=0, atol=0)


def test_flatness_of_gaussian_noise_is_three():
    rng = np.random.default_rng(1)
    q = rng.standard_normal((4, 64, 64))
    out = analysis.structure_functions(q, q, 5, 0, 4)
    assert np.allclose(out["S2_uz"], 2.0, rtol=0.03)
    assert np.allclose(out["S4_uz"] / out["S2_uz"] ** 2, 3.0, rtol=0.05)


def test_histogram_bins_and_totals():
    T = np.array([0.30, 0.31, 0.3199, 0.32, 0.40, 0.10])[:, None, None] * np.ones((6, 1, 2))
    rho = np.array([1.0, 1.5, 1.99, 2.0, 1.0, 1.0])[:, None, None] * np.ones((6, 1, 2))
    c = analysis.histogram_T_rho(rho, T, 0, 6, 2, (0.30, 0.34), 2, (1.0, 2.0))
    # T bins [0.30,0.32) [0.32,0.34); rho bins [1.0,1.5) [1.5,2.0); v == hi and out-of-range excluded
    assert c.tolist() == [[2, 4], [0, 0]]
    assert analysis.histogram_T_rho(rho, T, 1, 3, 2, (0.30, 0.34), 2, (1.0, 2.0)).sum() == 4


def test_profiles_of_a_state_at_rest():
    p = lbm.Params(4, 3, 5, 1.0, 1.0, 0.0, 0.1, T_d=0.36, T_u=0.30)
    z = (torch.arange(5, dtype=DT) + 0.5) / 5
    T = (0.36 - 0.06 * z)[:, None, None].expand(5, 3, 4).clone()
    rho = (1.0 / 3.0) / T
    f, g = lbm.init_state(rho, T, p)
    r_z, T_z, PD_z = analysis.profiles(f, g, p)
    assert torch.allclose(T_z, T[:, 0, 0], rtol=1e-14, atol=0)
    assert torch.allclose(r_z, rho[:, 0, 0], rtol=1e-14, atol=0)
    assert PD_z.abs().max() < 1e-15


def test_heat_flux_pdf_of_a_state_at_rest_and_of_a_shear():
    """At rest q = rho U u_z = 0 everywhere (one bin, zero mean and variance); for a state with
    u_z = A sin(2 pi x / L) at uniform rho, T the mean is 0, the variance (rho U A)^2 / 2, and the
    counts follow the arcsine law of the sampled sinusoid."""
    import torch
    from oracle import analysis, lbm
    L = 16
    p = lbm.Params(L, 2, 3, 1.0, 1.0, -2.7, 0.05, T_d=1 / 3, T_u=1 / 3)
    rho = torch.full((3, 2, L), 1.7, dtype=torch.float64)
    T = torch.full_like(rho, 1 / 3)
    f, g = lbm.init_state(rho, T, p)
    counts, (n, mean, var) = analysis.heat_flux_pdf(f, g, p, 0, 3, 4, (-1.0, 1.0))
    assert n == 3 * 2 * L and mean == 0.0 and var == 0.0 and counts[2] == n
    A = 1e-3
    u = torch.zeros((3,) + tuple(rho.shape), dtype=torch.float64)
    u[2] = A * torch.sin(2 * math.pi * torch.arange(L, dtype=torch.float64) / L)[None, None, :]
    # a state whose physical velocity is u: no force at uniform rho (F = rho g_z = 0)
    f = lbm.equilibrium_f(rho, u, T)
    g = lbm.equilibrium_g(rho, T, u, p.lam)
    U = float(lbm.internal_energy(rho, T, p)[0, 0, 0])
    qmax = 1.7 * U * A
    counts, (n, mean, var) = analysis.heat_flux_pdf(f, g, p, 0, 3, 8, (-qmax * 1.0001, qmax * 1.0001))
    assert abs(mean) < 1e-18 and abs(var / (0.5 * qmax ** 2) - 1) < 1e-12
    assert counts.sum() == n and counts[0] == counts[-1] and counts[0] > counts[3]
