"""Pins of the oracle's lattice, equilibria and boundary streaming against exact algebra."""
import itertools
import math

import numpy as np
import pytest
import torch

from oracle import lbm

DT = torch.float64


def test_d3q19_weights_and_isotropy():
    """Sum w = 1, odd moments vanish, sum w c_a c_b = d_ab/3, 4th moment = (dd+dd+dd)/9."""
    w = np.array(lbm.W)
    c = np.array(lbm.C, dtype=float)
    assert len(set(lbm.C)) == 19
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("l,la,lb->ab", w, c, c), np.eye(3) / 3, atol=1e-16)
    m4 = np.einsum("l,la,lb,lc,ld->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-16)
    for l, o in enumerate(lbm.OPP):
        assert tuple(-x for x in lbm.C[l]) == lbm.C[o]


def test_force_weights_normalisation_and_isotropy():
    """Eq. (9) weights: sum W c_a c_b = d_ab (so F -> -G psi grad psi) and isotropic 4th moment."""
    W = np.array([0.0] + [lbm.force_weight(l) for l in range(1, 19)])
    c = np.array(lbm.C, dtype=float)
    assert np.allclose(np.einsum("l,la,lb->ab", W, c, c), np.eye(3), atol=1e-15)
    m4 = np.einsum("l,la,lb,lc,ld->abcd", W, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 3
    assert np.allclose(m4, iso, atol=1e-15)


def _rand(shape, lo, hi, seed):
    g = torch.Generator().manual_seed(seed)
    return lo + (hi - lo) * torch.rand(shape, generator=g, dtype=DT)


def test_f_equilibrium_moments():
    """sum f^eq = rho, sum c f^eq = rho v, sum c c f^eq = rho T I + rho v v (text after Eq. (9))."""
    sh = (3, 4, 5)
    rho, T = _rand(sh, 0.4, 2.5, 1), _rand(sh, 0.25, 0.4, 2)
    v = torch.stack([_rand(sh, -0.1, 0.1, s) for s in (3, 4, 5)])
    feq = lbm.equilibrium_f(rho, v, T)
    c = torch.tensor(lbm.C, dtype=DT)
    assert torch.allclose(feq.sum(0), rho, rtol=1e-14, atol=0)
    assert torch.allclose(torch.einsum("la,l...->a...", c, feq), rho * v, rtol=0, atol=1e-15)
    P = torch.einsum("la,lb,l...->ab...", c, c, feq)
    I = torch.eye(3, dtype=DT)[:, :, None, None, None]
    expect = rho * T * I + rho * torch.einsum("a...,b...->ab...", v, v)
    assert torch.allclose(P, expect, rtol=0, atol=1e-14)


def test_g_equilibrium_moments():
    """sum g^eq = rho T, sum c g^eq = rho T u, sum c c g^eq = lam T I + rho T u u."""
    sh = (2, 3, 4)
    rho, T = _rand(sh, 0.4, 2.5, 6), _rand(sh, 0.25, 0.4, 7)
    u = torch.stack([_rand(sh, -0.1, 0.1, s) for s in (8, 9, 10)])
    lam = 0.17
    geq = lbm.equilibrium_g(rho, T, u, lam)
    c = torch.tensor(lbm.C, dtype=DT)
    assert torch.allclose(geq.sum(0), rho * T, rtol=1e-14, atol=0)
    assert torch.allclose(torch.einsum("la,l...->a...", c, geq), rho * T * u, rtol=0, atol=1e-15)
    P = torch.einsum("la,lb,l...->ab...", c, c, geq)
    I = torch.eye(3, dtype=DT)[:, :, None, None, None]
    expect = lam * T * I + rho * T * torch.einsum("a...,b...->ab...", u, u)
    assert torch.allclose(P, expect, rtol=0, atol=1e-14)


def test_streaming_moves_each_population_by_its_velocity():
    """Pull streaming of a single marked node: population l lands at x + c_l (periodic x, y);
    at a wall it is reflected into opp(l) at the same node (halfway bounce-back)."""
    p = lbm.Params(5, 4, 6, 1.0, 1.0, 0.0, 0.1, T_d=0.3, T_u=0.3)
    for (x, y, z) in [(2, 1, 3), (0, 0, 0), (4, 3, 5)]:
        fstar = torch.zeros((19, 6, 4, 5), dtype=DT)
        for l in range(19):
            fstar[l, z, y, x] = l + 1.0
        rho_wall = torch.zeros((6, 4, 5), dtype=DT)
        f, g = lbm.stream(fstar, torch.zeros_like(fstar), rho_wall, p)
        for l in range(19):
            cx, cy, cz = lbm.C[l]
            zz = z + cz
            if 0 <= zz < 6:
                assert f[l, zz, (y + cy) % 4, (x + cx) % 5] == l + 1.0
            else:
                assert f[lbm.OPP[l], z, y, x] == l + 1.0
        assert f.sum() == fstar.sum()          # no population lost or duplicated


def test_thermal_wall_rule_returns_wall_equilibrium():
    """Anti-bounce-back: if g* at the wall node is the rest equilibrium at T_w, the populations
    arriving from the wall equal that equilibrium (even part), so a wall in equilibrium is steady."""
    p = lbm.Params(3, 3, 4, 1.0, 0.8, 0.0, 0.05, T_d=0.37, T_u=0.29)
    rho = torch.full((4, 3, 3), 1.3, dtype=DT)
    T = torch.tensor([p.T_d, 0.33, 0.31, p.T_u], dtype=DT)[:, None, None].expand(4, 3, 3).clone()
    zero = torch.zeros((3, 4, 3, 3), dtype=DT)
    geq = lbm.equilibrium_g(rho, T, zero, p.lam)
    f, g = lbm.stream(torch.zeros_like(geq), geq, rho, p)
    for l in range(19):
        if lbm.C[l][2] > 0:
            assert torch.allclose(g[l, 0], geq[l, 0], rtol=1e-15, atol=1e-17)
        if lbm.C[l][2] < 0:
            assert torch.allclose(g[l, -1], geq[l, -1], rtol=1e-15, atol=1e-17)


def test_mirror_index():
    assert [lbm.mirror_z(k, 5) for k in (-2, -1, 0, 4, 5, 6)] == [1, 0, 0, 4, 4, 3]
    assert [lbm.mirror_z(k, 1) for k in (-2, -1, 1, 2)] == [0, 0, 0, 0]
