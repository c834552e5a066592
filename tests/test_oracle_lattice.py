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


def _z_profile(nz, nx=3, ny=2):
    """A density that varies only in z, steep next to both walls: rho(z) = 1.3 + 0.4 tanh(z - 1)
    - 0.3 exp(-(nz - 1 - z))."""
    z = torch.arange(nz, dtype=DT)
    r = 1.3 + 0.4 * torch.tanh(z - 1.0) - 0.3 * torch.exp(-(nz - 1 - z))
    return r[:, None, None].expand(nz, ny, nx).clone()


@pytest.mark.parametrize("nz", [1, 2, 3, 7])
def test_wall_force_of_a_z_profile_is_the_mirrored_closed_form(nz):
    """Eq. (9) for a density that depends on z only: the 6 links with c_z = +-1 (one axis link
    of weight 1/6, four diagonals of weight 1/12) give F_z(z) = -(G/2) psi(z) [psi(z+1) - psi(z-1)]
    and F_x = F_y = 0. With halfway walls and the neutral-wetting ghosts the plane beyond a wall
    carries the density of its mirror image: psi(-1) = psi(rho(0)), psi(nz) = psi(rho(nz-1)),
    so F_z(0) = -(G/2) psi(0) [psi(1) - psi(0)]. A ghost mirrored about the node (psi(-1) = psi(1),
    no force on plane 0) or psi = 0 beyond the wall fails this."""
    p = lbm.Params(3, 2, nz, 1.0, 1.0, G=-2.7, kappa=0.1)
    rho = _z_profile(nz)
    F = lbm.force(rho, p)
    ps = torch.exp(-1.0 / rho[:, 0, 0])
    ext = [ps[lbm.mirror_z(k, nz)] for k in range(-1, nz + 1)]   # planes -1 .. nz
    for z in range(nz):
        want = -(p.G / 2.0) * ps[z] * (ext[z + 2] - ext[z])
        assert torch.allclose(F[2, z], want.expand_as(F[2, z]), rtol=1e-14, atol=1e-15), z
    assert float(F[0].abs().max()) < 1e-15 and float(F[1].abs().max()) < 1e-15
    if nz >= 3:
        # the explicit first-plane form: the bottom ghost is plane 0 itself
        want0 = -(p.G / 2.0) * ps[0] * (ps[1] - ps[0])
        assert abs(float(F[2, 0, 0, 0]) - float(want0)) < 1e-15
        assert abs(float(F[2, 0, 0, 0]) - float(-(p.G / 2.0) * ps[0] * (ps[1] - ps[1]))) > 1e-3


@pytest.mark.parametrize("nz", [1, 2, 5])
def test_wall_ghosts_are_the_even_and_odd_extensions(nz):
    """Across a halfway wall the force of Eq. (9) sees the even extension of rho and the divergence
    sees the odd extension of u_z: on a 3-D random field, the wall-bounded force and divergence
    equal those of the fully periodic cell of height 2 nz that holds the field and its mirror
    image (rho(2nz-1-z) = rho(z); u_z(2nz-1-z) = -u_z(z), u_x and u_y likewise reversed, as the
    ghost rule u -> -u states)."""
    g = torch.Generator().manual_seed(7)
    nx, ny = 5, 4
    rho = 1.2 + 0.5 * torch.rand((nz, ny, nx), generator=g, dtype=DT)
    u = 0.02 * (torch.rand((3, nz, ny, nx), generator=g, dtype=DT) - 0.5)
    p = lbm.Params(nx, ny, nz, 1.0, 1.0, G=-2.7, kappa=0.1)
    q = lbm.Params(nx, ny, 2 * nz, 1.0, 1.0, G=-2.7, kappa=0.1, periodic_z=True)
    rho_ext = torch.cat([rho, torch.flip(rho, dims=(0,))])
    u_ext = torch.cat([u, -torch.flip(u, dims=(1,))], dim=1)
    F = lbm.force(rho, p)
    F_ext = lbm.force(rho_ext, q)
    assert torch.allclose(F, F_ext[:, :nz], rtol=0, atol=1e-15)
    D = lbm.divergence(u, p)
    D_ext = lbm.divergence(u_ext, q)
    assert torch.allclose(D, D_ext[:nz], rtol=0, atol=1e-16)
