"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle's tests.

This module holds no arithmetic of the lattice Boltzmann method: only the counter-based
random generator (SplitMix64, Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014, with Vigna's published finaliser constants) and the initial-field
recipes of the synthetic workloads. Fields are numpy float64 arrays shaped [nz, ny, nx]
(x fastest), i.e. node index idx = x + nx*(y + ny*z).
"""
from __future__ import annotations

import numpy as np

SEED = 20111105

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(n: int, seed: int = SEED, offset: int = 0) -> np.ndarray:
    """The n outputs number offset+1 .. offset+n of SplitMix64 seeded with `seed`, as uint64."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(n: int, seed: int = SEED, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [-1, 1): the top 53 bits of each SplitMix64 output scaled to [0,1)."""
    u = (splitmix64(n, seed, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def noise_field(nx: int, ny: int, nz: int, seed: int = SEED, offset: int = 0) -> np.ndarray:
    """Uniform [-1,1) noise filled in node-index order, shaped [nz, ny, nx]."""
    return uniform_pm1(nx * ny * nz, seed, offset).reshape(nz, ny, nx)


def linear_T(nx: int, ny: int, nz: int, T_d: float, T_u: float) -> np.ndarray:
    """Conduction profile between halfway walls at z=-1/2 (T_d) and z=nz-1/2 (T_u)."""
    z = (np.arange(nz, dtype=np.float64) + 0.5) / nz
    T = T_d + (T_u - T_d) * z
    return np.broadcast_to(T[:, None, None], (nz, ny, nx)).copy()


def boiling_fields(nx, ny, nz, rho_mean, T_d, T_u, amp=0.01, seed=SEED):
    """Density rho_mean*(1 + amp*xi) with seeded xi, temperature linear in z."""
    rho = rho_mean * (1.0 + amp * noise_field(nx, ny, nz, seed))
    return rho, linear_T(nx, ny, nz, T_d, T_u)


def single_phase_fields(nx, ny, nz, rho_mean, T_d, T_u, amp=0.01, seed=SEED):
    """Uniform density, temperature linear in z with seeded relative noise amp on T."""
    rho = np.full((nz, ny, nx), rho_mean, dtype=np.float64)
    T = linear_T(nx, ny, nz, T_d, T_u) * (1.0 + amp * noise_field(nx, ny, nz, seed))
    return rho, T


def noise_block(nx, ny, nz, x0, y0, z0, sx, sy, sz, seed=SEED) -> np.ndarray:
    """The [z0, z0+sz) x [y0, y0+sy) x [x0, x0+sx) block of noise_field(nx, ny, nz, seed), drawn
    row by row from the generator's counter (no full field is formed), shaped [sz, sy, sx]."""
    out = np.empty((sz, sy, sx), dtype=np.float64)
    for k in range(sz):
        for j in range(sy):
            out[k, j] = uniform_pm1(sx, seed, offset=x0 + nx * ((y0 + j) + ny * (z0 + k)))
    return out


def boiling_block(nx, ny, nz, x0, y0, z0, sx, sy, sz, rho_mean, T_d, T_u, amp=0.01, seed=SEED):
    """The same block of boiling_fields(nx, ny, nz, ...): density and temperature values equal to
    those of the full cell at the block's nodes."""
    rho = rho_mean * (1.0 + amp * noise_block(nx, ny, nz, x0, y0, z0, sx, sy, sz, seed))
    T = linear_T(1, 1, nz, T_d, T_u)[z0:z0 + sz, 0, 0]
    return rho, np.broadcast_to(T[:, None, None], (sz, sy, sx)).copy()
