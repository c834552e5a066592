"""Plain FP64 CPU oracle of the thermal pseudopotential D3Q19 lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the benchmark's CPU-baseline leg
may import this module. The product path never calls it and shares no code with it.

Biferale, Perlekar, Sbragaglia, Toschi, "Convection in multiphase flows using Lattice
Boltzmann methods" (arXiv:1111.0905). Equations are cited by their number in the paper:
(1) Navier-Stokes with gravity [ns], (2) internal energy [internal], (3) temperature
equations [eq], (4) layer heat balance [heat2], (5) integral constraint [flux],
(6)-(7) the two BGK lattice equations [LBEQ, LBEQ2], (8) hydrodynamic moments [HYDRO],
(9) pseudopotential force [FORCE]. The "Algorithm" paragraph is the only description of
the scheme; where it is silent the readings below are used (the same ones the CUDA path
implements, written independently).

Readings (the paper leaves these open):
  * 19 velocities l = 0..18 including rest; the force sum of Eq. (9) runs over l = 1..18.
  * Eq. (9) weights W(1) = 1/6, W(2) = 1/12 (= w_l / c_s^2); then the bulk pressure is
    P = rho*T + (G/2) exp(-2/rho), so the paper's calligraphic G equals G/2 here.
  * The temperature from g enters f^eq through its second moment rho*T*I + rho*v*v.
  * g^eq carries rho*T as zeroth moment and lambda*T*I (+rho*T*u*u) as second moment with
    lambda = kappa / (c_v (tau_kappa - 1/2)): conduction -kappa grad T with constant kappa.
  * Equilibrium velocity u' = (j + tau_nu F)/rho (velocity shift); physical velocity
    u = (j + F/2)/rho, used in g^eq, in the divergence, in Nu and in exported fields.
  * Counter term: S = -rho*T*div(u)/c_v added as w_l*S to the g collision; div by
    6-point central differences of the physical u.
  * Halfway walls at z=-1/2 and z=nz-1/2, periodic x and y. Across a wall rho (so psi) is
    mirrored, u -> -u of the mirror node, T -> 2 T_wall - T(mirror).
  * Walls: halfway bounce-back for f; anti-bounce-back for g with the even part of g^eq at
    the wall temperature and the density of the wall node at the colliding step.
  * Gravity: full-rho body force rho*g_z*z_hat added to F.

Variants for comparison (Params.forcing, Params.psi_kind; the paper's scheme is the default):
  * Guo forcing: f^eq at the physical velocity u plus (1 - 1/(2 tau_nu)) S_l with
    S_l = w_l [3 (c_l - u).F + 9 (c_l.u)(c_l.F)] (Guo, Zheng, Shi, Phys. Rev. E 65, 046308).
  * Van der Waals-type pseudopotential psi = sqrt(2 rho^2 (b T_v/(1 - b rho) - a)/G): the bulk
    pressure is rho T + the non-ideal van der Waals pressure at the temperature T_v.

State convention: the state at time n is the pre-collision (post-streaming) pair (f, g),
each a tensor [19, nz, ny, nx] (x fastest). All arithmetic is float64, sums over l in
ascending order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

DT = torch.float64

# D3Q19 velocity set (Algorithm paragraph). Rest, 6 axis, 12 face diagonals in +/- pairs.
C = (
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
)
Q = 19
# Lattice weights: rest 1/3, axis 1/18, diagonal 1/36 (sound speed squared 1/3).
W = tuple([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)
# Opposite direction of each l.
OPP = tuple(C.index((-c[0], -c[1], -c[2])) for c in C)
# |c_l|^2.
C2 = tuple(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] for c in C)


@dataclass
class Params:
    nx: int
    ny: int
    nz: int
    tau_nu: float          # relaxation time of f, Eq. (6)
    tau_kappa: float       # relaxation time of g, Eq. (7)
    G: float               # pseudopotential coupling of Eq. (9) (attractive < 0)
    kappa: float           # thermal conductivity, Eqs. (2)-(3)
    c_v: float = 1.0       # specific heat at constant volume, Eq. (3)
    g_z: float = 0.0       # signed gravity along z, Eq. (1)
    T_d: float = 1.0 / 3.0  # bottom wall temperature
    T_u: float = 1.0 / 3.0  # top wall temperature
    periodic_z: bool = False  # test-only: replace the walls by periodic z
    # Variants (comparisons, not the paper's scheme): forcing "shift" (the paper's velocity
    # shift) or "guo" (tau-independent source term); pseudopotential "exp" (the paper's
    # exp(-1/rho)) or "vdw" (van der Waals attraction and excluded volume at temperature vdw_T).
    forcing: str = "shift"
    psi_kind: str = "exp"
    vdw_a: float = 5.0 / 42.0
    vdw_b: float = 2.0 / 21.0
    vdw_T: float = 1.0 / 3.0

    @property
    def lam(self) -> float:
        """lambda = kappa / (c_v (tau_kappa - 1/2)), second-moment coefficient of g^eq."""
        return self.kappa / (self.c_v * (self.tau_kappa - 0.5))


# ---------------------------------------------------------------------------------------
# Equilibria (Algorithm paragraph; second moments constrained as stated after Eq. (9)).
# ---------------------------------------------------------------------------------------

def equilibrium_f(rho, v, T):
    """f^eq_l = w_l rho [1 + 3 c.v + 4.5 (c.v)^2 - 1.5 v.v + 4.5 (T - 1/3)(|c|^2 - 1)].

    Moments: sum = rho, sum c = rho v, sum c c = rho T I + rho v v.
    """
    vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2]
    out = []
    for l in range(Q):
        cv = C[l][0] * v[0] + C[l][1] * v[1] + C[l][2] * v[2]
        out.append(W[l] * rho * (1.0 + 3.0 * cv + 4.5 * cv * cv - 1.5 * vv
                                 + 4.5 * (T - 1.0 / 3.0) * (C2[l] - 1)))
    return torch.stack(out)


def equilibrium_g(rho, T, u, lam):
    """g^eq_l = w_l [rho T (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u) + 4.5 (lam T - rho T/3)(|c|^2-1)].

    Moments: sum = rho T, sum c = rho T u, sum c c = lam T I + rho T u u.
    """
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    E = rho * T
    out = []
    for l in range(Q):
        cu = C[l][0] * u[0] + C[l][1] * u[1] + C[l][2] * u[2]
        out.append(W[l] * (E * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)
                           + 4.5 * (lam * T - E / 3.0) * (C2[l] - 1)))
    return torch.stack(out)


# ---------------------------------------------------------------------------------------
# Moments, Eq. (8).
# ---------------------------------------------------------------------------------------

def density_momentum(f):
    """rho = sum_l f_l, j = sum_l c_l f_l (ascending l)."""
    rho = f[0].clone()
    for l in range(1, Q):
        rho = rho + f[l]
    j = []
    for a in range(3):
        s = torch.zeros_like(rho)
        for l in range(Q):
            if C[l][a] != 0:
                s = s + C[l][a] * f[l]
        j.append(s)
    return rho, torch.stack(j)


def energy(g):
    """rho T = sum_l g_l (ascending l)."""
    E = g[0].clone()
    for l in range(1, Q):
        E = E + g[l]
    return E


# ---------------------------------------------------------------------------------------
# Neighbour access with the boundary rules: periodic x, y; mirrored ghosts across z walls.
# ---------------------------------------------------------------------------------------

def mirror_z(k: int, nz: int) -> int:
    """Plane index of the reflection of plane k across the halfway walls (repeated)."""
    m = k % (2 * nz)
    return m if m < nz else 2 * nz - 1 - m


def shifted(field, dx, dy, dz, p: Params, z_sign: float = 1.0):
    """field(x+dx, y+dy, z+dz) for a [nz, ny, nx] field.

    Periodic in x, y. Across a z wall the value of the mirrored plane is used, multiplied
    by z_sign (+1 for rho/psi, -1 for u). With p.periodic_z the z direction is periodic.
    """
    out = torch.roll(field, shifts=(-dy, -dx), dims=(1, 2))
    if dz == 0:
        return out
    nz = p.nz
    if p.periodic_z:
        return torch.roll(out, shifts=-dz, dims=0)
    planes = []
    for z in range(nz):
        k = z + dz
        if 0 <= k < nz:
            planes.append(out[k])
        else:
            planes.append(z_sign * out[mirror_z(k, nz)])
    return torch.stack(planes)


# ---------------------------------------------------------------------------------------
# Pseudopotential and force, Eq. (9) plus gravity of Eq. (1).
# ---------------------------------------------------------------------------------------

def psi(rho):
    """psi(rho) = exp(-1/rho) (Algorithm paragraph, thermodynamic consistency)."""
    return torch.exp(-1.0 / rho)


def force_weight(l: int) -> float:
    """W(|c|^2): 1/6 for |c|^2 = 1, 1/12 for |c|^2 = 2 (w_l / c_s^2)."""
    return {1: 1.0 / 6.0, 2: 1.0 / 12.0}[C2[l]]


def psi_vdw(rho, p: Params):
    """Pseudopotential whose bulk pressure rho T + (G/2) psi^2 has the non-ideal part of the van
    der Waals pressure at temperature T_v, rho T_v/(1 - b rho) - a rho^2 - rho T_v:
    psi = sqrt(2 rho^2 (b T_v/(1 - b rho) - a) / G) (G < 0; real for b T_v < a (1 - b rho))."""
    return torch.sqrt(2.0 * rho * rho * (p.vdw_b * p.vdw_T / (1.0 - p.vdw_b * rho) - p.vdw_a) / p.G)


def psi_of(rho, p: Params):
    """The pseudopotential of the run: exp(-1/rho) (the paper) or the van der Waals variant."""
    if p.psi_kind == "vdw":
        return psi_vdw(rho, p)
    return psi(rho)


def force(rho, p: Params):
    """F = -G psi(x) sum_{l=1..18} W_l c_l psi(x + c_l) + rho g_z z_hat."""
    ps = psi_of(rho, p)
    acc = [torch.zeros_like(rho) for _ in range(3)]
    for l in range(1, Q):
        nb = shifted(ps, C[l][0], C[l][1], C[l][2], p)
        for a in range(3):
            if C[l][a] != 0:
                acc[a] = acc[a] + (force_weight(l) * C[l][a]) * nb
    F = [-p.G * ps * acc[a] for a in range(3)]
    F[2] = F[2] + rho * p.g_z
    return torch.stack(F)


def divergence(u, p: Params):
    """div u = sum_a [u_a(x+e_a) - u_a(x-e_a)]/2; across walls u -> -u(mirror)."""
    d = torch.zeros_like(u[0])
    e = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
    for a in range(3):
        up = shifted(u[a], e[a][0], e[a][1], e[a][2], p, z_sign=-1.0)
        um = shifted(u[a], -e[a][0], -e[a][1], -e[a][2], p, z_sign=-1.0)
        d = d + 0.5 * (up - um)
    return d


# ---------------------------------------------------------------------------------------
# Macroscopic fields of a state.
# ---------------------------------------------------------------------------------------

def macroscopic(f, g, p: Params):
    """rho, j, T, F, equilibrium velocity u', physical velocity u of the state (f, g)."""
    rho, j = density_momentum(f)
    T = energy(g) / rho
    F = force(rho, p)
    u = (j + 0.5 * F) / rho
    # velocity shift (the paper): f^eq at u' = (j + tau F)/rho; Guo forcing: f^eq at u
    u_eq = u if p.forcing == "guo" else (j + p.tau_nu * F) / rho
    return rho, j, T, F, u_eq, u


# ---------------------------------------------------------------------------------------
# One time step: collision (right-hand sides of Eqs. (6)-(7)) then streaming (left-hand
# sides) with the wall rules.
# ---------------------------------------------------------------------------------------

def guo_source(u, F):
    """S_l = w_l [3 (c_l - u).F + 9 (c_l.u)(c_l.F)] (Guo, Zheng, Shi 2002, with c_s^2 = 1/3).

    Moments: sum = 0, sum c = F, sum c c = u F + F u.
    """
    uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2]
    out = []
    for l in range(Q):
        cu = C[l][0] * u[0] + C[l][1] * u[1] + C[l][2] * u[2]
        cF = C[l][0] * F[0] + C[l][1] * F[1] + C[l][2] * F[2]
        out.append(W[l] * (3.0 * (cF - uF) + 9.0 * cu * cF))
    return torch.stack(out)


def collide(f, g, p: Params):
    """Post-collision f*, g* and the density used by the thermal wall rule."""
    rho, j, T, F, u_eq, u = macroscopic(f, g, p)
    feq = equilibrium_f(rho, u_eq, T)
    fstar = f - (f - feq) / p.tau_nu
    if p.forcing == "guo":
        fstar = fstar + (1.0 - 0.5 / p.tau_nu) * guo_source(u, F)
    D = divergence(u, p)
    S = -rho * T * D / p.c_v
    geq = equilibrium_g(rho, T, u, p.lam)
    gstar = g - (g - geq) / p.tau_kappa
    gstar = gstar + torch.stack([W[l] * S for l in range(Q)])
    return fstar, gstar, rho


def wall_g_even(l: int, rho, T_w: float, lam: float):
    """Even part of g^eq_l at rest and at the wall temperature: w_l[rho T_w + 4.5 (lam T_w - rho T_w/3)(|c|^2-1)]."""
    return W[l] * (rho * T_w + 4.5 * (lam * T_w - rho * T_w / 3.0) * (C2[l] - 1))


def stream(fstar, gstar, rho_wall, p: Params):
    """Pull streaming f_l(x) = f*_l(x - c_l); periodic x, y; bounce-back at the z walls."""
    f = torch.empty_like(fstar)
    g = torch.empty_like(gstar)
    lam = p.lam
    for l in range(Q):
        cx, cy, cz = C[l]
        sf = torch.roll(fstar[l], shifts=(cy, cx), dims=(1, 2))
        sg = torch.roll(gstar[l], shifts=(cy, cx), dims=(1, 2))
        if p.periodic_z or cz == 0:
            f[l] = torch.roll(sf, shifts=cz, dims=0)
            g[l] = torch.roll(sg, shifts=cz, dims=0)
            continue
        if cz > 0:   # arrives from below; the bottom layer receives it from the wall
            f[l, 1:] = sf[:-1]
            g[l, 1:] = sg[:-1]
            zw, T_w = 0, p.T_d
        else:        # arrives from above; the top layer receives it from the wall
            f[l, :-1] = sf[1:]
            g[l, :-1] = sg[1:]
            zw, T_w = p.nz - 1, p.T_u
        lb = OPP[l]
        f[l, zw] = fstar[lb, zw]
        g[l, zw] = -gstar[lb, zw] + 2.0 * wall_g_even(l, rho_wall[zw], T_w, lam)
    return f, g


def step(f, g, p: Params):
    """State at time n -> state at time n+1."""
    fstar, gstar, rho = collide(f, g, p)
    return stream(fstar, gstar, rho, p)


def init_state(rho, T, p: Params):
    """f = f^eq(rho, 0, T), g = g^eq(rho, T, 0)."""
    rho = torch.as_tensor(rho, dtype=DT)
    T = torch.as_tensor(T, dtype=DT)
    zero = torch.zeros((3,) + tuple(rho.shape), dtype=DT)
    return equilibrium_f(rho, zero, T), equilibrium_g(rho, T, zero, p.lam)


def run(f, g, p: Params, nsteps: int):
    for _ in range(nsteps):
        f, g = step(f, g, p)
    return f, g


# ---------------------------------------------------------------------------------------
# Diagnostics: layer-averaged heat flux of Eq. (4) normalised as a Nusselt number.
# ---------------------------------------------------------------------------------------

def internal_energy(rho, T, p: Params):
    """U = c_v T + int_0^rho P_NI(s)/s^2 ds (Eq. (2), zero at rho -> 0): (G/4) exp(-2/rho) for
    the paper's psi; -T_v ln(1 - b rho) - a rho for the van der Waals variant."""
    if p.psi_kind == "vdw":
        return p.c_v * T - p.vdw_T * torch.log(1.0 - p.vdw_b * rho) - p.vdw_a * rho
    return p.c_v * T + 0.25 * p.G * torch.exp(-2.0 / rho)


def nusselt(f, g, p: Params):
    """Nu(z) = <rho U u_z - kappa dT/dz>_{x,y} / (kappa (T_d - T_u)/nz), and its mean over z.

    dT/dz by central differences with wall ghosts T(-1) = 2T_d - T(0), T(nz) = 2T_u - T(nz-1).
    """
    rho, j, T, F, u_eq, u = macroscopic(f, g, p)
    U = internal_energy(rho, T, p)
    nz = p.nz
    Tp = torch.cat([T[1:], (2.0 * p.T_u - T[nz - 1]).unsqueeze(0)])
    Tm = torch.cat([(2.0 * p.T_d - T[0]).unsqueeze(0), T[:-1]])
    dTdz = 0.5 * (Tp - Tm)
    flux = rho * U * u[2] - p.kappa * dTdz
    nu_z = flux.mean(dim=(1, 2)) / (p.kappa * (p.T_d - p.T_u) / nz)
    return nu_z.mean(), nu_z


def moments_out(f, g, p: Params):
    """rho, (u_x, u_y, u_z) physical, T of the state, as exported by lb_moments."""
    rho, j, T, F, u_eq, u = macroscopic(f, g, p)
    return rho, u, T


# ---------------------------------------------------------------------------------------
# Objective of the adjoint: time-averaged Nusselt number.
# ---------------------------------------------------------------------------------------

def time_averaged_nusselt(rho0, T0, p: Params, nsteps: int):
    """J = (1/N) sum_{n=1..N} Nu_mean(state n), starting from the equilibrium of (rho0, T0).

    Differentiable (PyTorch autograd) in T0 and in p.T_d, p.T_u, p.G when those are tensors:
    the reverse pass of autograd through these plain steps is the exact discrete gradient.
    """
    f, g = init_state(rho0, T0, p)
    J = 0.0
    for _ in range(nsteps):
        f, g = step(f, g, p)
        J = J + nusselt(f, g, p)[0]
    return J / nsteps
