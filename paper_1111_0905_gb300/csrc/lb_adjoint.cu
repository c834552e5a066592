// lb_adjoint.cu -- discrete adjoint of the thermal D3Q19 step (reverse mode, FP64).
//
// Objective: J = (1/N) sum_{n=1..N} Nu_mean(x_n), the time-averaged Nusselt number of Eq. (4),
// x_n the pre-collision state at step n, x_{n+1} = Phi(x_n) the step of Eqs. (6)-(9) with the
// readings of the forward kernels. Gradients: dJ/dT_d, dJ/dT_u, dJ/dG and dJ/dT0 (the initial
// temperature field of lb_init). The adjoint state lambda_n = dJ/dx_n obeys
//   lambda_N = (1/N) dNu/dx_N,  lambda_n = (dPhi/dx_n)^T lambda_{n+1} + [n >= 1] (1/N) dNu/dx_n.
// One reverse step, for state n, in the reverse order of the forward operations:
//   streaming^T (push of lambda_{n+1}, bounce-back transposed, the thermal wall rule's density
//   and T_w terms) -> collision^T (f^eq(rho, u', T), g^eq(rho, T, u), counter term) -> the Nu
//   terms of state n -> divergence^T (radius-1 gather) -> velocities^T (u, u' -> j, F, rho) ->
//   force^T (radius-1 psi gather with the mirrored wall ghosts; dJ/dG) -> moments^T.
// The forward states are recomputed per segment from checkpoints taken every K steps; the
// macroscopic fields of a state are recomputed per reverse step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lb_ctx.h"

namespace tlbm {
namespace adj {

struct Geom { int nx, ny, nz, plane, N; };
struct Par {
  double tau, om, omk, G, gz, lam, cv, kappa, Td, Tu;
  double Kc;        // 1 / (N_t kappa (T_d - T_u) nx ny): weight of sum_x rho U u_z in J
  int include_nu;   // add (1/N_t) dNu_mean/dx of this state
};

// fields of M (forward macros of one state, MF_* of lb_kernels.cuh), each [N]
// fields of A (adjoints of the macros), each [N]
enum { AF_RHO = 0, AF_T, AF_UX, AF_UY, AF_UZ, AF_VX, AF_VY, AF_VZ, AF_D, AF_FX, AF_FY, AF_FZ, AF_JX, AF_JY,
       AF_JZ, AF_COUNT };
// per-block parameter partials
enum { P_TD = 0, P_TU, P_G, P_J, P_COUNT };

constexpr int kBlocks = 1024;
constexpr int kThreads = 256;

__device__ __forceinline__ void coords(int idx, const Geom& g, int& x, int& y, int& z) {
  x = idx % g.nx;
  y = (idx / g.nx) % g.ny;
  z = idx / g.plane;
}
__device__ __forceinline__ int at(const Geom& g, int x, int y, int z) {
  return z * g.plane + wrapi(y, g.ny) * g.nx + wrapi(x, g.nx);
}

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
  return s;
}

// rho, j, E, T, psi of state X ([38][N]: f then g, pre-collision, float64)
__global__ void macro_kernel(const double* __restrict__ X, Geom g, double* __restrict__ M) {
  const size_t N = g.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
    double f[Q], E = 0.0;
#pragma unroll
    for (int l = 0; l < Q; ++l) f[l] = X[l * N + i];
#pragma unroll
    for (int l = 0; l < Q; ++l) E += X[(Q + l) * N + i];
    double rho, jx, jy, jz;
    density_momentum<double>(f, rho, jx, jy, jz);
    M[MF_RHO * N + i] = rho; M[MF_JX * N + i] = jx; M[MF_JY * N + i] = jy; M[MF_JZ * N + i] = jz;
    M[MF_E * N + i] = E; M[MF_T * N + i] = E / rho; M[MF_PSI * N + i] = exp(-1.0 / rho);
  }
}

// Eq. (9): A_a = sum_{l>=1} W_l c_la psi(x + c_l) (mirrored ghosts), F = -G psi A + rho g_z z,
// u = (j + F/2)/rho, u' = (j + tau F)/rho
__global__ void force_fwd_kernel(Geom g, Par p, double* __restrict__ M) {
  const size_t N = g.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(i, g, x, y, z);
    double A[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int l = 1; l < Q; ++l) {
      const double nb = M[MF_PSI * N + at(g, x + CX(l), y + CY(l), mirror_z(z + CZ(l), g.nz))];
      if (CX(l)) A[0] += FW<double>(l) * CX(l) * nb;
      if (CY(l)) A[1] += FW<double>(l) * CY(l) * nb;
      if (CZ(l)) A[2] += FW<double>(l) * CZ(l) * nb;
    }
    const double rho = M[MF_RHO * N + i], psi = M[MF_PSI * N + i];
    const double F[3] = {-p.G * psi * A[0], -p.G * psi * A[1], -p.G * psi * A[2] + rho * p.gz};
    for (int a = 0; a < 3; ++a) {
      const double j = M[(MF_JX + a) * N + i];
      M[(MF_AX + a) * N + i] = A[a];
      M[(MF_FX + a) * N + i] = F[a];
      M[(MF_UX + a) * N + i] = (j + 0.5 * F[a]) / rho;
      M[(MF_VX + a) * N + i] = (j + p.tau * F[a]) / rho;
    }
  }
}

// D = sum_a [u_a(x+e_a) - u_a(x-e_a)]/2, u_z -> -u_z across the walls
__global__ void div_fwd_kernel(Geom g, double* __restrict__ M) {
  const size_t N = g.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(i, g, x, y, z);
    const double uz0 = M[MF_UZ * N + i];
    const double uzp = (z + 1 < g.nz) ? M[MF_UZ * N + i + g.plane] : -uz0;
    const double uzm = (z - 1 >= 0) ? M[MF_UZ * N + i - g.plane] : -uz0;
    double D = 0.5 * (M[MF_UX * N + at(g, x + 1, y, z)] - M[MF_UX * N + at(g, x - 1, y, z)]);
    D += 0.5 * (M[MF_UY * N + at(g, x, y + 1, z)] - M[MF_UY * N + at(g, x, y - 1, z)]);
    D += 0.5 * (uzp - uzm);
    M[MF_D * N + i] = D;
  }
}

// streaming^T, wall rules^T, collision^T and the Nu terms, per node
// adjoint of post-collision population l at node (x, y, z): lambda'_l(x + c_l), or through a wall
// the bounce-back that delivered f*_l(x) as f'_{opp(l)}(x) (g: with a minus sign)
__device__ __forceinline__ void adj_pull(const double* __restrict__ Ln, const Geom& g, int l, int i,
                                         int x, int y, int z, double& lf, double& lg) {
  const size_t N = g.N;
  const int zn = z + CZ(l);
  if (zn < 0 || zn >= g.nz) {
    lf = Ln[OPP(l) * N + i];
    lg = -Ln[(Q + OPP(l)) * N + i];
  } else {
    const int j = at(g, x + CX(l), y + CY(l), zn);
    lf = Ln[l * N + j];
    lg = Ln[(Q + l) * N + j];
  }
}

// collision^T, one node per thread. The populations are taken in pairs (l, opp(l)), whose
// equilibria share the part even in c_l and differ in sign in the odd part: with s = a_l + a_opp
// and d = a_l - a_opp the pair contributes s (even part) + d (odd part) to each adjoint.
__global__ void __launch_bounds__(256) coll_adj_kernel(const double* __restrict__ X, const double* __restrict__ M,
                                                       const double* __restrict__ Ln, Geom g, Par p,
                                                       double* __restrict__ L, double* __restrict__ A,
                                                       double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t N = g.N;
  double pTd = 0.0, pTu = 0.0, pG = 0.0, pJ = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(i, g, x, y, z);
    const double rho = M[MF_RHO * N + i], T = M[MF_T * N + i], E = rho * T;
    const double ux = M[MF_UX * N + i], uy = M[MF_UY * N + i], uz = M[MF_UZ * N + i];
    const double vx = M[MF_VX * N + i], vy = M[MF_VY * N + i], vz = M[MF_VZ * N + i];
    const double D = M[MF_D * N + i];
    double a_rho = 0.0;
    if (Ln) {
      // thermal wall rule: g'_m(x_w) = ... + 2 w_m [rho T_w + 4.5 (lam T_w - rho T_w/3)(|c_m|^2-1)]
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        const bool bot = (CZ(m) > 0 && z == 0), top = (CZ(m) < 0 && z == g.nz - 1);
        if (bot || top) {
          const double Tw = bot ? p.Td : p.Tu;
          const double lm = Ln[(Q + m) * N + i];
          const double k = CSQ(m) - 1;
          a_rho += 2.0 * WT<double>(m) * Tw * (1.0 - 1.5 * k) * lm;
          const double dTw = 2.0 * WT<double>(m) * (rho + 4.5 * (p.lam - rho / 3.0) * k) * lm;
          if (bot) pTd += dTw; else pTu += dTw;
        }
      }
    }
    // collision^T: f* = (1 - om) f + om f^eq(rho, v, T), g* = (1 - omk) g + omk g^eq(rho, T, u) + w S
    const double vv = vx * vx + vy * vy + vz * vz, uu = ux * ux + uy * uy + uz * uz;
    double a_T = 0.0, lS = 0.0;
    double sfk = 0.0, sf = 0.0, sg = 0.0;          // sums of s_f k, s_f and s_g over the pairs
    double avx = 0.0, avy = 0.0, avz = 0.0, aux = 0.0, auy = 0.0, auz = 0.0;
    const double Tm = 4.5 * (T - 1.0 / 3.0), lk = 4.5 * (p.lam - rho / 3.0);
    const double ev0 = 1.0 - 1.5 * vv, eu0 = 1.0 - 1.5 * uu;   // the velocity-squared parts
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      if (l != 0 && (l & 1) == 0) continue;    // with its odd partner
      const int o = (l == 0) ? 0 : OPP(l);
      double lf = 0.0, lg = 0.0, lfo = 0.0, lgo = 0.0;
      if (Ln) {
        adj_pull(Ln, g, l, i, x, y, z, lf, lg);
        if (l != 0) adj_pull(Ln, g, o, i, x, y, z, lfo, lgo);
      }
      L[l * N + i] = (1.0 - p.om) * lf;
      L[(Q + l) * N + i] = (1.0 - p.omk) * lg;
      if (l != 0) {
        L[o * N + i] = (1.0 - p.om) * lfo;
        L[(Q + o) * N + i] = (1.0 - p.omk) * lgo;
      }
      // class factor k = |c_l|^2 - 1 (-1 rest, 0 axis, +1 diagonal) taken by branches that fold,
      // so that no multiply by k is executed
      const int kc = CSQ(l) - 1;
      const double w = WT<double>(l);
      const double af = p.om * w * lf, ag = p.omk * w * lg;
      // f^eq: even 1 + 4.5 (c.v)^2 - 1.5 v.v + 4.5 (T - 1/3) k, odd 3 c.v; d/dT 4.5 k rho;
      // d/dv rho (3 c + 9 (c.v) c - 3 v)
      // g^eq: rho T P(u) + 4.5 (lam T - rho T/3) k, P even 1 + 4.5 (c.u)^2 - 1.5 u.u, odd 3 c.u
      if (l == 0) {
        // the rest population (c = 0, k = -1): even parts only
        a_rho += af * (ev0 - Tm) + T * (ag * (eu0 + 1.5));
        a_T += rho * (ag * eu0) - ag * lk;
        sfk -= af;
        sf += af;
        sg += ag;
        lS += w * lg;
      } else {
        const double cv = cdot<double>(l, vx, vy, vz);
        const double cu = cdot<double>(l, ux, uy, uz);
        const double afo = p.om * w * lfo, ago = p.omk * w * lgo;
        const double s_f = af + afo, d_f = af - afo, s_g = ag + ago, d_g = ag - ago;
        const double evf = kc == 0 ? ev0 : ev0 + Tm;          // axis: k = 0, diagonal: k = 1
        a_rho += s_f * (evf + 4.5 * cv * cv) + d_f * (3.0 * cv);
        if (kc != 0) sfk += s_f;
        sf += s_f;
        const double ef = 3.0 * d_f + 9.0 * s_f * cv;
        cadd<double>(l, ef, avx, avy, avz);
        const double Pe = eu0 + 4.5 * cu * cu, Po = 3.0 * cu;
        const double Pk = kc == 0 ? Pe : Pe - 1.5;
        a_rho += T * (s_g * Pk + d_g * Po);
        a_T += rho * (s_g * Pe + d_g * Po);
        if (kc != 0) a_T += s_g * lk;
        sg += s_g;
        const double eg = 3.0 * d_g + 9.0 * s_g * cu;
        cadd<double>(l, eg, aux, auy, auz);
        lS += w * (lg + lgo);
      }
    }
    a_T += 4.5 * rho * sfk;
    double a_v[3] = {rho * (avx - 3.0 * vx * sf), rho * (avy - 3.0 * vy * sf), rho * (avz - 3.0 * vz * sf)};
    double a_u[3] = {E * (aux - 3.0 * ux * sg), E * (auy - 3.0 * uy * sg), E * (auz - 3.0 * uz * sg)};
    // counter term S = -rho T D / c_v
    a_rho += lS * (-T * D / p.cv);
    a_T += lS * (-rho * D / p.cv);
    const double a_D = lS * (-E / p.cv);
    // Nu terms: J_n = (1/N_t)[1 + sum_x rho U u_z / (kappa (T_d - T_u) nx ny)], U = c_v T + (G/4) e^{-2/rho}
    if (p.include_nu) {
      const double psi = M[MF_PSI * N + i];
      const double e2 = psi * psi;            // e^{-2/rho} = psi^2
      const double U = p.cv * T + 0.25 * p.G * e2;
      a_rho += p.Kc * (U * uz + uz * 0.5 * p.G * e2 / rho);
      a_T += p.Kc * rho * p.cv * uz;
      a_u[2] += p.Kc * rho * U;
      pG += p.Kc * rho * uz * 0.25 * e2;
      pJ += p.Kc * rho * U * uz;       // J = 1 + sum_n sum_x Kc rho U u_z (conduction telescopes)
      const double conv = p.Kc * rho * U * uz / (p.Td - p.Tu);
      pTd -= conv;
      pTu += conv;
    }
    A[AF_RHO * N + i] = a_rho; A[AF_T * N + i] = a_T; A[AF_D * N + i] = a_D;
    A[AF_UX * N + i] = a_u[0]; A[AF_UY * N + i] = a_u[1]; A[AF_UZ * N + i] = a_u[2];
    A[AF_VX * N + i] = a_v[0]; A[AF_VY * N + i] = a_v[1]; A[AF_VZ * N + i] = a_v[2];
  }
  const double s0 = block_sum(pTd, sh), s1 = block_sum(pTu, sh), s2 = block_sum(pG, sh);
  const double s3 = block_sum(pJ, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * P_COUNT + P_TD] += s0;
    part[blockIdx.x * P_COUNT + P_TU] += s1;
    part[blockIdx.x * P_COUNT + P_G] += s2;
    part[blockIdx.x * P_COUNT + P_J] += s3;
  }
}

// divergence^T (radius-1 gather) and velocities^T: u = (j + F/2)/rho, u' = (j + tau F)/rho
__global__ void vel_adj_kernel(const double* __restrict__ M, Geom g, Par p, double* __restrict__ A) {
  const size_t N = g.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(i, g, x, y, z);
    double lu[3] = {A[AF_UX * N + i], A[AF_UY * N + i], A[AF_UZ * N + i]};
    lu[0] += 0.5 * (A[AF_D * N + at(g, x - 1, y, z)] - A[AF_D * N + at(g, x + 1, y, z)]);
    lu[1] += 0.5 * (A[AF_D * N + at(g, x, y - 1, z)] - A[AF_D * N + at(g, x, y + 1, z)]);
    const double dm = (z >= 1) ? A[AF_D * N + i - g.plane] : A[AF_D * N + i];
    const double dp = (z <= g.nz - 2) ? A[AF_D * N + i + g.plane] : A[AF_D * N + i];
    lu[2] += 0.5 * (dm - dp);
    const double inv = 1.0 / M[MF_RHO * N + i];   // one division per node on the FP64 pipe
    double a_rho = A[AF_RHO * N + i];
    for (int a = 0; a < 3; ++a) {
      const double lv = A[(AF_VX + a) * N + i];
      A[(AF_JX + a) * N + i] = (lv + lu[a]) * inv;
      A[(AF_FX + a) * N + i] = (p.tau * lv + 0.5 * lu[a]) * inv;
      a_rho -= (M[(MF_VX + a) * N + i] * lv + M[(MF_UX + a) * N + i] * lu[a]) * inv;
    }
    A[AF_RHO * N + i] = a_rho;
  }
}

// c_l . (lambda_Fx, lambda_Fy, lambda_Fz) at node j, loading only the components c_l has
__device__ __forceinline__ double cdot_at(int l, const double* __restrict__ A, size_t N, int j) {
  const double x = CX(l) != 0 ? A[AF_FX * N + j] : 0.0;
  const double y = CY(l) != 0 ? A[AF_FY * N + j] : 0.0;
  const double z = CZ(l) != 0 ? A[AF_FZ * N + j] : 0.0;
  return cdot<double>(l, x, y, z);
}

// force^T (psi gather with mirrored ghosts), psi^T, T = E/rho ^T and moments^T
__global__ void force_adj_kernel(const double* __restrict__ M, Geom g, Par p,
                                 const double* __restrict__ A, double* __restrict__ L,
                                 double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t N = g.N;
  double pG = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(i, g, x, y, z);
    const double psi = M[MF_PSI * N + i], rho = M[MF_RHO * N + i], T = M[MF_T * N + i];
    const double lF[3] = {A[AF_FX * N + i], A[AF_FY * N + i], A[AF_FZ * N + i]};
    // own psi factor of F(x) = -G psi(x) A(x)
    double lpsi = -p.G * (lF[0] * M[MF_AX * N + i] + lF[1] * M[MF_AY * N + i] + lF[2] * M[MF_AZ * N + i]);
    pG -= psi * (lF[0] * M[MF_AX * N + i] + lF[1] * M[MF_AY * N + i] + lF[2] * M[MF_AZ * N + i]);
    // psi(y) enters F(x) for every (x, l) with mirror(x + c_l) = y
#pragma unroll
    for (int l = 1; l < Q; ++l) {
      const double W = FW<double>(l);
      const int zi = z - CZ(l);          // interior link x = y - c_l
      if (zi >= 0 && zi < g.nz) {
        const int j = at(g, x - CX(l), y - CY(l), zi);
        const double cl = cdot_at(l, A, N, j);
        lpsi += -p.G * W * cl * M[MF_PSI * N + j];
      }
      const int zg = z + CZ(l);          // ghost link: x in this plane, x + c_l beyond a wall
      if (CZ(l) != 0 && (zg < 0 || zg >= g.nz)) {
        const int j = at(g, x - CX(l), y - CY(l), z);
        const double cl = cdot_at(l, A, N, j);
        lpsi += -p.G * W * cl * M[MF_PSI * N + j];
      }
    }
    const double inv = 1.0 / rho;
    double a_rho = A[AF_RHO * N + i] + p.gz * lF[2] + lpsi * psi * inv * inv;
    const double a_T = A[AF_T * N + i];
    const double a_E = a_T * inv;
    a_rho -= a_T * T * inv;
    const double lj[3] = {A[AF_JX * N + i], A[AF_JY * N + i], A[AF_JZ * N + i]};
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      L[l * N + i] += (l == 0) ? a_rho : a_rho + cdot<double>(l, lj[0], lj[1], lj[2]);
      L[(Q + l) * N + i] += a_E;
    }
  }
  const double s = block_sum(pG, sh);
  if (threadIdx.x == 0) part[blockIdx.x * P_COUNT + P_G] += s;
}

// dJ/dT0 from lambda_0: x_0 = (f^eq(rho0, 0, T0), g^eq(rho0, T0, 0))
__global__ void init_grad_kernel(const double* __restrict__ L0, const double* __restrict__ M0, Geom g,
                                 double lam, double* __restrict__ out) {
  const size_t N = g.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
    const double rho = M0[MF_RHO * N + i];
    double s = 0.0;
    for (int l = 0; l < Q; ++l) {
      const double k = CSQ(l) - 1, w = WT<double>(l);
      s += L0[l * N + i] * w * rho * 4.5 * k + L0[(Q + l) * N + i] * w * (rho + 4.5 * (lam - rho / 3.0) * k);
    }
    out[i] = s;
  }
}

}  // namespace adj
}  // namespace tlbm

using namespace tlbm;

namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace

extern "C" int lb_adjoint_step(lb_ctx* c, long long nsteps, int checkpoint_every, double* J,
                               double* dJ_dTd, double* dJ_dTu, double* dJ_dG, double* dJ_dT0) {
  using namespace tlbm::adj;
  if (!c) return LB_EINVAL;
  if (nsteps < 1 || checkpoint_every < 0) return lb_fail(c, LB_EINVAL, "nsteps must be >= 1 and checkpoint_every >= 0");
  if (dJ_dT0 && (c->step != 0 || !c->from_init))
    return lb_fail(c, LB_EINVAL, "dJ_dT0 needs the state of lb_init (step 0)");
  if (!(c->p.T_d != c->p.T_u)) return lb_fail(c, LB_EINVAL, "T_d == T_u: Nu is undefined");
  if (c->p.forcing != FORCE_SHIFT || c->p.psi_kind != PSI_EXP)
    return lb_fail(c, LB_EUNSUP, "the adjoint transposes the paper's scheme (velocity shift, psi = exp(-1/rho)) only");
  const size_t N = (size_t)c->N;
  const size_t pbytes = (size_t)c->ops->slots * N * c->ops->esize;
  const size_t sbytes = 2 * (size_t)Q * N * sizeof(double);
  const size_t mstate = (size_t)MF_COUNT * N;   // doubles per state's fields
  // device bytes of the call for segment length k (the allocations below)
  auto bytes_for = [&](long long k) -> double {
    const double nck_k = (double)((nsteps + k - 1) / k);
    return nck_k * 2.0 * (double)pbytes + 4.0 * (double)pbytes + 64.0 + 3.0 * (double)sbytes +
           (double)(k + 1) * (double)mstate * 8.0 + (double)AF_COUNT * (double)N * 8.0 +
           (double)kBlocks * P_COUNT * 8.0 + (dJ_dT0 ? (double)N * 8.0 : 0.0);
  };
  long long K = checkpoint_every < nsteps ? checkpoint_every : nsteps;
  if (checkpoint_every == 0) {
    // the longest segment whose buffers fit in 85 % of the free device memory: every state's
    // fields kept (no recomputation with FP64 storage) when they fit
    size_t free_b = 0, total_b = 0;
    LB_CU(c, cudaMemGetInfo(&free_b, &total_b));
    const double budget = 0.85 * (double)free_b;
    const double per_k = (double)mstate * 8.0;
    long long k = std::min<long long>(nsteps, (long long)std::max(1.0, budget / per_k));
    while (k > 1 && bytes_for(k) > budget) --k;
    if (bytes_for(k) > budget) return lb_fail(c, LB_ENOMEM, "adjoint buffers do not fit for any segment length");
    K = k;
  }
  const long long nck = (nsteps + K - 1) / K;
  cudaStream_t st = c->stream;
  Geom g{c->p.nx, c->p.ny, c->p.nz, c->plane, c->N};

  // FP64 storage: the step writes the fields of the state it reads (adj_m), so the reverse sweep
  // needs no separate moments, force and divergence passes; other storage recomputes them in
  // FP64 from the FP64 image of each state.
  const bool fields = (c->ops->esize == sizeof(double));
  DevBuf ck, rb, xs, mb, ab, lb, pt, d0;
  if (cudaMalloc(&ck.p, (size_t)nck * 2 * pbytes) != cudaSuccess ||
      cudaMalloc(&rb.p, 4 * pbytes + 64) != cudaSuccess ||
      cudaMalloc(&xs.p, sbytes) != cudaSuccess ||
      cudaMalloc(&mb.p, (size_t)(K + 1) * mstate * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ab.p, (size_t)AF_COUNT * N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&lb.p, 2 * sbytes) != cudaSuccess ||
      cudaMalloc(&pt.p, (size_t)kBlocks * P_COUNT * sizeof(double)) != cudaSuccess ||
      (dJ_dT0 && cudaMalloc(&d0.p, N * sizeof(double)) != cudaSuccess))
    return lb_fail(c, LB_ENOMEM, "adjoint buffers");
  unsigned char* ckp = static_cast<unsigned char*>(ck.p);
  unsigned char* rbp = static_cast<unsigned char*>(rb.p);
  double* X = static_cast<double*>(xs.p);        // FP64 image of one state
  double* Ms = static_cast<double*>(mb.p);       // fields of the segment's states n0..n1
  double* A = static_cast<double*>(ab.p);
  double* Lb[2] = {static_cast<double*>(lb.p), static_cast<double*>(lb.p) + 2 * Q * N};
  double* part = static_cast<double*>(pt.p);
  LB_CU(c, cudaMemsetAsync(part, 0, (size_t)kBlocks * P_COUNT * sizeof(double), st));
  const int frc = flush_sample(c);    // a Nu sample due for the time average of lb_nusselt
  if (frc) return frc;

  const double dT = c->p.T_d - c->p.T_u;
  Par par{c->p.tau_nu, 1.0 / c->p.tau_nu, 1.0 / c->p.tau_kappa, c->p.G, c->p.g_z, c->lam, c->p.c_v,
          c->p.kappa, c->p.T_d, c->p.T_u,
          1.0 / ((double)nsteps * c->p.kappa * dT * (double)c->p.nx * (double)c->p.ny), 0};
  const int nb = (int)std::min<long long>(kBlocks, ((long long)N + kThreads - 1) / kThreads);
  // fields of a state from its storage image (a.fin, a.gin) by the separate FP64 passes
  auto fields_by_passes = [&](const KArgs& a, double* Mn) -> int {
    LB_CU(c, c->ops->pops(a, X, X + Q * N, st));
    macro_kernel<<<nb, kThreads, 0, st>>>(X, g, Mn);
    force_fwd_kernel<<<nb, kThreads, 0, st>>>(g, par, Mn);
    div_fwd_kernel<<<nb, kThreads, 0, st>>>(g, Mn);
    LB_CU(c, cudaGetLastError());
    return LB_OK;
  };

  // forward: checkpoints every K steps; with FP64 storage the last segment's fields as it goes
  const dim3 grid = fused_grid(c);
  const long long n0_last = (nck - 1) * K;
  for (long long n = 0; n < nsteps; ++n) {
    if (n % K == 0) {
      unsigned char* dst = ckp + (size_t)(n / K) * 2 * pbytes;
      LB_CU(c, cudaMemcpyAsync(dst, c->f[c->cur], pbytes, cudaMemcpyDeviceToDevice, st));
      LB_CU(c, cudaMemcpyAsync(dst + pbytes, c->g[c->cur], pbytes, cudaMemcpyDeviceToDevice, st));
    }
    KArgs a = make_args(c);
    if (fields && n >= n0_last) a.adj_m = Ms + (size_t)(n - n0_last) * mstate;
    LB_CU(c, c->ops->fused(a, MODE_STEP, c->by, grid, st));
    c->cur ^= 1;
    c->step += 1;
  }
  if (fields) {
    const int rc = fields_by_passes(make_args(c), Ms + (size_t)(nsteps - n0_last) * mstate);
    if (rc != LB_OK) return rc;
  }

  int li = 0;   // Lb[li] = lambda_{n+1} (zero before the last state)
  bool have_next = false;
  for (long long s = nck - 1; s >= 0; --s) {
    const long long n0 = s * K;
    const long long n1 = (s == nck - 1) ? nsteps : (s + 1) * K - 1;   // states n0..n1 of this segment
    if (!(fields && s == nck - 1)) {
      // recompute the segment from its checkpoint: the fields of states n0..n1
      unsigned char* src = ckp + (size_t)s * 2 * pbytes;
      LB_CU(c, cudaMemcpyAsync(rbp, src, pbytes, cudaMemcpyDeviceToDevice, st));
      LB_CU(c, cudaMemcpyAsync(rbp + pbytes, src + pbytes, pbytes, cudaMemcpyDeviceToDevice, st));
      int rc = 0;
      for (long long n = n0; n <= n1; ++n) {
        KArgs a = make_args(c);
        a.fin = rbp + (size_t)rc * 2 * pbytes;
        a.gin = rbp + (size_t)rc * 2 * pbytes + pbytes;
        double* Mn = Ms + (size_t)(n - n0) * mstate;
        if (!fields || n == n1) {
          const int frc2 = fields_by_passes(a, Mn);
          if (frc2 != LB_OK) return frc2;
        } else {
          a.adj_m = Mn;
        }
        if (n < n1) {
          a.fout = rbp + (size_t)(1 - rc) * 2 * pbytes;
          a.gout = rbp + (size_t)(1 - rc) * 2 * pbytes + pbytes;
          LB_CU(c, c->ops->fused(a, MODE_STEP, c->by, grid, st));
          rc ^= 1;
        }
      }
    }
    for (long long n = n1; n >= n0; --n) {
      const double* Mn = Ms + (size_t)(n - n0) * mstate;
      par.include_nu = (n >= 1) ? 1 : 0;
      double* Lcur = Lb[1 - li];
      coll_adj_kernel<<<nb, kThreads, 0, st>>>(nullptr, Mn, have_next ? Lb[li] : nullptr, g, par, Lcur, A, part);
      vel_adj_kernel<<<nb, kThreads, 0, st>>>(Mn, g, par, A);
      force_adj_kernel<<<nb, kThreads, 0, st>>>(Mn, g, par, A, Lcur, part);
      LB_CU(c, cudaGetLastError());
      li = 1 - li;
      have_next = true;
    }
    if (s == 0 && dJ_dT0) {
      init_grad_kernel<<<nb, kThreads, 0, st>>>(Lb[li], Ms, g, c->lam, static_cast<double*>(d0.p));
      LB_CU(c, cudaGetLastError());
    }
  }
  std::vector<double> hp((size_t)kBlocks * P_COUNT);
  LB_CU(c, cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (dJ_dT0) LB_CU(c, cudaMemcpyAsync(dJ_dT0, d0.p, N * sizeof(double), cudaMemcpyDeviceToHost, st));
  LB_CU(c, cudaStreamSynchronize(st));
  double s[P_COUNT] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < kBlocks; ++b)
    for (int k = 0; k < P_COUNT; ++k) s[k] += hp[(size_t)b * P_COUNT + k];
  if (J) *J = 1.0 + s[P_J];
  if (dJ_dTd) *dJ_dTd = s[P_TD];
  if (dJ_dTu) *dJ_dTu = s[P_TU];
  if (dJ_dG) *dJ_dG = s[P_G];
  return LB_OK;
}
