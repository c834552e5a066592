// lb_kernels.cuh -- sm_103a kernels of the thermal pseudopotential D3Q19 lattice Boltzmann step.
//
// Biferale, Perlekar, Sbragaglia, Toschi, arXiv:1111.0905, "Algorithm" paragraph:
// Eqs. (6)-(7) (two BGK lattice equations), Eq. (8) (moments), Eq. (9) (pseudopotential force
// with psi = exp(-1/rho)), the velocity shift u' = u + tau_nu F/rho, the temperature from g in
// the f equilibrium, and the counter term that yields the P0 div(u) term of Eq. (3).
//
// Storage: structure of arrays, population l of node idx at base[l*N + idx], idx = x + nx*(y + ny*z).
// Streaming: pull with two lattices (ping-pong). The buffer between steps holds the
// post-collision populations f*(n); the state at time n+1 is their pull plus the wall rules.
//
// Fused step kernel: one CTA owns a 32 x BY column tile and a range of z planes and marches up
// in z. Per leading plane p it (M) pulls f on the tile plus a radius-2 ring and stores psi, rho,
// j in shared memory; (U) for plane p-1 forms the force F and the physical velocity
// u = (j + F/2)/rho on the tile plus a radius-1 ring; (C) for plane p-2 it pulls f and g of the
// tile, takes div(u) from the three u planes and collides. Shared memory holds rolling windows
// of psi and rho/j planes (3 or 4 deep), 3 u planes and 2 F planes, so the only HBM traffic is
// the populations (the ring pulls hit L1/L2). One or two barriers per plane.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#ifndef TLBM_STAGE
#define TLBM_STAGE 1
#endif

namespace tlbm {

constexpr int Q = 19;
constexpr int BX = 32;      // tile width in x: one warp per row
constexpr int NPART = 8;    // diagnostics partials per (plane, tile)

// D3Q19: 0 rest; 1..6 axis (+-x, +-y, +-z); 7..10 xy diagonals; 11..14 xz; 15..18 yz.
__host__ __device__ constexpr int CX(int l) {
  return (l == 1 || l == 7 || l == 9 || l == 11 || l == 13) ? 1
       : (l == 2 || l == 8 || l == 10 || l == 12 || l == 14) ? -1 : 0;
}
__host__ __device__ constexpr int CY(int l) {
  return (l == 3 || l == 7 || l == 10 || l == 15 || l == 17) ? 1
       : (l == 4 || l == 8 || l == 9 || l == 16 || l == 18) ? -1 : 0;
}
__host__ __device__ constexpr int CZ(int l) {
  return (l == 5 || l == 11 || l == 14 || l == 15 || l == 18) ? 1
       : (l == 6 || l == 12 || l == 13 || l == 16 || l == 17) ? -1 : 0;
}
__host__ __device__ constexpr int OPP(int l) { return l == 0 ? 0 : ((l & 1) ? l + 1 : l - 1); }
__host__ __device__ constexpr int CSQ(int l) { return l == 0 ? 0 : (l <= 6 ? 1 : 2); }
template <class R> __host__ __device__ constexpr R WT(int l) {
  return l == 0 ? R(1) / R(3) : (l <= 6 ? R(1) / R(18) : R(1) / R(36));
}
// Force weights of Eq. (9): W(1) = 1/6, W(2) = 1/12 (isotropic to 4th order with D3Q19 links).
template <class R> __host__ __device__ constexpr R FW(int l) {
  return CSQ(l) == 1 ? R(1) / R(6) : R(1) / R(12);
}

// ---------------------------------------------------------------------------------------
// Storage precision. Every form stores deviations from the reference equilibria,
// df_l = f_l - f^eq_l(rho0, 0, T0) and dg_l = g_l - g^eq_l(rho0, T0, 0), so that the moments
// and the collision work on small numbers (the 16-bit forms need it; FP32 gains accuracy).
// ---------------------------------------------------------------------------------------
// FP16 storage against local references. Each lattice holds, after its 19 population slots, two
// reference slots per node: for the node y that wrote them, the deviations of the rest
// equilibria f^eq(rho_y, 0, T_y) and g^eq(rho_y, T_y, 0) (of the colliding step) per class,
//   f: a1 = w1 drho, a2 = w2 (4.5 dE - 0.5 drho)  (axis, diagonal), a0 = 12 (a1 - a2) (rest),
//   g: b1 = w1 dE,   b2 = w2 (4.5 lam dT - 0.5 dE), b0 = 12 (b1 - b2),
// drho = rho - rho0, dE = rho T - rho0 T0, dT = T - T0, themselves rounded to FP16 (so that the
// writer and every reader use the same values). A population slot holds its deviation minus the
// reference of its class at the node that wrote it, rounded to FP16: a pull of population l from
// node y adds y's reference back. The stored numbers are then the non-equilibrium and velocity
// parts of the populations (|u| ~ 1e-2) instead of the density and temperature contrast between
// the node and the global reference state (O(1) across a liquid-vapour interface), which is
// what FP16's 11-bit significand rounds.
struct __align__(2) half_loc { __half h; };
template <class S> struct IsLoc { static constexpr bool v = false; };
template <> struct IsLoc<half_loc> { static constexpr bool v = true; };
// population slots per lattice: 19, plus the two reference slots of the local-reference storage
template <class S> __host__ __device__ constexpr int slots() { return IsLoc<S>::v ? Q + 2 : Q; }

template <class S> struct Store;
template <> struct Store<double> {
  using R = double;
  static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
  static __device__ __forceinline__ double rt(double v) { return v; }
};
template <> struct Store<float> {
  using R = float;
  static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
  static __device__ __forceinline__ float rt(float v) { return v; }
};
template <> struct Store<__nv_bfloat16> {
  using R = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float rt(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};
template <> struct Store<__half> {
  using R = float;
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ float rt(float v) { return __half2float(__float2half_rn(v)); }
};
template <> struct Store<half_loc> {
  using R = float;
  static __device__ __forceinline__ float ld(const half_loc* p) {
    return __half2float(__ldg(reinterpret_cast<const __half*>(p)));
  }
  static __device__ __forceinline__ void st(half_loc* p, float v) { p->h = __float2half_rn(v); }
  static __device__ __forceinline__ float rt(float v) { return __half2float(__float2half_rn(v)); }
};



// Parameters of the hot path in the compute precision R, precomputed on the host so that the
// FP32 kernels never convert from double (conversions run on GB300's narrow FP64 pipe).
template <class R> struct KPar {
  R tau_nu, omega_nu, omega_kappa, G, g_z, lam, inv_cv, T_d, T_u, rho0, T0, E0;
  R va, vb, vT, vk;   // van der Waals-type psi: a, b, T_v, 2/(-G)
  R psi0, irho0;      // psi(rho0) = exp(-1/rho0) and 1/rho0 (deviation form of psi)
};

// Scheme variants (comparisons with the paper's scheme, which is variant 0 of each).
constexpr int FORCE_SHIFT = 0;   // equilibrium velocity u' = (j + tau F)/rho (the paper)
constexpr int FORCE_GUO = 1;     // f^eq at u = (j + F/2)/rho plus (1 - 1/(2 tau)) S_l
constexpr int PSI_EXP = 0;       // psi = exp(-1/rho) (the paper)
constexpr int PSI_VDW = 1;       // psi = rho sqrt(2 (a - b T_v/(1 - b rho))/(-G))
// Kernel variant index: bit 0 = Guo forcing, bit 1 = van der Waals psi (0 = the paper's scheme;
// a compile-time choice, so the paper's scheme carries no code of the variants).
constexpr int VAR_GUO = 1, VAR_VDW = 2;
__host__ __device__ constexpr int variant_of(int forcing, int psi_kind) {
  return (forcing == FORCE_GUO ? VAR_GUO : 0) | (psi_kind == PSI_VDW ? VAR_VDW : 0);
}

// Forward fields of one state that the discrete adjoint linearises around, each [N] float64:
// density, momentum, rho T, T, psi, force, physical and equilibrium velocities, div(u) and the
// psi-gradient sums A of Eq. (9) (F = -G psi A + rho g_z z).
enum { MF_RHO = 0, MF_JX, MF_JY, MF_JZ, MF_E, MF_T, MF_PSI, MF_FX, MF_FY, MF_FZ, MF_UX, MF_UY, MF_UZ,
       MF_VX, MF_VY, MF_VZ, MF_D, MF_AX, MF_AY, MF_AZ, MF_COUNT };

struct KArgs {
  const void* fin; const void* gin;   // post-collision lattices of the previous step
  void* fout; void* gout;             // lattices written by this step
  int nx, ny, nz, plane, N;
  int tiles_x, ntiles, zc;
  int forcing, psi_kind;              // FORCE_*, PSI_*
  double tau_nu, omega_nu, omega_kappa, G, g_z, lam, inv_cv, c_v, kappa, T_d, T_u;
  double rho0, T0, E0;                // reference state of the deviations (E0 = rho0 T0)
  double fbase[3], gbase[3];          // f^eq(rho0,0,T0), g^eq(rho0,T0,0) per class: rest, axis, diagonal
  unsigned loff[19];                  // l N - c_lz plane (mod 2^32): lattice and plane part of a pull
  // moments mode outputs (any may be null)
  double* rho_out; double* ux_out; double* uy_out; double* uz_out; double* T_out;
  double* part;                       // [nz][ntiles][NPART] diagnostics partials (may be null)
  double* adj_m;                      // FP64 step: MF_* fields of the state read ([MF_COUNT][N]) or null
  double* pre;                        // FP64 form: rho, 1/rho, jx, jy, jz, psi of the state read ([6][N])
  KPar<double> pd;                    // the parameters above in double ...
  KPar<float> pf;                     // ... and in float
};

template <class R> __device__ __forceinline__ const KPar<R>& kpar(const KArgs& a);
template <> __device__ __forceinline__ const KPar<double>& kpar<double>(const KArgs& a) { return a.pd; }
template <> __device__ __forceinline__ const KPar<float>& kpar<float>(const KArgs& a) { return a.pf; }

__host__ __device__ __forceinline__ int wrapi(int a, int n) { int m = a % n; return m < 0 ? m + n : m; }
// Plane index of the reflection of plane k across the halfway walls (applied repeatedly).
__host__ __device__ __forceinline__ int mirror_z(int k, int nz) {
  int m = wrapi(k, 2 * nz);
  return m < nz ? m : 2 * nz - 1 - m;
}

template <class S>
__device__ __forceinline__ float loc_ref(const S* __restrict__ buf, unsigned e, int ls, unsigned N);

// Pull the 19 populations of node (col[1], row[1], pz): v_l = buf_l(x - c_l). Across a wall the
// bounce-back source buf_{opp(l)}(x) is returned (the g wall rule is applied by the caller).
template <class S, class R>
__device__ __forceinline__ void pull(R (&v)[Q], const S* __restrict__ buf, int N, int pz, int nz,
                                     int plane, const int (&col)[3], const int (&row)[3]) {
  const int own = pz * plane + row[1] + col[1];
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const int zs = pz - CZ(l);
    if (zs < 0 || zs >= nz) {
      v[l] = Store<S>::ld(buf + (size_t)OPP(l) * N + own);
      if constexpr (IsLoc<S>::v)
        v[l] = v[l] + loc_ref<S>(buf, (unsigned)OPP(l) * (unsigned)N + (unsigned)own, OPP(l), (unsigned)N);
    } else {
      const size_t e = (size_t)l * N + (size_t)(zs * plane + row[1 - CY(l)] + col[1 - CX(l)]);
      v[l] = Store<S>::ld(buf + e);
      if constexpr (IsLoc<S>::v) v[l] = v[l] + loc_ref<S>(buf, (unsigned)e, l, (unsigned)N);
    }
  }
}

// c_l . (x, y, z) from the nonzero components of c_l only (with l a compile-time constant the
// branches fold away). Written as R(c) * x + ..., an IEEE multiply by a zero component (and the
// add of its +-0) would still be executed: 0 * x cannot be folded (x may be a NaN or infinite).
template <class R>
__device__ __forceinline__ R cdot(int l, R x, R y, R z) {
  const int cx = CX(l), cy = CY(l), cz = CZ(l);
  R s;
  if (cx != 0) {
    s = cx > 0 ? x : -x;
    if (cy != 0) s = cy > 0 ? s + y : s - y;
    if (cz != 0) s = cz > 0 ? s + z : s - z;
  } else if (cy != 0) {
    s = cy > 0 ? y : -y;
    if (cz != 0) s = cz > 0 ? s + z : s - z;
  } else if (cz != 0) {
    s = cz > 0 ? z : -z;
  } else {
    s = R(0);
  }
  return s;
}
// c_l . (x, y, z) in the step kernel of storage S: from the nonzero components, except for the
// FP32 kernel, where the plain multiply form measured 0.6-1.0 % faster (its code schedules better)
template <class S, class R>
__device__ __forceinline__ R cdot_s(int l, R x, R y, R z) {
  if constexpr (std::is_same<S, float>::value) return R(CX(l)) * x + R(CY(l)) * y + R(CZ(l)) * z;
  else return cdot<R>(l, x, y, z);
}
// a += c_la v for the nonzero components c_la of c_l (a = (ax, ay, az))
template <class R>
__device__ __forceinline__ void cadd(int l, R v, R& ax, R& ay, R& az) {
  if (CX(l) != 0) ax = CX(l) > 0 ? ax + v : ax - v;
  if (CY(l) != 0) ay = CY(l) > 0 ? ay + v : ay - v;
  if (CZ(l) != 0) az = CZ(l) > 0 ? az + v : az - v;
}

// class of direction l: 0 rest, 1 axis, 2 diagonal (= |c_l|^2)
__host__ __device__ constexpr int CLS(int l) { return CSQ(l); }

// Sums of the deviations: drho = sum_l df_l (rho = rho0 + drho), j = sum_l c_l df_l (the reference
// equilibrium carries no momentum), ascending l.
template <class R>
__device__ __forceinline__ void density_momentum(const R (&f)[Q], R& rho, R& jx, R& jy, R& jz) {
  rho = f[0];
#pragma unroll
  for (int l = 1; l < Q; ++l) rho = rho + f[l];
  // ascending l over the nonzero components
  jx = f[1] - f[2]; jx = jx + f[7]; jx = jx - f[8]; jx = jx + f[9]; jx = jx - f[10];
  jx = jx + f[11]; jx = jx - f[12]; jx = jx + f[13]; jx = jx - f[14];
  jy = f[3] - f[4]; jy = jy + f[7]; jy = jy - f[8]; jy = jy - f[9]; jy = jy + f[10];
  jy = jy + f[15]; jy = jy - f[16]; jy = jy + f[17]; jy = jy - f[18];
  jz = f[5] - f[6]; jz = jz + f[11]; jz = jz - f[12]; jz = jz - f[13]; jz = jz + f[14];
  jz = jz + f[15]; jz = jz - f[16]; jz = jz - f[17]; jz = jz + f[18];
}

// Thermal wall rule (anti-bounce-back with the even part of g^eq at the wall temperature T_w):
// g_l = -g*_{opp(l)} + 2 w_l [rho_p T_w + 4.5 (lam T_w - rho_p T_w / 3)(|c_l|^2 - 1)], rho_p = the wall
// node's density at the colliding step = sum of its own post-collision f. In deviations:
// dg_l = -dg*_{opp(l)} + 2 (wall_even_l - gbase_l).
template <class R>
__device__ __forceinline__ R wall_even_dev(int l, R drho_p, R rho0, R T0, R Tw, R lam) {
  const R dP = drho_p * Tw + rho0 * (Tw - T0);   // rho_p T_w - rho0 T0
  return WT<R>(l) * (dP + R(4.5) * (lam * (Tw - T0) - dP / R(3)) * R(CSQ(l) - 1));
}

template <class S>
__device__ __forceinline__ float loc_ref(const S* __restrict__ buf, unsigned e, int ls, unsigned N);

template <class S, class R>
__device__ __forceinline__ void g_wall_fix(R (&g)[Q], const S* __restrict__ fin, int N, int own,
                                           int z, int nz, R rho0, R T0, R Td, R Tu, R lam) {
  if (z != 0 && z != nz - 1) return;
  R dp;
  if constexpr (IsLoc<S>::v) {
    // the stored post-collision f of the wall node, each with its node's reference added back
    dp = Store<S>::ld(fin + own) + loc_ref<S>(fin, (unsigned)own, 0, (unsigned)N);
#pragma unroll
    for (int m = 1; m < Q; ++m)
      dp = dp + (Store<S>::ld(fin + (size_t)m * N + own) +
                 loc_ref<S>(fin, (unsigned)m * (unsigned)N + (unsigned)own, m, (unsigned)N));
  } else {
    dp = Store<S>::ld(fin + own);
#pragma unroll
    for (int m = 1; m < Q; ++m) dp = dp + Store<S>::ld(fin + (size_t)m * N + own);
  }
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    if (CZ(l) > 0 && z == 0) g[l] = -g[l] + R(2) * wall_even_dev<R>(l, dp, rho0, T0, Td, lam);
    if (CZ(l) < 0 && z == nz - 1) g[l] = -g[l] + R(2) * wall_even_dev<R>(l, dp, rho0, T0, Tu, lam);
  }
}

// MODE_STEP: one time step. MODE_MOMENTS: the moments of the current state (fields and/or the
// diagnostics partials), no collision. MODE_STEP_DIAG: one time step that also forms the
// diagnostics partials of the state it reads (the Nu sample of that state, fused).
enum { MODE_STEP = 0, MODE_MOMENTS = 1, MODE_STEP_DIAG = 2 };

// Reciprocal and exponential per compute precision: IEEE for FP64 (parity form); the rounded
// MUFU-based forms for FP32 (relative error ~1e-7, far below the FP32 form's tolerance).
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ float fexp(float x) { return __expf(x); }

// e^t - 1 for the deviation form of psi (FP32 forms): the Taylor polynomial to t^6 for
// |t| <= 1/8 (truncation below 1e-9 of the result), the exponential minus one beyond, where the
// result is at least 0.11 in magnitude and the subtraction costs nothing beyond the rounding of
// the exponential itself.
__device__ __forceinline__ float expm1_dev(float t) {
  const float p = t * (1.0f + t * (0.5f + t * (1.0f / 6.0f + t * (1.0f / 24.0f + t * (1.0f / 120.0f +
                                                                                 t * (1.0f / 720.0f))))));
  return fabsf(t) <= 0.125f ? p : __expf(t) - 1.0f;
}

// van der Waals-type pseudopotential psi = rho sqrt(k (a - b T_v/(1 - b rho))), k = 2/(-G)
__device__ __forceinline__ double psi_vdw(double rho, const KPar<double>& p) {
  return rho * sqrt(p.vk * (p.va - p.vb * p.vT / (1.0 - p.vb * rho)));
}
__device__ __forceinline__ float psi_vdw(float rho, const KPar<float>& p) {
  return rho * sqrtf(p.vk * (p.va - p.vb * p.vT / (1.0f - p.vb * rho)));
}

template <int BY> struct Geo {
  static constexpr int NT = BX * BY;
  static constexpr int RX = BX + 4, RY = BY + 4, RXY = RX * RY;   // radius-2 ring (psi)
  static constexpr int HX = BX + 2, HY = BY + 2, HXY = HX * HY;   // radius-1 ring (rho, j, u)
  static constexpr int TXY = BX * BY;
  static constexpr int MAXM = (RXY + NT - 1) / NT;
  static constexpr int NHALO = 2 * BX + 2 * BY;
  // Depth D of the psi, rho/j and f-cache rings. With D = 4 the C stage of one z-iteration and
  // the M stage of the next need no barrier between them (the next M stage refills the slot of
  // plane p-3, last read before this iteration's barrier); with D = 3 a trailing barrier ends
  // each iteration. Measured: 4 for the 16-bit forms, 3 for FP32 (smaller shared-memory window,
  // larger L1 share) and FP64 (shared memory).
  template <class S> static constexpr int depth() { return sizeof(S) == 2 ? 4 : 3; }
  // R units: psi[D][RXY], rj[D][5][HXY] (rho, 1/rho, jx, jy, jz), u[3][3][HXY], F[2][3][TXY];
  // then either the pulled-f cache of the tile, fc[D][Q][TXY] in storage units S, or (STG) the
  // stage of the collision's pulled f and g, stg[2][Q][TXY] in 4-byte words.
  // fields of each F-ring plane: F, and for FP64 also the psi sums A (the adjoint's fields)
  template <class S> static constexpr int fslots() { return sizeof(S) == 8 ? 6 : 3; }
  template <class S> static constexpr size_t r_count() {
    return (size_t)(depth<S>() * (RXY + 5 * HXY) + 9 * HXY + 2 * fslots<S>() * TXY);
  }
  // local-reference storage: the g references of the collision's sources, a radius-1 window of
  // the tile in 4 planes, one 4-byte word (b1, b2) per node (tiles of 8 rows and more: at 4 rows
  // the window's registers would spill)
  template <class S> static constexpr bool gwin() { return IsLoc<S>::v && BY >= 8; }
  // the f cache of the tile's pulled populations (16-bit forms); FP64 takes its ring's moments and
  // psi from the per-node pre-pass and pulls the collision's f directly
  template <class S> static constexpr bool fcache() { return !std::is_same<S, double>::value; }
  template <class S> static constexpr size_t gwin_bytes() { return gwin<S>() ? sizeof(uint32_t) * 4 * HXY : 0; }
  template <class S, class R, bool STG> static constexpr size_t smem_bytes() {
    return sizeof(R) * r_count<S>() +
           (STG ? sizeof(uint32_t) * (size_t)(2 * Q * TXY)
                : (fcache<S>() ? sizeof(S) * (size_t)(depth<S>() * Q * TXY) : 0)) +
           gwin_bytes<S>();
  }
};

__device__ __forceinline__ int slot3(int p) { return (p + 6) % 3; }
__device__ __forceinline__ int slot2(int p) { return (p + 6) & 1; }
// slot of plane p in a ring of depth D (3 or 4); p >= -6
template <int D> __device__ __forceinline__ int ring(int p) { return D == 4 ? ((p + 8) & 3) : (p + 6) % 3; }

template <class R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class R> __device__ __forceinline__ R warp_min(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Pull the raw stored deviations of node (col[1], row[1], pz): v_l = buf_l(x - c_l); across a wall
// (only when WALL) the bounce-back source buf_{opp(l)}(x). Element offsets are 32-bit (19 N < 2^32).
template <class S, bool WALL>
__device__ __forceinline__ void pull_raw(S (&v)[Q], const S* __restrict__ buf, unsigned N, int pz,
                                         int nz, unsigned plane, const int (&col)[3], const int (&row)[3]) {
  const unsigned zb = (unsigned)pz * plane;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const int cz = CZ(l);
    if (WALL && ((cz > 0 && pz == 0) || (cz < 0 && pz == nz - 1))) {
      v[l] = buf[(unsigned)OPP(l) * N + zb + (unsigned)(row[1] + col[1])];
    } else {
      v[l] = buf[(unsigned)l * N + (zb - (unsigned)(cz * (int)plane)) +
                 (unsigned)(row[1 - CY(l)] + col[1 - CX(l)])];
    }
  }
}

// The same with the node given by its element index in the plane pz and the steps to its x/y
// neighbours (dy[0] to y-1, dy[1] to y+1, dx likewise; the periodic wrap folded in); loff as in
// KArgs. Used by the 16-bit forms' ring pulls (measured faster there; slower for FP32).
template <class S, bool WALL>
__device__ __forceinline__ void pull_rel(S (&v)[Q], const S* __restrict__ buf, unsigned N, int pz, int nz,
                                         unsigned own, const int (&dy)[2], const int (&dx)[2],
                                         const unsigned (&loff)[19]) {
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const int cz = CZ(l);
    if (WALL && ((cz > 0 && pz == 0) || (cz < 0 && pz == nz - 1))) {
      v[l] = buf[(unsigned)OPP(l) * N + own];
    } else {
      unsigned e = own + loff[l];
      if (CY(l) > 0) e += (unsigned)dy[0];
      if (CY(l) < 0) e += (unsigned)dy[1];
      if (CX(l) > 0) e += (unsigned)dx[0];
      if (CX(l) < 0) e += (unsigned)dx[1];
      v[l] = buf[e];
    }
  }
}

// Element index of the pulled source of population l at node (col[1], row[1], z) (through a wall,
// when WALL, the bounce-back source opp(l) of the node itself).
template <bool WALL>
__device__ __forceinline__ unsigned pull_index(int l, unsigned N, int z, int nz, unsigned plane,
                                               const int (&col)[3], const int (&row)[3]) {
  const int cz = CZ(l);
  if (WALL && ((cz > 0 && z == 0) || (cz < 0 && z == nz - 1)))
    return (unsigned)OPP(l) * N + (unsigned)z * plane + (unsigned)(row[1] + col[1]);
  return (unsigned)l * N + ((unsigned)z * plane - (unsigned)(cz * (int)plane)) +
         (unsigned)(row[1 - CY(l)] + col[1 - CX(l)]);
}

// Local-reference storage: the reference to add to slot ls (0..18) read at element index e. For
// ls >= 1 the reference of the slot's class (|c|^2 = 1 or 2) at the node of e, stored in slot
// Q - 1 + |c|^2; for the rest slot the node's a0 = 12 (a1 - a2) (its index e is the node's).
template <class S>
__device__ __forceinline__ float loc_ref(const S* __restrict__ buf, unsigned e, int ls, unsigned N) {
  if (ls == 0)
    return 12.0f * (Store<S>::ld(buf + e + (unsigned)Q * N) - Store<S>::ld(buf + e + (unsigned)(Q + 1) * N));
  return Store<S>::ld(buf + e + (unsigned)(Q - 1 + CSQ(ls) - ls) * N);
}

// The references of the populations that pull_rel reads (same addressing).
template <class S, bool WALL>
__device__ __forceinline__ void pull_rel_ref(float (&r)[Q], const S* __restrict__ buf, unsigned N, int pz,
                                             int nz, unsigned own, const int (&dy)[2], const int (&dx)[2],
                                             const unsigned (&loff)[19]) {
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const int cz = CZ(l);
    if (WALL && ((cz > 0 && pz == 0) || (cz < 0 && pz == nz - 1))) {
      r[l] = loc_ref<S>(buf, (unsigned)OPP(l) * N + own, OPP(l), N);
    } else {
      unsigned e = own + loff[l];
      if (CY(l) > 0) e += (unsigned)dy[0];
      if (CY(l) < 0) e += (unsigned)dy[1];
      if (CX(l) > 0) e += (unsigned)dx[0];
      if (CX(l) < 0) e += (unsigned)dx[1];
      r[l] = loc_ref<S>(buf, e, l, N);
    }
  }
}

// The references of the populations that pull_raw reads (same addressing).
template <class S, bool WALL>
__device__ __forceinline__ void pull_raw_ref(float (&r)[Q], const S* __restrict__ buf, unsigned N, int pz,
                                             int nz, unsigned plane, const int (&col)[3], const int (&row)[3]) {
  const unsigned zb = (unsigned)pz * plane;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const int cz = CZ(l);
    if (WALL && ((cz > 0 && pz == 0) || (cz < 0 && pz == nz - 1))) {
      r[l] = loc_ref<S>(buf, (unsigned)OPP(l) * N + zb + (unsigned)(row[1] + col[1]), OPP(l), N);
    } else {
      r[l] = loc_ref<S>(buf, (unsigned)l * N + (zb - (unsigned)(cz * (int)plane)) +
                                 (unsigned)(row[1 - CY(l)] + col[1 - CX(l)]), l, N);
    }
  }
}

// The references of the 19 pulled g of node cw (index in the radius-1 window) from the window
// of 4-byte words (b1 low, b2 high half) of planes z-1..z+1; across a wall (only when WALL) the
// node's own word (bounce-back source). Same values as pull_raw_ref on the g lattice.
template <bool WALL>
__device__ __forceinline__ void win_ref(float (&r)[Q], const uint32_t* __restrict__ win, int z, int nz, int cw,
                                        int hx, int hxy) {
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const int cz = CZ(l);
    const bool through = WALL && ((cz > 0 && z == 0) || (cz < 0 && z == nz - 1));
    const uint32_t w = through ? win[ring<4>(z) * hxy + cw]
                               : win[ring<4>(z - cz) * hxy + cw - CY(l) * hx - CX(l)];
    const float b1 = __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
    const float b2 = __half2float(__ushort_as_half((unsigned short)(w >> 16)));
    r[l] = l == 0 ? 12.0f * (b1 - b2) : (CSQ(l) == 1 ? b1 : b2);
  }
}

// The two stored references of a node (rounded to the storage format) from its moment deviations:
// f: a1 = w1 drho, a2 = w2 (4.5 dE - 0.5 drho); g: b1 = w1 dE, b2 = w2 (4.5 lam dT - 0.5 dE).
template <class S>
__device__ __forceinline__ void loc_refs_of(float drho, float dE, float dT, float lam, float& a1, float& a2,
                                            float& b1, float& b2) {
  a1 = Store<S>::rt(WT<float>(1) * drho);
  a2 = Store<S>::rt(WT<float>(7) * (4.5f * dE - 0.5f * drho));
  b1 = Store<S>::rt(WT<float>(1) * dE);
  b2 = Store<S>::rt(WT<float>(7) * (4.5f * lam * dT - 0.5f * dE));
}

// 4-byte asynchronous global -> shared copy (cp.async, cached in L1 and L2); a 16-bit element is
// copied as the aligned 4-byte word that contains it (population arrays carry 64 bytes of padding).
template <class S>
__device__ __forceinline__ void stage_word(uint32_t* dst, const S* base, unsigned e) {
  const S* src = base + (sizeof(S) == 2 ? (e & ~1u) : e);
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void stage_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <class S> __device__ __forceinline__ S word_elem(uint32_t w, unsigned e);
template <> __device__ __forceinline__ float word_elem<float>(uint32_t w, unsigned) { return __uint_as_float(w); }
template <> __device__ __forceinline__ __half word_elem<__half>(uint32_t w, unsigned e) {
  return __ushort_as_half((unsigned short)((e & 1u) ? (w >> 16) : (w & 0xffffu)));
}
template <> __device__ __forceinline__ __nv_bfloat16 word_elem<__nv_bfloat16>(uint32_t w, unsigned e) {
  return __ushort_as_bfloat16((unsigned short)((e & 1u) ? (w >> 16) : (w & 0xffffu)));
}
template <> __device__ __forceinline__ double word_elem<double>(uint32_t, unsigned) { return 0.0; }

template <class S, class R>
__device__ __forceinline__ R cvt(S v) { return Store<S>::ld(&v); }
template <> __device__ __forceinline__ double cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float cvt<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float cvt<__half, float>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float cvt<half_loc, float>(half_loc v) { return __half2float(v.h); }

// Resident CTAs per SM the register allocation must allow: 512 threads per SM for the FP32 and
// 16-bit forms (128 registers a thread); the FP64 form is limited by its shared memory anyway.
// Moments mode: per-warp partials of the last two collided planes (slot z & 1), combined over
// the warps by warp 0 after the next barrier (static shared memory of the moments kernels only).
template <class R, int BY> __device__ __forceinline__ R (*moments_red())[7][BY] {
  __shared__ R red[2][7][BY];
  return red;
}
// lanes 0..6 of warp 0 combine partial k of plane z over the BY warps, in warp order, in FP64
template <class R, int BY>
__device__ __forceinline__ void moments_combine(const KArgs& a, int z, int tile, int tid) {
  R (*red)[7][BY] = moments_red<R, BY>();
  if (tid < NPART) {
    double acc = 0.0;
    if (tid < 7) {
      const R* v = red[z & 1][tid];
      acc = double(v[0]);
      for (int w = 1; w < BY; ++w)
        acc = (tid == 4 || tid == 5) ? fmin(acc, double(v[w])) : acc + double(v[w]);
    }
    a.part[((size_t)z * a.ntiles + tile) * NPART + tid] = acc;
  }
}

template <class S, int BY> struct MinBlocks { static constexpr int v = 512 / (BX * BY) > 0 ? 512 / (BX * BY) : 1; };
template <int BY> struct MinBlocks<double, BY> { static constexpr int v = 2; };

template <class S, int BY, int MODE, int VAR = 0>
__global__ void __launch_bounds__(BX * BY, MinBlocks<S, BY>::v)
lb_fused_kernel(const KArgs a) {
  constexpr int FORCE = (VAR & VAR_GUO) ? FORCE_GUO : FORCE_SHIFT;
  constexpr bool VDW = (VAR & VAR_VDW) != 0;
  constexpr bool COLLIDE = MODE != MODE_MOMENTS, DIAG = MODE != MODE_STEP;
  // The FP32-compute forms keep psi of the paper's pseudopotential as its deviation
  // dpsi = psi - psi(rho0) = psi(rho0) (e^t - 1), t = 1/rho0 - 1/rho = drho/(rho rho0): the force
  // sum of Eq. (9) (sum_l W_l c_l = 0, so dpsi may replace psi there) then adds small numbers,
  // and its FP32 rounding is relative to the density variation, not to psi ~ 0.6.
  constexpr bool DPSI = sizeof(typename Store<S>::R) == 4 && !VDW;
  // Code shape for the register budget: the paper's forcing takes the unswitched staging loops
  // and 64-bit store addressing (fewer instructions); the Guo-forcing variants, short of
  // registers, keep the compact forms (measured: 36-48 against 20 bytes of spills otherwise).
  constexpr bool LEAN = FORCE != FORCE_GUO;
  using R = typename Store<S>::R;
  using GE = Geo<BY>;
  constexpr int NT = GE::NT, RX = GE::RX, RXY = GE::RXY, HX = GE::HX, HXY = GE::HXY;
  constexpr int TXY = GE::TXY, MAXM = GE::MAXM, NHALO = GE::NHALO;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool STG = std::is_same<S, float>::value && TLBM_STAGE;
  constexpr int D = GE::template depth<S>();
  constexpr bool PRE = std::is_same<S, double>::value;   // FP64: ring fields from lb_fields_kernel
  R* psi_s = reinterpret_cast<R*>(smem_raw);  // [D][RXY]
  R* rj_s = psi_s + D * RXY;                  // [D][5][HXY]  rho, 1/rho, jx, jy, jz
  R* u_s = rj_s + D * 5 * HXY;                // [3][3][HXY]  physical velocity
  constexpr int NFS = GE::template fslots<S>();
  R* F_s = u_s + 9 * HXY;                     // [2][NFS][TXY]  force (and FP64: psi sums A) on the tile
  // FP32 stages the collision's pulled f and g asynchronously; FP64 and the 16-bit forms keep
  // the f cache (measured faster for them) and pull g directly.
  S* fc_s = reinterpret_cast<S*>(F_s + 2 * NFS * TXY);                 // [D][Q][TXY] (not STG)
  uint32_t* stg_s = reinterpret_cast<uint32_t*>(F_s + 2 * NFS * TXY);  // [2][Q][TXY] (STG)
  constexpr bool GWIN = GE::template gwin<S>();
  uint32_t* gw_s = reinterpret_cast<uint32_t*>(fc_s + D * Q * TXY);   // [4][HXY] g references (GWIN)
  constexpr int NGW = (HXY + NT - 1) / NT;                               // window nodes per thread

  const S* __restrict__ fin = static_cast<const S*>(a.fin);
  const S* __restrict__ gin = static_cast<const S*>(a.gin);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const unsigned plane = (unsigned)a.plane, N = (unsigned)a.N;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
  const int tile = blockIdx.x;
  const int x0 = (tile % a.tiles_x) * BX, y0 = (tile / a.tiles_x) * BY;
  const int z0 = blockIdx.y * a.zc;
  const int z1 = min(z0 + a.zc, nz);

  const KPar<R>& kp = kpar<R>(a);
  const R rho0 = kp.rho0, E0 = kp.E0, T0 = kp.T0;
  const R G = kp.G, gz = kp.g_z, lam = kp.lam, Td = kp.T_d, Tu = kp.T_u;

  // Ring nodes of the M stage owned by this thread: wrapped columns/rows of x-1, x, x+1 (FP32,
  // FP64), or the node's in-plane index and its steps to the x/y neighbours (16-bit forms).
  constexpr bool REL = sizeof(S) == 2;
  int mcol[MAXM][3], mrow[MAXM][3];
  int mown[MAXM], mdy[MAXM][2], mdx[MAXM][2];
  short mh[MAXM], mt[MAXM];   // index in the radius-1 ring / in the tile, or -1
#pragma unroll
  for (int i = 0; i < MAXM; ++i) {
    const int k = tid + i * NT;
    const int rx = k % RX, ry = k / RX;
    const int gx = x0 + rx - 2, gy = y0 + ry - 2;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      mcol[i][j] = wrapi(gx - 1 + j, nx);
      mrow[i][j] = wrapi(gy - 1 + j, ny) * nx;
    }
    mown[i] = mrow[i][1] + mcol[i][1];
    mdx[i][0] = mcol[i][0] - mcol[i][1]; mdx[i][1] = mcol[i][2] - mcol[i][1];
    mdy[i][0] = mrow[i][0] - mrow[i][1]; mdy[i][1] = mrow[i][2] - mrow[i][1];
    mh[i] = (k < RXY && rx >= 1 && rx <= BX + 2 && ry >= 1 && ry <= BY + 2) ? (short)((ry - 1) * HX + (rx - 1)) : (short)-1;
    mt[i] = (k < RXY && rx >= 2 && rx < BX + 2 && ry >= 2 && ry < BY + 2) ? (short)((ry - 2) * BX + (rx - 2)) : (short)-1;
  }
  int ccol[3], crow[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    ccol[j] = wrapi(x0 + tx - 1 + j, nx);
    crow[j] = wrapi(y0 + ty - 1 + j, ny) * nx;
  }
  const bool cvalid = (x0 + tx < nx) && (y0 + ty < ny);

  // U-stage halo node of this thread (radius-1 ring minus corners), if any.
  int hx = 0, hy = 0;
  const bool has_halo = tid < NHALO;
  if (tid < BX) { hx = tid; hy = -1; }
  else if (tid < 2 * BX) { hx = tid - BX; hy = BY; }
  else if (tid < 2 * BX + BY) { hx = -1; hy = tid - 2 * BX; }
  else { hx = BX; hy = tid - 2 * BX - BY; }

  for (int p = z0 - 2; p <= z1 + 1; ++p) {
    const int z = p - 2;            // plane collided by this iteration's C stage
    const bool cplane = (z >= z0 && z < z1);
    const bool wallz = (z == 0 || z == nz - 1);
    // local-reference storage: load the g references (b1, b2) of plane p-1 on the radius-1 window
    // now; they are stored to the window behind the M stage (the collisions of planes p-2..p pull
    // from it). Slot ring<4>(p-1) was last read by the collision of plane p-5, which every warp
    // finished before the previous iteration's barrier.
    unsigned short gwv[GWIN ? 2 * NGW : 1];
    const int gq = p - 1;
    const bool gload = GWIN && gq >= 0 && gq < nz && gq >= z0 - 1 && gq <= z1;
    if constexpr (GWIN) {
      if (gload) {
        const unsigned short* gb = reinterpret_cast<const unsigned short*>(gin);
#pragma unroll
        for (int i = 0; i < NGW; ++i) {
          const int k = tid + i * NT;
          if (k < HXY) {
            const int gx = wrapi(x0 + k % HX - 1, nx), gy = wrapi(y0 + k / HX - 1, ny);
            const unsigned e = (unsigned)gq * plane + (unsigned)(gy * nx + gx);
            gwv[2 * i] = __ldg(gb + e + (unsigned)Q * N);
            gwv[2 * i + 1] = __ldg(gb + e + (unsigned)(Q + 1) * N);
          }
        }
      }
    }
    if constexpr (STG) {
      // start the copies of the collision's pulled f and g; they complete behind M and U
      if (cplane && cvalid) {
        const int t = ty * BX + tx;
        if constexpr (LEAN) {
          // unswitched on the wall test: the interior loop carries no bounce-back selects
          if (wallz) {
#pragma unroll
            for (int l = 0; l < Q; ++l) {
              const unsigned e = pull_index<true>(l, N, z, nz, plane, ccol, crow);
              stage_word<S>(stg_s + l * TXY + t, fin, e);
              stage_word<S>(stg_s + (Q + l) * TXY + t, gin, e);
            }
          } else {
#pragma unroll
            for (int l = 0; l < Q; ++l) {
              const unsigned e = pull_index<false>(l, N, z, nz, plane, ccol, crow);
              stage_word<S>(stg_s + l * TXY + t, fin, e);
              stage_word<S>(stg_s + (Q + l) * TXY + t, gin, e);
            }
          }
        } else {
#pragma unroll
          for (int l = 0; l < Q; ++l) {
            const unsigned e = wallz ? pull_index<true>(l, N, z, nz, plane, ccol, crow)
                                     : pull_index<false>(l, N, z, nz, plane, ccol, crow);
            stage_word<S>(stg_s + l * TXY + t, fin, e);
            stage_word<S>(stg_s + (Q + l) * TXY + t, gin, e);
          }
        }
      }
      stage_commit();
    }
    // ---------------- M: psi, rho, j of plane p on the radius-2 ring; f of the tile cached ----------------
    {
      const int pz = mirror_z(p, nz);
      const bool wallp = (pz == 0 || pz == nz - 1);
      const bool real = (p == pz);
      const int s3 = ring<D>(p);
      const unsigned zb = (unsigned)pz * plane;
#pragma unroll
      for (int i = 0; i < MAXM; ++i) {
        const int k = tid + i * NT;
        if constexpr (PRE) {
          // FP64: the ring node's moments and psi from the per-node pre-pass
          if (k < RXY) {
            const double* pr = a.pre + (zb + (unsigned)mown[i]);
            psi_s[s3 * RXY + k] = pr[5 * (size_t)N];
            if (mh[i] >= 0) {
              R* rj = rj_s + s3 * 5 * HXY + mh[i];
              rj[0] = pr[0]; rj[HXY] = pr[(size_t)N]; rj[2 * HXY] = pr[2 * (size_t)N];
              rj[3 * HXY] = pr[3 * (size_t)N]; rj[4 * HXY] = pr[4 * (size_t)N];
            }
          }
          continue;
        }
        if (k < RXY) {
          S fr[Q];
          if constexpr (REL) {
            if (wallp) pull_rel<S, true>(fr, fin, N, pz, nz, zb + (unsigned)mown[i], mdy[i], mdx[i], a.loff);
            else pull_rel<S, false>(fr, fin, N, pz, nz, zb + (unsigned)mown[i], mdy[i], mdx[i], a.loff);
          } else {
            if (wallp) pull_raw<S, true>(fr, fin, N, pz, nz, plane, mcol[i], mrow[i]);
            else pull_raw<S, false>(fr, fin, N, pz, nz, plane, mcol[i], mrow[i]);
          }
          R f[Q];
#pragma unroll
          for (int l = 0; l < Q; ++l) f[l] = cvt<S, R>(fr[l]);
          if constexpr (IsLoc<S>::v) {
            float rf[Q];
            if (wallp) pull_rel_ref<S, true>(rf, fin, N, pz, nz, zb + (unsigned)mown[i], mdy[i], mdx[i], a.loff);
            else pull_rel_ref<S, false>(rf, fin, N, pz, nz, zb + (unsigned)mown[i], mdy[i], mdx[i], a.loff);
#pragma unroll
            for (int l = 0; l < Q; ++l) f[l] = f[l] + rf[l];
          }
          R drho, jx, jy, jz;
          density_momentum<R>(f, drho, jx, jy, jz);
          const R rho = rho0 + drho;
          const R inv = rcp(rho);
          if constexpr (VDW) psi_s[s3 * RXY + k] = psi_vdw(rho, kp);
          else if constexpr (DPSI) psi_s[s3 * RXY + k] = kp.psi0 * expm1_dev(drho * inv * kp.irho0);
          else psi_s[s3 * RXY + k] = fexp(-inv);
          if (mh[i] >= 0) {
            R* rj = rj_s + s3 * 5 * HXY + mh[i];
            rj[0] = rho; rj[HXY] = inv; rj[2 * HXY] = jx; rj[3 * HXY] = jy; rj[4 * HXY] = jz;
          }
          if (!STG && real && mt[i] >= 0) {
            S* fc = fc_s + s3 * Q * TXY + mt[i];
#pragma unroll
            for (int l = 0; l < Q; ++l) fc[l * TXY] = fr[l];
          }
        }
      }
    }
    if constexpr (GWIN) {
      if (gload) {
        uint32_t* w = gw_s + ring<4>(gq) * HXY;
#pragma unroll
        for (int i = 0; i < NGW; ++i) {
          const int k = tid + i * NT;
          if (k < HXY) w[k] = (uint32_t)gwv[2 * i] | ((uint32_t)gwv[2 * i + 1] << 16);
        }
      }
    }
    __syncthreads();
    if constexpr (DIAG) {
      // the partials of the plane collided in the previous iteration are complete
      if (a.part != nullptr && p - 3 >= z0 && p - 3 < z1) moments_combine<R, BY>(a, p - 3, tile, tid);
    }
    // ---------------- U: F and u = (j + F/2)/rho of plane q = p-1 ----------------
    {
      const int q = p - 1;
      if (q >= z0 - 1 && q <= z1 && q >= 0 && q < nz) {
        const R* pm = psi_s + ring<D>(q - 1) * RXY;
        const R* p0 = psi_s + ring<D>(q) * RXY;
        const R* pp = psi_s + ring<D>(q + 1) * RXY;
        const R* rj = rj_s + ring<D>(q) * 5 * HXY;
        R* us = u_s + slot3(q) * 3 * HXY;
        R* Fs = F_s + slot2(q) * NFS * TXY;
        auto unode = [&](int xr, int yr, bool on_tile) {
          const int c = (yr + 2) * RX + (xr + 2);
          R ax = R(0), ay = R(0), az = R(0);
#pragma unroll
          for (int l = 1; l < Q; ++l) {
            const R* pl = CZ(l) == 0 ? p0 : (CZ(l) > 0 ? pp : pm);
            const R nb = pl[c + CY(l) * RX + CX(l)];
            if (CX(l) != 0) ax = ax + (FW<R>(l) * R(CX(l))) * nb;
            if (CY(l) != 0) ay = ay + (FW<R>(l) * R(CY(l))) * nb;
            if (CZ(l) != 0) az = az + (FW<R>(l) * R(CZ(l))) * nb;
          }
          const int h = (yr + 1) * HX + (xr + 1);
          const R rho = rj[h], inv = rj[HXY + h];
          const R mg = -G * (DPSI ? kp.psi0 + p0[c] : p0[c]);
          const R Fx = mg * ax, Fy = mg * ay, Fz = mg * az + rho * gz;
          us[h] = (rj[2 * HXY + h] + R(0.5) * Fx) * inv;
          us[HXY + h] = (rj[3 * HXY + h] + R(0.5) * Fy) * inv;
          us[2 * HXY + h] = (rj[4 * HXY + h] + R(0.5) * Fz) * inv;
          if (on_tile) {
            const int t = yr * BX + xr;
            Fs[t] = Fx; Fs[TXY + t] = Fy; Fs[2 * TXY + t] = Fz;
            if constexpr (NFS == 6) { Fs[3 * TXY + t] = ax; Fs[4 * TXY + t] = ay; Fs[5 * TXY + t] = az; }
          }
        };
        unode(tx, ty, true);
        if (has_halo) unode(hx, hy, false);
      }
    }
    // No barrier before C: of what this U stage writes, C reads u of plane p-1 and F only at the
    // thread's own node (written by itself); its ring reads are of planes finished one barrier ago.
    // ---------------- C: collide plane z = p-2 ----------------
    // moments-mode partials of this thread's node in the compute precision (neutral values when
    // it has none); warp sums in the compute precision, then FP64 across warps, tiles and planes
    R d_conv = R(0), d_T = R(0), d_rho = R(0), d_E = R(0);
    R d_mr = R(sizeof(R) == 8 ? 1e300 : 3.0e38), d_mT = d_mr;
    bool d_bad = false;
    if (cplane && cvalid) {
      const unsigned own = (unsigned)z * plane + (unsigned)(crow[1] + ccol[1]);
      const int t = ty * BX + tx;
      R g[Q], f[Q];
      if constexpr (STG) {
        stage_wait();                  // this thread's copies of the collision's f and g
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          const unsigned e = wallz ? pull_index<true>(l, N, z, nz, plane, ccol, crow)
                                   : pull_index<false>(l, N, z, nz, plane, ccol, crow);
          f[l] = cvt<S, R>(word_elem<S>(stg_s[l * TXY + t], e));
          g[l] = cvt<S, R>(word_elem<S>(stg_s[(Q + l) * TXY + t], e));
        }
      } else {
        S gr[Q];
        if (wallz) pull_raw<S, true>(gr, gin, N, z, nz, plane, ccol, crow);
        else pull_raw<S, false>(gr, gin, N, z, nz, plane, ccol, crow);
#pragma unroll
        for (int l = 0; l < Q; ++l) g[l] = cvt<S, R>(gr[l]);
        if constexpr (PRE) {
          // FP64 keeps no f cache: the collision pulls its f like its g
          S fr[Q];
          if (wallz) pull_raw<S, true>(fr, fin, N, z, nz, plane, ccol, crow);
          else pull_raw<S, false>(fr, fin, N, z, nz, plane, ccol, crow);
#pragma unroll
          for (int l = 0; l < Q; ++l) f[l] = cvt<S, R>(fr[l]);
        } else {
          const S* fc = fc_s + ring<D>(z) * Q * TXY + t;
#pragma unroll
          for (int l = 0; l < Q; ++l) f[l] = cvt<S, R>(fc[l * TXY]);
        }
        if constexpr (IsLoc<S>::v) {
          // the references of the sources: f's from its lattice, g's from the window (GWIN)
          float rf[Q], rg[Q];
          const int cw = (ty + 1) * HX + (tx + 1);
          if (wallz) {
            pull_raw_ref<S, true>(rf, fin, N, z, nz, plane, ccol, crow);
            if constexpr (GWIN) win_ref<true>(rg, gw_s, z, nz, cw, HX, HXY);
            else pull_raw_ref<S, true>(rg, gin, N, z, nz, plane, ccol, crow);
          } else {
            pull_raw_ref<S, false>(rf, fin, N, z, nz, plane, ccol, crow);
            if constexpr (GWIN) win_ref<false>(rg, gw_s, z, nz, cw, HX, HXY);
            else pull_raw_ref<S, false>(rg, gin, N, z, nz, plane, ccol, crow);
          }
#pragma unroll
          for (int l = 0; l < Q; ++l) { f[l] = f[l] + rf[l]; g[l] = g[l] + rg[l]; }
        }
      }
      if (wallz) g_wall_fix<S, R>(g, fin, (int)N, (int)own, z, nz, rho0, T0, Td, Tu, lam);
      const int cc = (ty + 1) * HX + (tx + 1);
      const R* rjc = rj_s + ring<D>(z) * 5 * HXY + cc;
      const R rho = rjc[0], inv = rjc[HXY];
      const R jx = rjc[2 * HXY], jy = rjc[3 * HXY], jz = rjc[4 * HXY];
      const R drho = rho - rho0;
      R dE = g[0];
#pragma unroll
      for (int l = 1; l < Q; ++l) dE = dE + g[l];
      const R E = E0 + dE;          // rho T
      const R T = E * inv;
      const R* u0 = u_s + slot3(z) * 3 * HXY;
      const R ux = u0[cc], uy = u0[HXY + cc], uz = u0[2 * HXY + cc];
      if constexpr (DIAG) {
        // U = c_v T + int_0^rho P_NI/s^2 ds: (G/4) e^{-2/rho}, or -T_v ln(1 - b rho) - a rho (vdW)
        if constexpr (sizeof(R) == 8) {
          const double U = a.c_v * T + (VDW ? -kp.vT * log(1.0 - kp.vb * rho) - kp.va * rho
                                            : 0.25 * a.G * exp(-2.0 / rho));
          d_conv = rho * U * uz;
        } else {
          // FP32-compute forms: the node's term in float (relative error ~1e-7, far inside these
          // forms' tolerance; on GB300 FP64 instructions cost more than the step itself)
          const R U = R(a.c_v) * T + (VDW ? -kp.vT * logf(R(1) - kp.vb * rho) - kp.va * rho
                                          : R(0.25) * G * fexp(R(-2) * inv));
          d_conv = rho * U * uz;
        }
        d_T = T; d_rho = rho; d_E = E; d_mr = rho; d_mT = T;
        d_bad = !(isfinite(rho) && isfinite(T) && isfinite(ux) && isfinite(uy) && isfinite(uz));
      }
      if constexpr (COLLIDE) {
        const R* Fs = F_s + slot2(z) * NFS * TXY;
        const R Fx = Fs[t], Fy = Fs[TXY + t], Fz = Fs[2 * TXY + t];
        const R* um = u_s + slot3(z - 1) * 3 * HXY;
        const R* up = u_s + slot3(z + 1) * 3 * HXY;
        const R uzm = (z - 1 >= 0) ? um[2 * HXY + cc] : -uz;
        const R uzp = (z + 1 < nz) ? up[2 * HXY + cc] : -uz;
        R D = R(0.5) * (u0[cc + 1] - u0[cc - 1]);
        D = D + R(0.5) * (u0[HXY + cc + HX] - u0[HXY + cc - HX]);
        D = D + R(0.5) * (uzp - uzm);
        // Output element of population l of this node: with LEAN from the node's own address, l N
        // in 64-bit arithmetic (one multiply-add per store), else the 32-bit element index.
        constexpr bool P64 = LEAN;
        S* __restrict__ fo = static_cast<S*>(a.fout) + (P64 ? own : 0u);
        S* __restrict__ go = static_cast<S*>(a.gout) + (P64 ? own : 0u);
        const size_t NS = N;
        auto sidx = [&](int l) -> size_t {
          if constexpr (P64) return (size_t)l * NS;
          else return (size_t)((unsigned)l * N + own);
        };
        // Local-reference storage: this node's references (of its moments at this step) go to the
        // two reference slots, and every population slot stores its value minus the reference of
        // its class (the readers add them back)
        R lrf[3] = {R(0), R(0), R(0)}, lrg[3] = {R(0), R(0), R(0)};
        if constexpr (IsLoc<S>::v) {
          float a1, a2, b1, b2;
          loc_refs_of<S>(drho, dE, T - T0, lam, a1, a2, b1, b2);
          lrf[0] = 12.0f * (a1 - a2); lrf[1] = a1; lrf[2] = a2;
          lrg[0] = 12.0f * (b1 - b2); lrg[1] = b1; lrg[2] = b2;
          Store<S>::st(fo + sidx(Q), a1); Store<S>::st(fo + sidx(Q + 1), a2);
          Store<S>::st(go + sidx(Q), b1); Store<S>::st(go + sidx(Q + 1), b2);
        }
        auto putf = [&](int l, R v) {
          if constexpr (IsLoc<S>::v) v = v - lrf[CSQ(l)];
          Store<S>::st(fo + sidx(l), v);
        };
        auto putg = [&](int l, R v) {
          if constexpr (IsLoc<S>::v) v = v - lrg[CSQ(l)];
          Store<S>::st(go + sidx(l), v);
        };
        // f: BGK towards f^eq(rho, u', T), u' = (j + tau F)/rho. f^eq - fbase per class:
        // w [drho - 1.5 rho v.v + 4.5 (|c|^2-1)(dE - drho/3) + 3 rho c.v + 4.5 rho (c.v)^2]
        // (rho (T - 1/3) - rho0 (T0 - 1/3) = dE - drho/3 since rho T = E).
        // Guo forcing (variant): v = u and the source (1 - om/2) w [3 (c - u).F + 9 (c.u)(c.F)],
        // split like f^eq into the part even in c (9 (c.u)(c.F) - 3 u.F) and the odd part 3 c.F.
        {
          const R tau = kp.tau_nu, om = kp.omega_nu, om1 = R(1) - om;
          const R vx = (FORCE == FORCE_GUO) ? ux : (jx + tau * Fx) * inv;
          const R vy = (FORCE == FORCE_GUO) ? uy : (jy + tau * Fy) * inv;
          const R vz = (FORCE == FORCE_GUO) ? uz : (jz + tau * Fz) * inv;
          if constexpr (NFS == 6) {
            // FP64: the fields of the state read, for the discrete adjoint's reverse sweep
            if (a.adj_m != nullptr) {
              double* m = a.adj_m + own;
              const size_t n = (size_t)N;
              m[MF_RHO * n] = rho; m[MF_T * n] = T;
              m[MF_PSI * n] = psi_s[ring<GE::template depth<S>()>(z) * RXY + (ty + 2) * RX + (tx + 2)];
              m[MF_UX * n] = ux; m[MF_UY * n] = uy; m[MF_UZ * n] = uz;
              m[MF_VX * n] = vx; m[MF_VY * n] = vy; m[MF_VZ * n] = vz; m[MF_D * n] = D;
              m[MF_AX * n] = Fs[3 * TXY + t]; m[MF_AY * n] = Fs[4 * TXY + t]; m[MF_AZ * n] = Fs[5 * TXY + t];
            }
          }
          const R ks = R(1) - R(0.5) * om;
          const R uF = ux * Fx + uy * Fy + uz * Fz;
          const R a0 = drho - R(1.5) * rho * (vx * vx + vy * vy + vz * vz);
          const R th = R(4.5) * (dE - drho * R(1.0 / 3.0));
          const R A[3] = {a0 - th, a0, a0 + th};
          const R r3 = R(3) * rho, r45 = R(4.5) * rho;
          if constexpr (FORCE == FORCE_GUO) {
#pragma unroll
            for (int l = 0; l < Q; ++l) {
              if (l != 0 && (l & 1) == 0) continue;     // handled with its odd partner
              const R cv = cdot_s<S, R>(l, vx, vy, vz);
              const R w = WT<R>(l) * om;
              const R sym = A[CLS(l)] + r45 * cv * cv;
              const R asym = r3 * cv;
              const R cF = cdot_s<S, R>(l, Fx, Fy, Fz);
              const R ws = WT<R>(l) * ks;
              const R ssym = ws * (R(9) * cv * cF - R(3) * uF), sasym = ws * (R(3) * cF);
              putf(l, om1 * f[l] + w * (sym + asym) + (ssym + sasym));
              if (l != 0)
                putf(OPP(l),
                             om1 * f[OPP(l)] + w * (sym - asym) + (ssym - sasym));
            }
          } else {
            // the relaxation weights folded into the per-class coefficients: the even part
            // w om (A + 4.5 rho (c.v)^2) = wA + q (c.v)^2, the odd part w om 3 rho (c.v) = s (c.v)
            const R o0 = WT<R>(0) * om, o1 = WT<R>(1) * om, o2 = WT<R>(7) * om;
            const R wA[3] = {o0 * A[0], o1 * A[1], o2 * A[2]};
            const R q[3] = {R(0), o1 * r45, o2 * r45}, sc[3] = {R(0), o1 * r3, o2 * r3};
            putf(0, om1 * f[0] + wA[0]);
#pragma unroll
            for (int l = 1; l < Q; l += 2) {
              const R cv = cdot_s<S, R>(l, vx, vy, vz);
              const R ev = q[CLS(l)] * (cv * cv) + wA[CLS(l)];
              const R od = sc[CLS(l)] * cv;
              putf(l, om1 * f[l] + (ev + od));
              putf(OPP(l), om1 * f[OPP(l)] + (ev - od));
            }
          }
        }
        // g: BGK towards g^eq(rho, T, u) plus the counter term w_l S, S = -rho T div(u)/c_v.
        // g^eq - gbase per class: w [dE - 1.5 E u.u + 4.5 (|c|^2-1)(lam (T-T0) - dE/3) + 3 E c.u
        // + 4.5 E (c.u)^2], T - T0 = (dE - T0 drho)/rho.
        {
          const R omk = kp.omega_kappa, omk1 = R(1) - omk;
          const R Ssrc = -E * D * kp.inv_cv;
          const R b0 = dE - R(1.5) * E * (ux * ux + uy * uy + uz * uz);
          const R tg = R(4.5) * (lam * ((dE - T0 * drho) * inv) - dE * R(1.0 / 3.0));
          const R B[3] = {b0 - tg, b0, b0 + tg};
          const R e3 = R(3) * E, e45 = R(4.5) * E;
          // per class: the even part w omk (B + 4.5 E (c.u)^2) + w S = P + q (c.u)^2, the odd
          // part w omk 3 E (c.u) = s (c.u)
          const R k0 = WT<R>(0) * omk, k1 = WT<R>(1) * omk, k2 = WT<R>(7) * omk;
          const R P[3] = {k0 * B[0] + WT<R>(0) * Ssrc, k1 * B[1] + WT<R>(1) * Ssrc, k2 * B[2] + WT<R>(7) * Ssrc};
          const R q[3] = {R(0), k1 * e45, k2 * e45}, sc[3] = {R(0), k1 * e3, k2 * e3};
          putg(0, omk1 * g[0] + P[0]);
#pragma unroll
          for (int l = 1; l < Q; l += 2) {
            const R cu = cdot_s<S, R>(l, ux, uy, uz);
            const R ev = q[CLS(l)] * (cu * cu) + P[CLS(l)];
            const R od = sc[CLS(l)] * cu;
            putg(l, omk1 * g[l] + (ev + od));
            putg(OPP(l), omk1 * g[OPP(l)] + (ev - od));
          }
        }
      } else {
        if (a.rho_out) a.rho_out[own] = double(rho);
        if (a.ux_out) a.ux_out[own] = double(ux);
        if (a.uy_out) a.uy_out[own] = double(uy);
        if (a.uz_out) a.uz_out[own] = double(uz);
        if (a.T_out) a.T_out[own] = double(T);
      }
    }
    if constexpr (DIAG) {
      if (a.part != nullptr && cplane) {
        // warp-shuffle reduction of the plane partials in the compute precision (the
        // non-finite count by ballot); combined over the warps in FP64 after the next barrier
        R (*red)[7][BY] = moments_red<R, BY>();
        d_conv = warp_sum(d_conv); d_T = warp_sum(d_T); d_rho = warp_sum(d_rho);
        d_E = warp_sum(d_E); d_mr = warp_min(d_mr); d_mT = warp_min(d_mT);
        const int nbad = __popc(__ballot_sync(0xffffffffu, d_bad));
        if (tx == 0) {
          R* r = &red[z & 1][0][ty];
          r[0] = d_conv; r[BY] = d_T; r[2 * BY] = d_rho; r[3 * BY] = d_E; r[4 * BY] = d_mr;
          r[5 * BY] = d_mT; r[6 * BY] = R(nbad);
        }
      }
    }
    // With D = 3 the next M stage refills the psi slot that this U stage read and the rho/j
    // (and f-cache) slot that this C stage read.
    if (D == 3) __syncthreads();
  }
  if constexpr (DIAG) {
    // the chunk's last plane
    if (a.part != nullptr) {
      __syncthreads();
      moments_combine<R, BY>(a, z1 - 1, tile, tid);
    }
  }
}

// ---------------------------------------------------------------------------------------
// FP64 form, before each step-kernel launch: rho, 1/rho, j (Eq. (8)) and psi of every node of the
// state a.fin, once per node, into a.pre ([6][N]). On GB300 the FP64 step is bound by its FP64
// instructions; its M stage would otherwise form these for the radius-2 ring of every tile, 1.69
// times per node. Same pulls (with the walls' bounce-back sources) and the same operations in the
// same order as the M stage, so the step's results are unchanged bit for bit. One node per thread.
// ---------------------------------------------------------------------------------------
template <bool VDW>
__global__ void __launch_bounds__(256) lb_fields_kernel(const KArgs a) {
  const double* __restrict__ fin = static_cast<const double*>(a.fin);
  const unsigned N = (unsigned)a.N, plane = (unsigned)a.plane;
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x = (int)(idx % (unsigned)nx), y = (int)((idx / (unsigned)nx) % (unsigned)ny);
  const int z = (int)(idx / plane);
  int col[3], row[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    col[j] = wrapi(x - 1 + j, nx);
    row[j] = wrapi(y - 1 + j, ny) * nx;
  }
  double f[Q];
  if (z == 0 || z == nz - 1) pull_raw<double, true>(f, fin, N, z, nz, plane, col, row);
  else pull_raw<double, false>(f, fin, N, z, nz, plane, col, row);
  double drho, jx, jy, jz;
  density_momentum<double>(f, drho, jx, jy, jz);
  const KPar<double>& kp = a.pd;
  const double rho = kp.rho0 + drho;
  const double inv = rcp(rho);
  double* o = a.pre + idx;
  o[0] = rho;
  o[(size_t)N] = inv;
  o[2 * (size_t)N] = jx;
  o[3 * (size_t)N] = jy;
  o[4 * (size_t)N] = jz;
  o[5 * (size_t)N] = VDW ? psi_vdw(rho, kp) : fexp(-inv);
}

// ---------------------------------------------------------------------------------------
// Initial state: buffer B0 whose pull gives f = f^eq(rho, 0, T), g = g^eq(rho, T, 0).
// B0_l(y) = eq_l(y + c_l) where y + c_l is inside, else the wall slot that the bounce-back of
// opp(l) at y pulls: f-slot = f^eq_{opp(l)}(y); g-slot chosen so that the thermal wall rule
// returns g^eq_{opp(l)}(y) with rho_p = the sum of the stored f-slots of y. Stored as deviations.
// ---------------------------------------------------------------------------------------
template <class S>
__global__ void lb_init_kernel(const KArgs a, const double* __restrict__ rho_in,
                               const double* __restrict__ T_in) {
  using R = typename Store<S>::R;
  S* __restrict__ fo = static_cast<S*>(a.fout);
  S* __restrict__ go = static_cast<S*>(a.gout);
  const int nx = a.nx, ny = a.ny, nz = a.nz, plane = a.plane, N = a.N;
  const R rho0 = R(a.rho0), E0 = R(a.E0), T0 = R(a.T0), lam = R(a.lam);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
    const int x = idx % nx, y = (idx / nx) % ny, z = idx / plane;
    // local-reference storage: the node's references from its own initial fields
    R lrf[3] = {R(0), R(0), R(0)}, lrg[3] = {R(0), R(0), R(0)};
    if constexpr (IsLoc<S>::v) {
      const R r = R(rho_in[idx]), T = R(T_in[idx]);
      float a1, a2, b1, b2;
      loc_refs_of<S>(r - rho0, r * T - E0, T - T0, lam, a1, a2, b1, b2);
      lrf[0] = 12.0f * (a1 - a2); lrf[1] = a1; lrf[2] = a2;
      lrg[0] = 12.0f * (b1 - b2); lrg[1] = b1; lrg[2] = b2;
      Store<S>::st(fo + (size_t)Q * N + idx, a1); Store<S>::st(fo + (size_t)(Q + 1) * N + idx, a2);
      Store<S>::st(go + (size_t)Q * N + idx, b1); Store<S>::st(go + (size_t)(Q + 1) * N + idx, b2);
    }
    R fb[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const int zn = z + CZ(l);
      const bool wall = (zn < 0 || zn >= nz);
      const int src = wall ? idx : zn * plane + wrapi(y + CY(l), ny) * nx + wrapi(x + CX(l), nx);
      const int le = wall ? OPP(l) : l;   // direction whose equilibrium this slot carries
      const R r = R(rho_in[src]), T = R(T_in[src]);
      const R drho = r - rho0, dE = r * T - E0;
      const R df = WT<R>(le) * (drho + R(4.5) * (dE - drho / R(3)) * R(CSQ(le) - 1));
      Store<S>::st(fo + (size_t)l * N + idx, df - lrf[CSQ(l)]);
      fb[l] = Store<S>::rt(df - lrf[CSQ(l)]) + lrf[CSQ(l)];   // the value a later pull returns
    }
    R dp = fb[0];                 // rho_p - rho0 as the step kernel forms it
#pragma unroll
    for (int m = 1; m < Q; ++m) dp = dp + fb[m];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const int zn = z + CZ(l);
      const bool wall = (zn < 0 || zn >= nz);
      const int src = wall ? idx : zn * plane + wrapi(y + CY(l), ny) * nx + wrapi(x + CX(l), nx);
      const int le = wall ? OPP(l) : l;
      const R r = R(rho_in[src]), T = R(T_in[src]);
      const R dE = r * T - E0;
      R dg = WT<R>(le) * (dE + R(4.5) * (lam * (T - T0) - dE / R(3)) * R(CSQ(le) - 1));
      if (wall) {
        const R Tw = (CZ(le) > 0) ? R(a.T_d) : R(a.T_u);
        dg = R(2) * wall_even_dev<R>(le, dp, rho0, T0, Tw, lam) - dg;
      }
      Store<S>::st(go + (size_t)l * N + idx, dg - lrg[CSQ(l)]);
    }
  }
}

// Given pre-collision state (float64 [19][N] each, the layout of lb_pops_kernel's output) stored
// as the post-collision buffer B whose pull with the wall rules returns it: B_l(y) = f_l(y + c_l)
// where y + c_l is inside; otherwise B_l(y) is the bounce-back source of f_{opp(l)} at y, so
// B_l(y) = f_{opp(l)}(y), and for g the thermal wall rule is inverted:
// B^g_l(y) = 2 (even part of g^eq_{opp(l)} at T_w, rho_p) - g_{opp(l)}(y) with rho_p the sum of the
// stored f-slots of y (the density the step forms at the wall node). Stored as deviations.
template <class S>
__global__ void lb_setpops_kernel(const KArgs a, const double* __restrict__ f_in,
                                  const double* __restrict__ g_in) {
  using R = typename Store<S>::R;
  S* __restrict__ fo = static_cast<S*>(a.fout);
  S* __restrict__ go = static_cast<S*>(a.gout);
  const int nx = a.nx, ny = a.ny, nz = a.nz, plane = a.plane, N = a.N;
  const R rho0 = R(a.rho0), T0 = R(a.T0), lam = R(a.lam);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
    const int x = idx % nx, y = (idx / nx) % ny, z = idx / plane;
    // local-reference storage: the node's references from the moments of the given state at it
    R lrf[3] = {R(0), R(0), R(0)}, lrg[3] = {R(0), R(0), R(0)};
    if constexpr (IsLoc<S>::v) {
      double rr = 0.0, EE = 0.0;
      for (int l = 0; l < Q; ++l) { rr += f_in[(size_t)l * N + idx]; EE += g_in[(size_t)l * N + idx]; }
      float a1, a2, b1, b2;
      loc_refs_of<S>(float(rr - a.rho0), float(EE - a.E0), float(EE / rr - a.T0), lam, a1, a2, b1, b2);
      lrf[0] = 12.0f * (a1 - a2); lrf[1] = a1; lrf[2] = a2;
      lrg[0] = 12.0f * (b1 - b2); lrg[1] = b1; lrg[2] = b2;
      Store<S>::st(fo + (size_t)Q * N + idx, a1); Store<S>::st(fo + (size_t)(Q + 1) * N + idx, a2);
      Store<S>::st(go + (size_t)Q * N + idx, b1); Store<S>::st(go + (size_t)(Q + 1) * N + idx, b2);
    }
    R fb[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const int zn = z + CZ(l);
      const bool wall = (zn < 0 || zn >= nz);
      const int src = wall ? idx : zn * plane + wrapi(y + CY(l), ny) * nx + wrapi(x + CX(l), nx);
      const int le = wall ? OPP(l) : l;   // population of the given state this slot returns
      const R df = R(f_in[(size_t)le * N + src] - a.fbase[CSQ(le)]);
      Store<S>::st(fo + (size_t)l * N + idx, df - lrf[CSQ(l)]);
      fb[l] = Store<S>::rt(df - lrf[CSQ(l)]) + lrf[CSQ(l)];
    }
    R dp = fb[0];
#pragma unroll
    for (int m = 1; m < Q; ++m) dp = dp + fb[m];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const int zn = z + CZ(l);
      const bool wall = (zn < 0 || zn >= nz);
      const int src = wall ? idx : zn * plane + wrapi(y + CY(l), ny) * nx + wrapi(x + CX(l), nx);
      const int le = wall ? OPP(l) : l;
      R dg = R(g_in[(size_t)le * N + src] - a.gbase[CSQ(le)]);
      if (wall) {
        const R Tw = (CZ(le) > 0) ? R(a.T_d) : R(a.T_u);
        dg = R(2) * wall_even_dev<R>(le, dp, rho0, T0, Tw, lam) - dg;
      }
      Store<S>::st(go + (size_t)l * N + idx, dg - lrg[CSQ(l)]);
    }
  }
}

// Pre-collision state (pull + wall rules) exported as float64 [19][N].
template <class S>
__global__ void lb_pops_kernel(const KArgs a, double* __restrict__ fo, double* __restrict__ go) {
  using R = typename Store<S>::R;
  const S* __restrict__ fin = static_cast<const S*>(a.fin);
  const S* __restrict__ gin = static_cast<const S*>(a.gin);
  const int nx = a.nx, ny = a.ny, nz = a.nz, plane = a.plane, N = a.N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
    const int x = idx % nx, y = (idx / nx) % ny, z = idx / plane;
    int col[3], row[3];
    for (int j = 0; j < 3; ++j) { col[j] = wrapi(x - 1 + j, nx); row[j] = wrapi(y - 1 + j, ny) * nx; }
    R f[Q], g[Q];
    pull<S, R>(f, fin, N, z, nz, plane, col, row);
    pull<S, R>(g, gin, N, z, nz, plane, col, row);
    g_wall_fix<S, R>(g, fin, N, idx, z, nz, R(a.rho0), R(a.T0), R(a.T_d), R(a.T_u), R(a.lam));
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      if (fo) fo[(size_t)l * N + idx] = double(f[l]) + a.fbase[CSQ(l)];
      if (go) go[(size_t)l * N + idx] = double(g[l]) + a.gbase[CSQ(l)];
    }
  }
}

}  // namespace tlbm
