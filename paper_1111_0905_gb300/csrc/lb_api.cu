// lb_api.cu -- C ABI of the thermal pseudopotential D3Q19 lattice Boltzmann step (include/lb.h).
//
// Host side: parameter validation, device memory of the context (two ping-pong population
// lattices per distribution, diagnostics scratch), launch geometry, checkpoints. Every step of
// the method runs in the kernels of lb_kernels.cuh; this file only marshals and orders them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_launch.cuh"
#include "lb_ctx.h"

namespace tlbm {

// Diagnostics finalisation, in two launches so that the FP64 sums (1/64 of the FP32 rate on
// GB300) spread over the SMs. Every sum has a fixed assignment of terms to threads and a fixed
// combination tree, so the result does not depend on timing. out layout:
// [0, nz) Nu(z) of Eq. (4) (normalised by kappa (T_d - T_u)/nz); nz: Nu_mean; nz+1: min rho;
// nz+2: min T; nz+3: non-finite count; nz+4: sum rho; nz+5: sum rho T;
// [nz+8, 8nz+8) per-plane sums over the tiles, [7][nz] (scratch).
// If acc != null, acc[0] += Nu_mean, acc[1] += 1.

// 1) one CTA (128 threads) per plane: the plane's 7 partials summed (minima taken) over the tiles
__global__ void __launch_bounds__(128) lb_diag_planes(const double* __restrict__ part, int nz, int ntiles,
                                                      double* __restrict__ out) {
  __shared__ double red[7][4];
  const int z = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[7] = {0.0, 0.0, 0.0, 0.0, 1e300, 1e300, 0.0};
  for (int k = threadIdx.x; k < ntiles; k += blockDim.x) {
    const double* p = part + ((size_t)z * ntiles + k) * NPART;
#pragma unroll
    for (int q = 0; q < 7; ++q) v[q] = (q == 4 || q == 5) ? fmin(v[q], p[q]) : v[q] + p[q];
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) v[q] = (q == 4 || q == 5) ? warp_min(v[q]) : warp_sum(v[q]);
  if (lane == 0)
    for (int q = 0; q < 7; ++q) red[q][warp] = v[q];
  __syncthreads();
  if (threadIdx.x < 7) {
    const int q = threadIdx.x;
    double a = red[q][0];
    for (int w = 1; w < 4; ++w) a = (q == 4 || q == 5) ? fmin(a, red[q][w]) : a + red[q][w];
    out[nz + 8 + (size_t)q * nz + z] = a;
  }
}

// 2) one CTA: Nu(z) from the plane sums with the wall ghosts, Nu_mean and the global values
__global__ void __launch_bounds__(1024) lb_diag_finalize(int nz, int nxy, double kappa, double T_d,
                                                         double T_u, double* __restrict__ out,
                                                         double* __restrict__ acc) {
  __shared__ double red[6][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const double* ps = out + nz + 8;   // [7][nz]: conv, T, rho, rho T, min rho, min T, non-finite
  const double* sT = ps + nz;
  const double norm = kappa * (T_d - T_u) / nz;
  double s = 0.0, sr = 0.0, sE = 0.0, mr = 1e300, mT = 1e300, bad = 0.0;
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    const double Tp = (z + 1 < nz) ? sT[z + 1] : 2.0 * T_u * nxy - sT[nz - 1];
    const double Tm = (z - 1 >= 0) ? sT[z - 1] : 2.0 * T_d * nxy - sT[0];
    const double flux = (ps[z] - kappa * 0.5 * (Tp - Tm)) / nxy;
    const double nu = flux / norm;
    out[z] = nu;
    s += nu;
    sr += ps[2 * nz + z]; sE += ps[3 * nz + z];
    mr = fmin(mr, ps[4 * nz + z]); mT = fmin(mT, ps[5 * nz + z]); bad += ps[6 * nz + z];
  }
  s = warp_sum(s); sr = warp_sum(sr); sE = warp_sum(sE); bad = warp_sum(bad);
  mr = warp_min(mr); mT = warp_min(mT);
  if (lane == 0) {
    red[0][warp] = s; red[1][warp] = sr; red[2][warp] = sE; red[3][warp] = bad;
    red[4][warp] = mr; red[5][warp] = mT;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a[6] = {red[0][0], red[1][0], red[2][0], red[3][0], red[4][0], red[5][0]};
    for (int w = 1; w < nwarp; ++w) {
      for (int k = 0; k < 4; ++k) a[k] += red[k][w];
      a[4] = fmin(a[4], red[4][w]); a[5] = fmin(a[5], red[5][w]);
    }
    const double mean = a[0] / nz;
    out[nz] = mean; out[nz + 1] = a[4]; out[nz + 2] = a[5]; out[nz + 3] = a[3];
    out[nz + 4] = a[1]; out[nz + 5] = a[2];
    if (acc) { acc[0] += mean; acc[1] += 1.0; }
  }
}


// Validation of initial fields: per-block count of bad entries and sums (fixed order).
__global__ void lb_validate_kernel(const double* __restrict__ rho, const double* __restrict__ T,
                                   int N, double rho_lim, double* __restrict__ out /* [gridDim.x][3] */) {
  __shared__ double sh[3][256];
  double bad = 0.0, sr = 0.0, sT = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double r = rho[i], t = T[i];
    if (!(r > 0.0) || !(r < rho_lim) || !(t > 0.0) || !isfinite(r) || !isfinite(t)) bad += 1.0;
    sr += r; sT += t;
  }
  sh[0][threadIdx.x] = bad; sh[1][threadIdx.x] = sr; sh[2][threadIdx.x] = sT;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) out[blockIdx.x * 3 + k] = sh[k][0];
}

}  // namespace tlbm

using namespace tlbm;

namespace {

const char* kNullCtxMsg = "null context";


const PrecOps* ops_for(int prec) {
  switch (prec) {
    case LB_FP64: return &kOpsF64;
    case LB_FP32: return &kOpsF32;
    case LB_BF16_DEV: return &kOpsBF16;
    case LB_FP16_DEV: return &kOpsF16;
    case LB_FP16_LOC: return &kOpsF16Loc;
    default: return nullptr;
  }
}

}  // namespace

KArgs make_args(const lb_ctx* c) {
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.fin = c->f[c->cur]; a.gin = c->g[c->cur];
  a.fout = c->f[1 - c->cur]; a.gout = c->g[1 - c->cur];
  a.pre = c->pre;
  a.nx = c->p.nx; a.ny = c->p.ny; a.nz = c->p.nz; a.plane = c->plane; a.N = c->N;
  a.tiles_x = c->tiles_x; a.ntiles = c->ntiles; a.zc = c->zc;
  a.forcing = c->p.forcing; a.psi_kind = c->p.psi_kind;
  a.tau_nu = c->p.tau_nu; a.omega_nu = 1.0 / c->p.tau_nu; a.omega_kappa = 1.0 / c->p.tau_kappa;
  a.G = c->p.G; a.g_z = c->p.g_z; a.lam = c->lam; a.inv_cv = 1.0 / c->p.c_v; a.c_v = c->p.c_v;
  a.kappa = c->p.kappa; a.T_d = c->p.T_d; a.T_u = c->p.T_u;
  a.rho0 = c->rho0; a.T0 = c->T0; a.E0 = c->rho0 * c->T0;
  const double vk = c->p.psi_kind == PSI_VDW ? 2.0 / (-c->p.G) : 0.0;
  a.pd = {a.tau_nu, a.omega_nu, a.omega_kappa, a.G, a.g_z, a.lam, a.inv_cv, a.T_d, a.T_u,
          a.rho0, a.T0, a.E0, c->p.vdw_a, c->p.vdw_b, c->p.vdw_T, vk};
  a.pf = {(float)a.tau_nu, (float)a.omega_nu, (float)a.omega_kappa, (float)a.G, (float)a.g_z,
          (float)a.lam, (float)a.inv_cv, (float)a.T_d, (float)a.T_u, (float)a.rho0, (float)a.T0,
          (float)a.E0, (float)c->p.vdw_a, (float)c->p.vdw_b, (float)c->p.vdw_T, (float)vk};
  a.pd.psi0 = std::exp(-1.0 / c->rho0);
  a.pd.irho0 = 1.0 / c->rho0;
  a.pf.psi0 = (float)a.pd.psi0;
  a.pf.irho0 = (float)a.pd.irho0;
  // reference equilibria per class (rest, axis, diagonal): f^eq(rho0, 0, T0), g^eq(rho0, T0, 0)
  const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
  for (int k = 0; k < 3; ++k) {
    a.fbase[k] = w[k] * c->rho0 * (1.0 + 4.5 * (c->T0 - 1.0 / 3.0) * (k - 1));
    a.gbase[k] = w[k] * (a.E0 + 4.5 * (c->lam * c->T0 - a.E0 / 3.0) * (k - 1));
  }
  for (int l = 0; l < Q; ++l)
    a.loff[l] = (unsigned)((long long)l * c->N - (long long)CZ(l) * c->plane);
  return a;
}

dim3 fused_grid(const lb_ctx* c) { return dim3(c->ntiles, c->nchunks); }

namespace {

void free_all(lb_ctx* c) {
  if (!c) return;
  for (int k = 0; k < 2; ++k) { cudaFree(c->f[k]); cudaFree(c->g[k]); }
  cudaFree(c->part); cudaFree(c->diag); cudaFree(c->nu_acc);
  cudaFree(c->fields); cudaFree(c->pops); cudaFree(c->pre);
}

}  // namespace

// Moments pass into the plane partials, then Nu(z) and the global health values into diag;
// Nu_mean is added to acc[0] (and 1 to acc[1]) when acc is not null.
int finalize_diag(lb_ctx* c, double* acc) {
  lb_diag_planes<<<c->p.nz, 128, 0, c->stream>>>(c->part, c->p.nz, c->ntiles, c->diag);
  lb_diag_finalize<<<1, 1024, 0, c->stream>>>(c->p.nz, c->p.nx * c->p.ny, c->p.kappa, c->p.T_d,
                                               c->p.T_u, c->diag, acc);
  LB_CU(c, cudaGetLastError());
  return LB_OK;
}

int run_diag_acc(lb_ctx* c, double* acc) {
  KArgs a = make_args(c);
  a.part = c->part;
  LB_CU(c, c->ops->fused(a, MODE_MOMENTS, c->by, fused_grid(c), c->stream));
  return finalize_diag(c, acc);
}

int run_diag(lb_ctx* c, bool accumulate) { return run_diag_acc(c, accumulate ? c->nu_acc : nullptr); }

int flush_sample(lb_ctx* c) {
  if (!c->sample_pending) return LB_OK;
  c->sample_pending = false;
  return run_diag(c, true);
}

namespace {

uint64_t fnv1a(uint64_t h, const unsigned char* p, size_t n) {
  for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
  return h;
}

struct CkptHeader {
  char magic[8];
  int32_t version, precision;
  int32_t nx, ny, nz, pad;
  int64_t step;
  double rho0, T0;
  double nu_acc[2];
  lb_params params;
  uint64_t checksum;
};

}  // namespace

extern "C" {

const char* lb_strerror(int code) {
  switch (code) {
    case LB_OK: return "ok";
    case LB_EINVAL: return "invalid argument";
    case LB_ENOMEM: return "out of memory";
    case LB_ECUDA: return "CUDA error";
    case LB_ENONPHYS: return "non-physical state (rho <= 0, T <= 0 or NaN)";
    case LB_EIO: return "checkpoint I/O error";
    case LB_EUNSUP: return "unsupported";
    default: return "unknown error";
  }
}

const char* lb_last_error(const lb_ctx* c) { return c ? c->err.c_str() : kNullCtxMsg; }

long long lb_step_count(const lb_ctx* c) { return c ? c->step : -1; }

int lb_launch_info(lb_ctx* c, int* out) {
  if (!c || !out) return LB_EINVAL;
  int k[4] = {0, 0, 0, 0};
  LB_CU(c, c->ops->info(c->by, variant_of(c->p.forcing, c->p.psi_kind), k));
  const dim3 grid = fused_grid(c);
  out[0] = (int)grid.x; out[1] = (int)grid.y;
  out[2] = k[0]; out[3] = k[1]; out[4] = k[2]; out[5] = k[3];
  return LB_OK;
}

int lb_init(const lb_params* params, const double* rho_init, const double* T_init,
            int init_on_device, void* cuda_stream, lb_ctx** out) {
  if (!out) return LB_EINVAL;
  *out = nullptr;
  if (!params || !rho_init || !T_init) return LB_EINVAL;
  const lb_params& p = *params;
  if (p.nx < 1 || p.ny < 1 || p.nz < 1) return LB_EINVAL;
  const long long N = (long long)p.nx * p.ny * p.nz;
  if (N >= (1ll << 31) || (long long)p.nz * 2 >= (1ll << 30)) return LB_EINVAL;
  if (!(p.tau_nu > 0.5) || !(p.tau_kappa > 0.5) || !(p.kappa > 0.0) || !(p.c_v > 0.0)) return LB_EINVAL;
  if (!std::isfinite(p.G) || !std::isfinite(p.g_z) || !(p.T_d > 0.0) || !(p.T_u > 0.0)) return LB_EINVAL;
  const PrecOps* ops = ops_for(p.precision);
  if (!ops) return LB_EINVAL;
  // default tile height 32 x 8 (measured best on the 128^3/256^3 cells for every form)
  int by = p.tile_y != 0 ? p.tile_y : 8;
  if (by != 4 && by != 8 && by != 16) return LB_EINVAL;
  if (!ops->tile_ok(by)) return LB_EINVAL;
  if ((long long)ops->slots * N >= (1ll << 32)) return LB_EINVAL;   // 32-bit population offsets
  if (p.z_chunk < 0 || p.nu_every < 0 || p.check_every < 0) return LB_EINVAL;
  if (p.forcing != FORCE_SHIFT && p.forcing != FORCE_GUO) return LB_EINVAL;
  if (p.psi_kind != PSI_EXP && p.psi_kind != PSI_VDW) return LB_EINVAL;
  // van der Waals psi: real for rho < (1 - b T_v/a)/b; every initial density must be below it
  double rho_lim = INFINITY;
  if (p.psi_kind == PSI_VDW) {
    if (!(p.G < 0.0) || !(p.vdw_a > 0.0) || !(p.vdw_b > 0.0) || !(p.vdw_T > 0.0) ||
        !(p.vdw_b * p.vdw_T < p.vdw_a))
      return LB_EINVAL;
    rho_lim = (1.0 - p.vdw_b * p.vdw_T / p.vdw_a) / p.vdw_b;
  }

  lb_ctx* c = new (std::nothrow) lb_ctx();
  if (!c) return LB_ENOMEM;
  c->p = p;
  c->ops = ops;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->N = (int)N;
  c->plane = p.nx * p.ny;
  c->by = by;
  c->lam = p.kappa / (p.c_v * (p.tau_kappa - 0.5));
  c->tiles_x = (p.nx + BX - 1) / BX;
  c->tiles_y = (p.ny + by - 1) / by;
  c->ntiles = c->tiles_x * c->tiles_y;

  auto bail = [&](int code) { free_all(c); delete c; return code; };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(LB_ECUDA);
  if (ops->prepare() != cudaSuccess) return bail(LB_ECUDA);
  if (p.z_chunk > 0) {
    c->zc = p.z_chunk < p.nz ? p.z_chunk : p.nz;
  } else {
    // Planes per chunk: each chunk adds 4 prologue planes (M stages without collisions) and the
    // CTAs run in waves of (resident CTAs per SM) x SMs, so a launch takes about
    // ceil(CTAs / slots) * (zc + 4) plane-steps. Take the chunk count (zc from 8 to 128, or nz)
    // that minimises it; ties go to the larger chunk.
    int k[4] = {0, 0, 0, 0}, sms = 0;
    if (ops->info(by, variant_of(p.forcing, p.psi_kind), k) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
      return bail(LB_ECUDA);
    const long long slots = (long long)(k[2] > 0 ? k[2] : 1) * (sms > 0 ? sms : 1);
    c->zc = p.nz;
    long long best = -1;
    for (int nch = 1; nch <= p.nz; ++nch) {
      const int zc = (p.nz + nch - 1) / nch;
      if (zc > 128) continue;
      if (zc < 8 && nch > 1) break;
      const long long ctas = (long long)c->ntiles * ((p.nz + zc - 1) / zc);
      const long long cost = ((ctas + slots - 1) / slots) * (zc + 4);
      if (best < 0 || cost < best) { best = cost; c->zc = zc; }
    }
  }
  c->nchunks = (p.nz + c->zc - 1) / c->zc;

  // validate the initial fields and form their means on the device (fixed-order sums)
  const double* d_rho = rho_init;
  const double* d_T = T_init;
  double* staging = nullptr;
  const size_t fbytes = (size_t)N * sizeof(double);
  if (!init_on_device) {
    if (cudaMalloc(&staging, 2 * fbytes) != cudaSuccess) return bail(LB_ENOMEM);
    if (cudaMemcpyAsync(staging, rho_init, fbytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(staging + N, T_init, fbytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
      cudaFree(staging);
      return bail(LB_ECUDA);
    }
    d_rho = staging;
    d_T = staging + N;
  }
  const int vblocks = 256;
  double* vpart = nullptr;
  if (cudaMalloc(&vpart, vblocks * 3 * sizeof(double)) != cudaSuccess) { cudaFree(staging); return bail(LB_ENOMEM); }
  lb_validate_kernel<<<vblocks, 256, 0, c->stream>>>(d_rho, d_T, c->N, rho_lim, vpart);
  std::vector<double> hv(vblocks * 3);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(hv.data(), vpart, hv.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaFree(vpart); cudaFree(staging);
    return bail(LB_ECUDA);
  }
  cudaFree(vpart);
  double bad = 0, sr = 0, sT = 0;
  for (int b = 0; b < vblocks; ++b) { bad += hv[b * 3]; sr += hv[b * 3 + 1]; sT += hv[b * 3 + 2]; }
  if (bad > 0) { cudaFree(staging); return bail(LB_EINVAL); }
  c->rho0 = p.rho0 > 0 ? p.rho0 : sr / N;
  c->T0 = p.T0 > 0 ? p.T0 : sT / N;

  // 64 bytes of padding: a word-wide copy of a 16-bit element (stage_word) reads the 4-byte word
  // that contains it
  const size_t pbytes = (size_t)ops->slots * N * ops->esize + 64;
  for (int k = 0; k < 2; ++k) {
    if (cudaMalloc(&c->f[k], pbytes) != cudaSuccess || cudaMalloc(&c->g[k], pbytes) != cudaSuccess) {
      cudaFree(staging);
      return bail(LB_ENOMEM);
    }
  }
  // FP64: per-node moments and psi that each step kernel's ring reads (lb_fields_kernel)
  if (ops->esize == sizeof(double) && cudaMalloc(&c->pre, 6 * (size_t)N * sizeof(double)) != cudaSuccess) {
    cudaFree(staging);
    return bail(LB_ENOMEM);
  }
  if (cudaMalloc(&c->part, (size_t)p.nz * c->ntiles * NPART * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->diag, (size_t)(8 * p.nz + 8) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->nu_acc, 2 * sizeof(double)) != cudaSuccess) {
    cudaFree(staging);
    return bail(LB_ENOMEM);
  }
  if (cudaMemsetAsync(c->nu_acc, 0, 2 * sizeof(double), c->stream) != cudaSuccess) { cudaFree(staging); return bail(LB_ECUDA); }
  c->cur = 0;
  KArgs a = make_args(c);
  a.fout = c->f[0]; a.gout = c->g[0];
  if (ops->init(a, d_rho, d_T, c->stream) != cudaSuccess) { cudaFree(staging); return bail(LB_ECUDA); }
  if (staging) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) { cudaFree(staging); return bail(LB_ECUDA); }
    cudaFree(staging);
  }
  c->step = 0;
  *out = c;
  return LB_OK;
}

int lb_step(lb_ctx* c, long long nsteps) {
  if (!c) return LB_EINVAL;
  if (nsteps < 0) return lb_fail(c, LB_EINVAL, "nsteps < 0");
  const dim3 grid = fused_grid(c);
  // a Nu sample of state n is taken by the launch of step n -> n+1 (the paper's scheme; the
  // variants take it with a separate moments pass)
  const bool fuse = variant_of(c->p.forcing, c->p.psi_kind) == 0;
  for (long long s = 0; s < nsteps; ++s) {
    KArgs a = make_args(c);
    if (c->sample_pending && fuse) {
      a.part = c->part;
      LB_CU(c, c->ops->fused(a, MODE_STEP_DIAG, c->by, grid, c->stream));
      c->sample_pending = false;
      const int rc = finalize_diag(c, c->nu_acc);
      if (rc) return rc;
    } else {
      const int rc = flush_sample(c);
      if (rc) return rc;
      LB_CU(c, c->ops->fused(a, MODE_STEP, c->by, grid, c->stream));
    }
    c->cur ^= 1;
    c->step += 1;
    if (c->p.nu_every > 0 && c->step % c->p.nu_every == 0) c->sample_pending = true;
    if (c->p.check_every > 0 && c->step % c->p.check_every == 0) {
      int rc = c->sample_pending ? flush_sample(c) : run_diag(c, false);
      if (rc) return rc;
      double h[4];
      LB_CU(c, cudaMemcpyAsync(h, c->diag + c->p.nz, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      LB_CU(c, cudaStreamSynchronize(c->stream));
      if (!(h[1] > 0.0) || !(h[2] > 0.0) || h[3] != 0.0)
        return lb_fail(c, LB_ENONPHYS, "health check failed at step " + std::to_string(c->step));
    }
  }
  return LB_OK;
}

int lb_moments(lb_ctx* c, double* rho, double* ux, double* uy, double* uz, double* T, int on_device) {
  if (!c) return LB_EINVAL;
  KArgs a = make_args(c);
  double* outs[5] = {rho, ux, uy, uz, T};
  const size_t N = (size_t)c->N;
  if (!on_device) {
    if (!c->fields && cudaMalloc(&c->fields, 5 * N * sizeof(double)) != cudaSuccess)
      return lb_fail(c, LB_ENOMEM, "moments staging");
    for (int k = 0; k < 5; ++k) if (outs[k]) outs[k] = c->fields + k * N;
  }
  a.rho_out = outs[0]; a.ux_out = outs[1]; a.uy_out = outs[2]; a.uz_out = outs[3]; a.T_out = outs[4];
  a.part = nullptr;
  LB_CU(c, c->ops->fused(a, MODE_MOMENTS, c->by, fused_grid(c), c->stream));
  if (!on_device) {
    double* host[5] = {rho, ux, uy, uz, T};
    for (int k = 0; k < 5; ++k)
      if (host[k])
        LB_CU(c, cudaMemcpyAsync(host[k], c->fields + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CU(c, cudaStreamSynchronize(c->stream));
  }
  return LB_OK;
}

int lb_nusselt(lb_ctx* c, double* nu_mean, double* nu_z, double* nu_time_avg) {
  if (!c || !nu_mean) return c ? lb_fail(c, LB_EINVAL, "nu_mean is null") : LB_EINVAL;
  int rc = c->sample_pending ? flush_sample(c) : run_diag(c, false);
  if (rc) return rc;
  const int nz = c->p.nz;
  std::vector<double> h(nz + 1);
  double acc[2];
  LB_CU(c, cudaMemcpyAsync(h.data(), c->diag, (nz + 1) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaMemcpyAsync(acc, c->nu_acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  *nu_mean = h[nz];
  if (nu_z) std::memcpy(nu_z, h.data(), nz * sizeof(double));
  if (nu_time_avg) *nu_time_avg = acc[1] > 0 ? acc[0] / acc[1] : NAN;
  return LB_OK;
}

int lb_diagnostics(lb_ctx* c, double out[5]) {
  if (!c || !out) return c ? lb_fail(c, LB_EINVAL, "out is null") : LB_EINVAL;
  int rc = c->sample_pending ? flush_sample(c) : run_diag(c, false);
  if (rc) return rc;
  double h[5];
  LB_CU(c, cudaMemcpyAsync(h, c->diag + c->p.nz + 1, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 5; ++k) out[k] = h[k];
  return LB_OK;
}

int lb_populations(lb_ctx* c, double* f, double* g, int on_device) {
  if (!c) return LB_EINVAL;
  const size_t n = (size_t)Q * c->N;
  double* df = f;
  double* dg = g;
  if (!on_device) {
    if (!c->pops && cudaMalloc(&c->pops, 2 * n * sizeof(double)) != cudaSuccess)
      return lb_fail(c, LB_ENOMEM, "population staging");
    df = f ? c->pops : nullptr;
    dg = g ? c->pops + n : nullptr;
  }
  KArgs a = make_args(c);
  LB_CU(c, c->ops->pops(a, df, dg, c->stream));
  if (!on_device) {
    if (f) LB_CU(c, cudaMemcpyAsync(f, df, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (g) LB_CU(c, cudaMemcpyAsync(g, dg, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CU(c, cudaStreamSynchronize(c->stream));
  }
  return LB_OK;
}

int lb_set_populations(lb_ctx* c, const double* f, const double* g, int on_device) {
  if (!c) return LB_EINVAL;
  if (!f || !g) return lb_fail(c, LB_EINVAL, "f and g are both required");
  const size_t n = (size_t)Q * c->N;
  const double* df = f;
  const double* dg = g;
  if (!on_device) {
    if (!c->pops && cudaMalloc(&c->pops, 2 * n * sizeof(double)) != cudaSuccess)
      return lb_fail(c, LB_ENOMEM, "population staging");
    LB_CU(c, cudaMemcpyAsync(c->pops, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LB_CU(c, cudaMemcpyAsync(c->pops + n, g, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    df = c->pops;
    dg = c->pops + n;
  }
  // a Nu sample due for the replaced state is dropped; the buffer written is the current one
  c->sample_pending = false;
  KArgs a = make_args(c);
  a.fout = c->f[c->cur]; a.gout = c->g[c->cur];
  LB_CU(c, c->ops->setpops(a, df, dg, c->stream));
  if (!on_device) LB_CU(c, cudaStreamSynchronize(c->stream));
  c->from_init = false;
  return LB_OK;
}

int lb_save(lb_ctx* c, const char* path) {
  if (!c || !path) return c ? lb_fail(c, LB_EINVAL, "path is null") : LB_EINVAL;
  const int frc = flush_sample(c);    // the saved time average includes every due sample
  if (frc) return frc;
  const size_t pbytes = (size_t)c->ops->slots * c->N * c->ops->esize;
  std::vector<unsigned char> buf(2 * pbytes);
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "TLBMCKP2", 8);
  h.version = 2; h.precision = c->p.precision;
  h.nx = c->p.nx; h.ny = c->p.ny; h.nz = c->p.nz;
  h.step = c->step; h.rho0 = c->rho0; h.T0 = c->T0; h.params = c->p;
  LB_CU(c, cudaMemcpyAsync(buf.data(), c->f[c->cur], pbytes, cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaMemcpyAsync(buf.data() + pbytes, c->g[c->cur], pbytes, cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaMemcpyAsync(h.nu_acc, c->nu_acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  h.checksum = fnv1a(1469598103934665603ull, buf.data(), buf.size());
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return lb_fail(c, LB_EIO, std::string("cannot open ") + path);
  bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? LB_OK : lb_fail(c, LB_EIO, std::string("write failed: ") + path);
}

int lb_load(lb_ctx* c, const char* path) {
  if (!c || !path) return c ? lb_fail(c, LB_EINVAL, "path is null") : LB_EINVAL;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return lb_fail(c, LB_EIO, std::string("cannot open ") + path);
  CkptHeader h;
  const size_t pbytes = (size_t)c->ops->slots * c->N * c->ops->esize;
  std::vector<unsigned char> buf(2 * pbytes);
  bool ok = std::fread(&h, sizeof(h), 1, fp) == 1 && std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
  std::fclose(fp);
  if (!ok) return lb_fail(c, LB_EIO, "short read");
  if (std::memcmp(h.magic, "TLBMCKP2", 8) != 0 || h.version != 2) return lb_fail(c, LB_EIO, "bad magic/version");
  if (h.nx != c->p.nx || h.ny != c->p.ny || h.nz != c->p.nz || h.precision != c->p.precision)
    return lb_fail(c, LB_EIO, "grid or precision mismatch");
  // the physics parameters must be the context's: a state saved under other relaxation times,
  // coupling, conductivity, gravity, wall temperatures or scheme variant is refused (the
  // reference state rho0, T0 of the deviation storage is restored from the file)
  {
    const lb_params& q = h.params;
    const lb_params& p = c->p;
    const bool same = q.tau_nu == p.tau_nu && q.tau_kappa == p.tau_kappa && q.G == p.G &&
                      q.kappa == p.kappa && q.c_v == p.c_v && q.g_z == p.g_z && q.T_d == p.T_d &&
                      q.T_u == p.T_u && q.forcing == p.forcing && q.psi_kind == p.psi_kind &&
                      (p.psi_kind != PSI_VDW ||
                       (q.vdw_a == p.vdw_a && q.vdw_b == p.vdw_b && q.vdw_T == p.vdw_T));
    if (!same) return lb_fail(c, LB_EIO, "checkpoint parameters differ from the context's");
  }
  if (fnv1a(1469598103934665603ull, buf.data(), buf.size()) != h.checksum)
    return lb_fail(c, LB_EIO, "checksum mismatch");
  LB_CU(c, cudaMemcpyAsync(c->f[c->cur], buf.data(), pbytes, cudaMemcpyHostToDevice, c->stream));
  LB_CU(c, cudaMemcpyAsync(c->g[c->cur], buf.data() + pbytes, pbytes, cudaMemcpyHostToDevice, c->stream));
  LB_CU(c, cudaMemcpyAsync(c->nu_acc, h.nu_acc, 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  c->step = h.step;
  c->sample_pending = false;
  c->rho0 = h.rho0;
  c->T0 = h.T0;
  return LB_OK;
}

void lb_free(lb_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

}  // extern "C"
