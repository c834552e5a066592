// lb_analysis.cu -- statistics of the current state (the paper's single-point and two-point
// analyses): per-plane profiles, the T-rho joint histogram and horizontal structure functions.
// Each is a reduction over the macroscopic fields of the state (rho, u, T of Eq. (8), the
// physical velocity u = (j + F/2)/rho), which a moments pass writes into the context's staging
// fields first. All sums are FP64 in a fixed order (deterministic); the histogram counts are
// integers.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "lb_ctx.h"

namespace tlbm {
namespace ana {

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

// One block per plane z: sums of rho, T and P div(u), P = rho T + (G/2) e^{-2/rho} (or, for
// the van der Waals psi, rho T + rho^2 (b T_v/(1 - b rho) - a)), div(u) by central differences
// with u_z -> -u_z across the walls (the step's divergence).
__global__ void profiles_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                                const double* __restrict__ uy, const double* __restrict__ uz,
                                const double* __restrict__ T, int nx, int ny, int nz, double G,
                                int psi_kind, double va, double vb, double vT,
                                double* __restrict__ out /* [nz][3] */) {
  __shared__ double sh[32];
  const int z = blockIdx.x;
  const int nxy = nx * ny;
  const size_t base = (size_t)z * nxy;
  double sr = 0.0, sT = 0.0, sPD = 0.0;
  for (int i = threadIdx.x; i < nxy; i += blockDim.x) {
    const int x = i % nx, y = i / nx;
    const size_t k = base + i;
    const double r = rho[k], t = T[k];
    const double uzp = (z + 1 < nz) ? uz[k + nxy] : -uz[k];
    const double uzm = (z - 1 >= 0) ? uz[k - nxy] : -uz[k];
    const double D = 0.5 * (ux[base + y * nx + (x + 1) % nx] - ux[base + y * nx + (x + nx - 1) % nx]) +
                     0.5 * (uy[base + ((y + 1) % ny) * nx + x] - uy[base + ((y + ny - 1) % ny) * nx + x]) +
                     0.5 * (uzp - uzm);
    const double P = r * t + ((psi_kind == PSI_VDW) ? r * r * (vb * vT / (1.0 - vb * r) - va)
                                                    : 0.5 * G * exp(-2.0 / r));
    sr += r; sT += t; sPD += P * D;
  }
  const double a = block_sum(sr, sh), b = block_sum(sT, sh), c = block_sum(sPD, sh);
  if (threadIdx.x == 0) {
    out[3 * z] = a / nxy; out[3 * z + 1] = b / nxy; out[3 * z + 2] = c / nxy;
  }
}

// Joint histogram of (T, rho) over planes [z_lo, z_hi): bin = floor((v - lo)/(hi - lo) * n) for
// lo <= v < hi (values outside are not counted); shared-memory counts, then global atomics.
__global__ void histogram_kernel(const double* __restrict__ rho, const double* __restrict__ T,
                                 size_t begin, size_t end, int nT, double Tlo, double Thi, int nr,
                                 double rlo, double rhi, unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned int hs[];
  const int nb = nT * nr;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hs[b] = 0u;
  __syncthreads();
  for (size_t k = begin + blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < end;
       k += (size_t)gridDim.x * blockDim.x) {
    const double t = T[k], r = rho[k];
    if (t >= Tlo && t < Thi && r >= rlo && r < rhi) {
      int it = (int)floor((t - Tlo) / (Thi - Tlo) * nT);
      int ir = (int)floor((r - rlo) / (rhi - rlo) * nr);
      it = it < nT - 1 ? it : nT - 1;
      ir = ir < nr - 1 ? ir : nr - 1;
      atomicAdd(&hs[it * nr + ir], 1u);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (hs[b]) atomicAdd(&counts[b], (unsigned long long)hs[b]);
}

// Structure functions for horizontal increments: block (r-1, z - z_lo) sums over plane z of
// (q(x + r e_x) - q(x))^p + (q(x + r e_y) - q(x))^p for q = u_z, T and p = 2, 4.
__global__ void structure_kernel(const double* __restrict__ uz, const double* __restrict__ T,
                                 int nx, int ny, int z_lo, double* __restrict__ out /* [rmax][nzs][4] */,
                                 int nzs) {
  __shared__ double sh[32];
  const int r = blockIdx.x + 1;
  const int zi = blockIdx.y;
  const int z = z_lo + zi;
  const int nxy = nx * ny;
  const size_t base = (size_t)z * nxy;
  double a2 = 0.0, a4 = 0.0, b2 = 0.0, b4 = 0.0;
  for (int i = threadIdx.x; i < nxy; i += blockDim.x) {
    const int x = i % nx, y = i / nx;
    const size_t k = base + i;
    const size_t kx = base + y * nx + (x + r) % nx;
    const size_t ky = base + ((y + r) % ny) * nx + x;
    const double du1 = uz[kx] - uz[k], du2 = uz[ky] - uz[k];
    const double dt1 = T[kx] - T[k], dt2 = T[ky] - T[k];
    const double du1s = du1 * du1, du2s = du2 * du2, dt1s = dt1 * dt1, dt2s = dt2 * dt2;
    a2 += du1s + du2s; a4 += du1s * du1s + du2s * du2s;
    b2 += dt1s + dt2s; b4 += dt1s * dt1s + dt2s * dt2s;
  }
  const double s0 = block_sum(a2, sh), s1 = block_sum(a4, sh), s2 = block_sum(b2, sh), s3 = block_sum(b4, sh);
  if (threadIdx.x == 0) {
    double* o = out + ((size_t)(r - 1) * nzs + zi) * 4;
    o[0] = s0; o[1] = s1; o[2] = s2; o[3] = s3;
  }
}

// Local convective heat flux q = rho U u_z, U = c_v T + U_NI(rho) (the bulk term of Nu, Eq. (4)).
struct FluxArgs {
  double c_v, G, va, vb, vT;
  int psi_kind;
};
__device__ __forceinline__ double flux_q(double r, double t, double w, const FluxArgs& fa) {
  const double uni = (fa.psi_kind == PSI_VDW) ? -fa.vT * log(1.0 - fa.vb * r) - fa.va * r
                                              : 0.25 * fa.G * exp(-2.0 / r);
  return r * (fa.c_v * t + uni) * w;
}

// Pass 1 of the heat-flux pdf: counts of lo <= q < hi in n bins (shared counts, global integer
// atomics) and this block's sum of q (fixed thread-to-node assignment and reduction order).
__global__ void flux_hist_kernel(const double* __restrict__ rho, const double* __restrict__ uz,
                                 const double* __restrict__ T, size_t begin, size_t end, FluxArgs fa,
                                 int nb, double lo, double hi, unsigned long long* __restrict__ counts,
                                 double* __restrict__ part) {
  extern __shared__ unsigned int hq[];
  __shared__ double sh[32];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hq[b] = 0u;
  __syncthreads();
  double s = 0.0;
  for (size_t k = begin + blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < end;
       k += (size_t)gridDim.x * blockDim.x) {
    const double q = flux_q(rho[k], T[k], uz[k], fa);
    s += q;
    if (q >= lo && q < hi) {
      int b = (int)floor((q - lo) / (hi - lo) * nb);
      b = b < nb - 1 ? b : nb - 1;
      atomicAdd(&hq[b], 1u);
    }
  }
  const double bs = block_sum(s, sh);
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (hq[b]) atomicAdd(&counts[b], (unsigned long long)hq[b]);
  if (threadIdx.x == 0) part[blockIdx.x] = bs;
}

// Pass 2: this block's sum of (q - mean)^2.
__global__ void flux_var_kernel(const double* __restrict__ rho, const double* __restrict__ uz,
                                const double* __restrict__ T, size_t begin, size_t end, FluxArgs fa,
                                double mean, double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t k = begin + blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < end;
       k += (size_t)gridDim.x * blockDim.x) {
    const double d = flux_q(rho[k], T[k], uz[k], fa) - mean;
    s += d * d;
  }
  const double bs = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = bs;
}

}  // namespace ana
}  // namespace tlbm

using namespace tlbm;

namespace {

// macroscopic fields of the current state in the context's staging arrays (device)
int fields_on_device(lb_ctx* c, double** rho, double** ux, double** uy, double** uz, double** T) {
  const size_t N = (size_t)c->N;
  if (!c->fields && cudaMalloc(&c->fields, 5 * N * sizeof(double)) != cudaSuccess)
    return lb_fail(c, LB_ENOMEM, "field staging");
  *rho = c->fields; *ux = c->fields + N; *uy = c->fields + 2 * N; *uz = c->fields + 3 * N;
  *T = c->fields + 4 * N;
  return lb_moments(c, *rho, *ux, *uy, *uz, *T, 1);
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace

extern "C" int lb_profiles(lb_ctx* c, double* rho_z, double* T_z, double* PdivU_z) {
  if (!c) return LB_EINVAL;
  double *rho, *ux, *uy, *uz, *T;
  int rc = fields_on_device(c, &rho, &ux, &uy, &uz, &T);
  if (rc) return rc;
  const int nz = c->p.nz;
  DevBuf out;
  if (cudaMalloc(&out.p, (size_t)3 * nz * sizeof(double)) != cudaSuccess) return lb_fail(c, LB_ENOMEM, "profiles");
  ana::profiles_kernel<<<nz, 256, 0, c->stream>>>(rho, ux, uy, uz, T, c->p.nx, c->p.ny, nz, c->p.G,
                                                  c->p.psi_kind, c->p.vdw_a, c->p.vdw_b, c->p.vdw_T,
                                                  static_cast<double*>(out.p));
  LB_CU(c, cudaGetLastError());
  std::vector<double> h((size_t)3 * nz);
  LB_CU(c, cudaMemcpyAsync(h.data(), out.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  for (int z = 0; z < nz; ++z) {
    if (rho_z) rho_z[z] = h[3 * z];
    if (T_z) T_z[z] = h[3 * z + 1];
    if (PdivU_z) PdivU_z[z] = h[3 * z + 2];
  }
  return LB_OK;
}

extern "C" int lb_histogram_T_rho(lb_ctx* c, int z_lo, int z_hi, int nT, double T_lo, double T_hi,
                                  int nrho, double rho_lo, double rho_hi, unsigned long long* counts) {
  if (!c || !counts) return c ? lb_fail(c, LB_EINVAL, "counts is null") : LB_EINVAL;
  if (z_lo < 0 || z_hi > c->p.nz || z_lo >= z_hi || nT < 1 || nrho < 1 || (long long)nT * nrho > 12288 ||
      !(T_hi > T_lo) || !(rho_hi > rho_lo))
    return lb_fail(c, LB_EINVAL, "histogram ranges");
  double *rho, *ux, *uy, *uz, *T;
  int rc = fields_on_device(c, &rho, &ux, &uy, &uz, &T);
  if (rc) return rc;
  const int nb = nT * nrho;
  DevBuf cnt;
  if (cudaMalloc(&cnt.p, (size_t)nb * sizeof(unsigned long long)) != cudaSuccess) return lb_fail(c, LB_ENOMEM, "histogram");
  LB_CU(c, cudaMemsetAsync(cnt.p, 0, (size_t)nb * sizeof(unsigned long long), c->stream));
  const size_t plane = (size_t)c->plane;
  ana::histogram_kernel<<<304, 256, (size_t)nb * sizeof(unsigned int), c->stream>>>(
      rho, T, (size_t)z_lo * plane, (size_t)z_hi * plane, nT, T_lo, T_hi, nrho, rho_lo, rho_hi,
      static_cast<unsigned long long*>(cnt.p));
  LB_CU(c, cudaGetLastError());
  LB_CU(c, cudaMemcpyAsync(counts, cnt.p, (size_t)nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

extern "C" int lb_structure_functions(lb_ctx* c, int rmax, int z_lo, int z_hi, double* S2_uz,
                                      double* S4_uz, double* S2_T, double* S4_T) {
  if (!c) return LB_EINVAL;
  if (rmax < 1 || rmax >= c->p.nx || rmax >= c->p.ny || z_lo < 0 || z_hi > c->p.nz || z_lo >= z_hi)
    return lb_fail(c, LB_EINVAL, "structure-function ranges");
  double *rho, *ux, *uy, *uz, *T;
  int rc = fields_on_device(c, &rho, &ux, &uy, &uz, &T);
  if (rc) return rc;
  const int nzs = z_hi - z_lo;
  DevBuf out;
  const size_t n = (size_t)rmax * nzs * 4;
  if (cudaMalloc(&out.p, n * sizeof(double)) != cudaSuccess) return lb_fail(c, LB_ENOMEM, "structure functions");
  ana::structure_kernel<<<dim3(rmax, nzs), 256, 0, c->stream>>>(uz, T, c->p.nx, c->p.ny, z_lo,
                                                                static_cast<double*>(out.p), nzs);
  LB_CU(c, cudaGetLastError());
  std::vector<double> h(n);
  LB_CU(c, cudaMemcpyAsync(h.data(), out.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  const double cnt = 2.0 * (double)c->plane * nzs;   // x and y increments of every bulk node
  for (int r = 0; r < rmax; ++r) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int z = 0; z < nzs; ++z)
      for (int k = 0; k < 4; ++k) s[k] += h[((size_t)r * nzs + z) * 4 + k];
    if (S2_uz) S2_uz[r] = s[0] / cnt;
    if (S4_uz) S4_uz[r] = s[1] / cnt;
    if (S2_T) S2_T[r] = s[2] / cnt;
    if (S4_T) S4_T[r] = s[3] / cnt;
  }
  return LB_OK;
}

extern "C" int lb_heat_flux_pdf(lb_ctx* c, int z_lo, int z_hi, int nbins, double q_lo, double q_hi,
                                unsigned long long* counts, double* stats) {
  if (!c) return LB_EINVAL;
  if (z_lo < 0 || z_hi > c->p.nz || z_lo >= z_hi || nbins < 1 || nbins > 12288 || !(q_hi > q_lo))
    return lb_fail(c, LB_EINVAL, "heat-flux pdf ranges");
  double *rho, *ux, *uy, *uz, *T;
  int rc = fields_on_device(c, &rho, &ux, &uy, &uz, &T);
  if (rc) return rc;
  const int blocks = 304;
  DevBuf cnt, part;
  if (cudaMalloc(&cnt.p, (size_t)nbins * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&part.p, 2 * blocks * sizeof(double)) != cudaSuccess)
    return lb_fail(c, LB_ENOMEM, "heat-flux pdf");
  LB_CU(c, cudaMemsetAsync(cnt.p, 0, (size_t)nbins * sizeof(unsigned long long), c->stream));
  const size_t plane = (size_t)c->plane, begin = (size_t)z_lo * plane, end = (size_t)z_hi * plane;
  const ana::FluxArgs fa = {c->p.c_v, c->p.G, c->p.vdw_a, c->p.vdw_b, c->p.vdw_T, c->p.psi_kind};
  double* pd = static_cast<double*>(part.p);
  ana::flux_hist_kernel<<<blocks, 256, (size_t)nbins * sizeof(unsigned int), c->stream>>>(
      rho, uz, T, begin, end, fa, nbins, q_lo, q_hi, static_cast<unsigned long long*>(cnt.p), pd);
  LB_CU(c, cudaGetLastError());
  std::vector<double> h(blocks);
  LB_CU(c, cudaMemcpyAsync(h.data(), pd, blocks * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  const double n = (double)(end - begin);
  double s = 0.0;
  for (int b = 0; b < blocks; ++b) s += h[b];
  const double mean = s / n;
  ana::flux_var_kernel<<<blocks, 256, 0, c->stream>>>(rho, uz, T, begin, end, fa, mean, pd + blocks);
  LB_CU(c, cudaGetLastError());
  LB_CU(c, cudaMemcpyAsync(h.data(), pd + blocks, blocks * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (counts)
    LB_CU(c, cudaMemcpyAsync(counts, cnt.p, (size_t)nbins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  LB_CU(c, cudaStreamSynchronize(c->stream));
  double v = 0.0;
  for (int b = 0; b < blocks; ++b) v += h[b];
  if (stats) { stats[0] = n; stats[1] = mean; stats[2] = v / n; }
  return LB_OK;
}
