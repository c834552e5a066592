// lb_noalloc.cu -- Nusselt profile from caller-owned device fields, with no device allocation.
//
// Some callers cannot call cudaMalloc: applications that hand all device memory to their own
// pool allocator up front and forbid further allocations, and latency-critical loops where
// cudaMalloc's implicit device synchronisation is not acceptable. For them this entry point
// computes the same per-plane reduction as the diagnostics path of lb_nusselt, but keeps its
// per-plane partial sums in a fixed file-scope device array instead of context scratch.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lb.h"

namespace {

constexpr int kMaxPlanes = LB_NOALLOC_MAX_NZ;
constexpr int kMaxDevices = 64;

// Per-plane partials (sum rho U u_z, sum T), two doubles per plane. Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) double g_plane_sums[2 * kMaxPlanes];

// Device address of g_plane_sums for each device (host code may not use the symbol itself).
double* g_scratch[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One block per plane z: fixed-order FP64 sums of rho U u_z and T, with the internal energy of
// the paper's pseudopotential psi = exp(-1/rho), U = c_v T + (G/4) e^{-2/rho} (Eq. (2)).
__global__ void plane_sums_kernel(const double* __restrict__ rho, const double* __restrict__ uz,
                                  const double* __restrict__ T, int nxy, double c_v, double G,
                                  double* __restrict__ sums) {
  __shared__ double sh[2][32];
  const int z = blockIdx.x;
  const size_t base = (size_t)z * nxy;
  double c = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < nxy; i += blockDim.x) {
    const double r = rho[base + i], Ti = T[base + i];
    const double U = c_v * Ti + 0.25 * G * exp(-2.0 / r);
    c += r * U * uz[base + i];
    t += Ti;
  }
  c = warp_sum_d(c);
  t = warp_sum_d(t);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sh[0][w] = c; sh[1][w] = t; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double cs = 0.0, ts = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { cs += sh[0][k]; ts += sh[1][k]; }
    sums[2 * z] = cs;
    sums[2 * z + 1] = ts;
  }
}

// Nu(z) = (<rho U u_z> - kappa (T(z+1) - T(z-1))/2) / (kappa (T_d - T_u)/nz), wall ghosts
// 2 T_wall - T; nu_out[nz] = mean over z (fixed order).
__global__ void finalize_kernel(const double* __restrict__ sums, int nz, int nxy, double kappa,
                                double T_d, double T_u, double* __restrict__ nu_out) {
  const double norm = kappa * (T_d - T_u) / nz;
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    const double Tp = (z + 1 < nz) ? sums[2 * (z + 1) + 1] : 2.0 * T_u * nxy - sums[2 * (nz - 1) + 1];
    const double Tm = (z - 1 >= 0) ? sums[2 * (z - 1) + 1] : 2.0 * T_d * nxy - sums[1];
    nu_out[z] = ((sums[2 * z] - kappa * 0.5 * (Tp - Tm)) / nxy) / norm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += nu_out[z];
    nu_out[nz] = s / nz;
  }
}

// Device address of the scratch array on the current device, looked up once per device.
int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LB_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_plane_sums) != cudaSuccess || p == nullptr) return LB_ECUDA;
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return LB_OK;
}

}  // namespace

extern "C" int lb_nusselt_fields_noalloc(const double* rho, const double* uz, const double* T,
                                         int nx, int ny, int nz, double kappa, double G, double c_v,
                                         double T_d, double T_u, double* nu_out, void* cuda_stream) {
  if (!rho || !uz || !T || !nu_out) return LB_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1 || nz > kMaxPlanes) return LB_EINVAL;
  if ((long long)nx * ny >= (1ll << 31)) return LB_EINVAL;
  if (!(kappa > 0.0) || !(c_v > 0.0) || !(T_d != T_u)) return LB_EINVAL;
  double* sums = nullptr;
  int rc = scratch_for_current_device(&sums);
  if (rc != LB_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int nxy = nx * ny;
  // Launch errors are taken from cudaLaunchKernel's own return value. The runtime's last-error
  // slot is only peeked at, never cleared: an error that the caller's earlier work left there
  // stays for the caller, and is not reported as this call's failure.
  const cudaError_t before = cudaPeekAtLastError();
  void* a1[] = {(void*)&rho, (void*)&uz, (void*)&T, (void*)&nxy, (void*)&c_v, (void*)&G, (void*)&sums};
  cudaError_t e = cudaLaunchKernel((const void*)plane_sums_kernel, dim3(nz), dim3(256), a1, 0, st);
  if (e != cudaSuccess && e != before) return LB_ECUDA;
  void* a2[] = {(void*)&sums, (void*)&nz, (void*)&nxy, (void*)&kappa, (void*)&T_d, (void*)&T_u, (void*)&nu_out};
  e = cudaLaunchKernel((const void*)finalize_kernel, dim3(1), dim3(256), a2, 0, st);
  if (e != cudaSuccess && e != before) return LB_ECUDA;
  return LB_OK;
}
