// lb_bound.cu -- the memory access pattern of one time step with none of its arithmetic.
//
// A step of the scheme pulls the 19 f and 19 g populations of every node from the neighbours
// x - c_l (streaming, Eqs. (6)-(7)) and writes 19 + 19 collided values back: 76 values per
// node. This kernel does exactly those loads and stores, in the same [19][nz][ny][nx] layout and
// element size, and nothing else, so its bandwidth is what the access pattern itself reaches at
// a given number of resident warps. The fused step's bandwidth divided by this kernel's at the
// fused step's own residency separates the cost of the pattern from the cost of the step's
// arithmetic and barriers. It is a measurement aid; its output is not a physical state.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lb.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxCtasPerSm = 4;   // the launch bound below: 32 warps per SM, <= 64 registers

// D3Q19 in the library's order: 0 rest; 1..6 axis (+-x, +-y, +-z); 7..10 xy; 11..14 xz; 15..18 yz.
__device__ __forceinline__ int dx(int l) {
  return (l == 1 || l == 7 || l == 9 || l == 11 || l == 13) ? 1
       : (l == 2 || l == 8 || l == 10 || l == 12 || l == 14) ? -1 : 0;
}
__device__ __forceinline__ int dy(int l) {
  return (l == 3 || l == 7 || l == 10 || l == 15 || l == 17) ? 1
       : (l == 4 || l == 8 || l == 9 || l == 16 || l == 18) ? -1 : 0;
}
__device__ __forceinline__ int dz(int l) {
  return (l == 5 || l == 11 || l == 14 || l == 15 || l == 18) ? 1
       : (l == 6 || l == 12 || l == 13 || l == 16 || l == 17) ? -1 : 0;
}

// Node idx takes population l from its pull source x - c_l: periodic in x and y, z clamped into
// [0, nz) (the step itself bounces back at the walls; the clamp keeps the same locality). All 38
// loads are issued before the first store, as the step has them in flight.
template <class T>
__global__ void __launch_bounds__(kThreads, kMaxCtasPerSm)
stream_bound_kernel(const T* __restrict__ fin, const T* __restrict__ gin, T* __restrict__ fout,
                    T* __restrict__ gout, int nx, int ny, int nz) {
  const unsigned plane = (unsigned)nx * (unsigned)ny;
  const unsigned N = plane * (unsigned)nz;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) {
    const int x = (int)(idx % (unsigned)nx);
    const int y = (int)((idx / (unsigned)nx) % (unsigned)ny);
    const int z = (int)(idx / plane);
    T f[19], g[19];
#pragma unroll
    for (int l = 0; l < 19; ++l) {
      int xs = x - dx(l);
      xs += xs < 0 ? nx : (xs >= nx ? -nx : 0);
      int ys = y - dy(l);
      ys += ys < 0 ? ny : (ys >= ny ? -ny : 0);
      int zs = z - dz(l);
      zs = zs < 0 ? 0 : (zs >= nz ? nz - 1 : zs);
      const unsigned e = (unsigned)l * N + (unsigned)zs * plane + (unsigned)ys * (unsigned)nx + (unsigned)xs;
      f[l] = __ldg(fin + e);
      g[l] = __ldg(gin + e);
    }
#pragma unroll
    for (int l = 0; l < 19; ++l) {
      fout[(size_t)l * N + idx] = f[l];
      gout[(size_t)l * N + idx] = g[l];
    }
  }
}

template <class T>
int launch(const void* fin, const void* gin, void* fout, void* gout, int nx, int ny, int nz,
           int ctas_per_sm, int* max_ctas_out, cudaStream_t st) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stream_bound_kernel<T>, kThreads, 0) != cudaSuccess)
    return LB_ECUDA;
  if (max_ctas_out) *max_ctas_out = occ;
  if (ctas_per_sm > occ) return LB_EINVAL;
  const unsigned N = (unsigned)nx * (unsigned)ny * (unsigned)nz;
  const unsigned blocks = ctas_per_sm == 0 ? (N + kThreads - 1) / kThreads : (unsigned)(sms * ctas_per_sm);
  stream_bound_kernel<T><<<blocks, kThreads, 0, st>>>(static_cast<const T*>(fin), static_cast<const T*>(gin),
                                                      static_cast<T*>(fout), static_cast<T*>(gout), nx, ny, nz);
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

}  // namespace

extern "C" int lb_stream_bound(int elem_bytes, const void* f_in, const void* g_in, void* f_out,
                               void* g_out, int nx, int ny, int nz, int ctas_per_sm,
                               int* max_ctas_per_sm, void* cuda_stream) {
  if (!f_in || !g_in || !f_out || !g_out || nx < 1 || ny < 1 || nz < 1 || ctas_per_sm < 0 ||
      (elem_bytes != 2 && elem_bytes != 4))
    return LB_EINVAL;
  if ((uint64_t)nx * (uint64_t)ny * (uint64_t)nz * 19u > 0xffffffffull) return LB_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return elem_bytes == 4
             ? launch<float>(f_in, g_in, f_out, g_out, nx, ny, nz, ctas_per_sm, max_ctas_per_sm, st)
             : launch<unsigned short>(f_in, g_in, f_out, g_out, nx, ny, nz, ctas_per_sm, max_ctas_per_sm, st);
}
