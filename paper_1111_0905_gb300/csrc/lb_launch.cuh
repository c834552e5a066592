// lb_launch.cuh -- per-precision launch table of the kernels in lb_kernels.cuh.
// Each precision is compiled in its own translation unit (lb_prec_*.cu) that defines one table.
#pragma once
#include "lb_kernels.cuh"

namespace tlbm {

struct PrecOps {
  size_t esize;        // bytes per stored population
  int deviation;       // 1 if populations are stored as deviations from w_l * ref
  cudaError_t (*prepare)();   // per-device kernel attributes (call with the device current)
  cudaError_t (*fused)(const KArgs&, int mode, int by, dim3 grid, cudaStream_t);
  cudaError_t (*init)(const KArgs&, const double*, const double*, cudaStream_t);
  cudaError_t (*pops)(const KArgs&, double*, double*, cudaStream_t);
  bool (*tile_ok)(int by);    // whether the tile height's shared-memory window fits a CTA
  // launch description of the step kernel for a tile height and variant: out = {threads per
  // CTA, dynamic shared memory bytes, resident CTAs per SM, registers per thread}
  cudaError_t (*info)(int by, int var, int out[4]);
  // store a given pre-collision state (float64 [19][N] f and g on the device) as the buffer
  cudaError_t (*setpops)(const KArgs&, const double*, const double*, cudaStream_t);
  int slots;           // stored slots per lattice and node: 19, or 21 with the local references
};

extern const PrecOps kOpsF64, kOpsF32, kOpsBF16, kOpsF16, kOpsF16Loc;

template <class S> struct OpsImpl {
  using R = typename Store<S>::R;

  // dynamic shared memory of a tile height; tile heights whose windows exceed the 227 KB a CTA
  // may use are not available, nor FP64 with BY = 16 (a CTA of 512 threads leaves the FP64
  // collision 128 registers per thread, too few for its 38 double-precision populations)
  static constexpr bool STG = std::is_same<S, float>::value && TLBM_STAGE;
  template <int BY> static constexpr size_t smem() { return Geo<BY>::template smem_bytes<S, R, STG>(); }
  template <int BY> static constexpr bool fits() {
    return smem<BY>() + 1024 <= 227u * 1024u && !(std::is_same<S, double>::value && BY > 8);
  }
  template <int BY, int MODE, int VAR = 0> static cudaError_t attr() {
    if constexpr (!fits<BY>()) {
      return cudaSuccess;
    } else {
      return cudaFuncSetAttribute(lb_fused_kernel<S, BY, MODE, VAR>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem<BY>());
    }
  }
  template <int BY> static cudaError_t attr_by() {
    cudaError_t e;
    if ((e = attr<BY, MODE_STEP, 0>()) != cudaSuccess) return e;
    if ((e = attr<BY, MODE_STEP, VAR_GUO>()) != cudaSuccess) return e;
    if ((e = attr<BY, MODE_STEP, VAR_VDW>()) != cudaSuccess) return e;
    if ((e = attr<BY, MODE_STEP, VAR_GUO | VAR_VDW>()) != cudaSuccess) return e;
    if ((e = attr<BY, MODE_STEP_DIAG, 0>()) != cudaSuccess) return e;
    if ((e = attr<BY, MODE_MOMENTS, 0>()) != cudaSuccess) return e;
    return attr<BY, MODE_MOMENTS, VAR_VDW>();
  }
  static cudaError_t prepare() {
    cudaError_t e;
    if ((e = attr_by<4>()) != cudaSuccess) return e;
    if ((e = attr_by<8>()) != cudaSuccess) return e;
    return attr_by<16>();
  }
  template <int BY, int VAR> static cudaError_t info_var(int out[4]) {
    if constexpr (!fits<BY>()) {
      return cudaErrorInvalidConfiguration;
    } else {
      cudaFuncAttributes fa;
      cudaError_t e = cudaFuncGetAttributes(&fa, lb_fused_kernel<S, BY, MODE_STEP, VAR>);
      if (e != cudaSuccess) return e;
      int n = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lb_fused_kernel<S, BY, MODE_STEP, VAR>,
                                                        BX * BY, smem<BY>());
      if (e != cudaSuccess) return e;
      out[0] = BX * BY; out[1] = (int)smem<BY>(); out[2] = n; out[3] = fa.numRegs;
      return cudaSuccess;
    }
  }
  template <int BY> static cudaError_t info_by(int var, int out[4]) {
    switch (var) {
      case 0: return info_var<BY, 0>(out);
      case VAR_GUO: return info_var<BY, VAR_GUO>(out);
      case VAR_VDW: return info_var<BY, VAR_VDW>(out);
      default: return info_var<BY, VAR_GUO | VAR_VDW>(out);
    }
  }
  static cudaError_t info(int by, int var, int out[4]) {
    if (by == 4) return info_by<4>(var, out);
    if (by == 8) return info_by<8>(var, out);
    if (by == 16) return info_by<16>(var, out);
    return cudaErrorInvalidValue;
  }
  static bool tile_ok(int by) {
    return (by == 4 && fits<4>()) || (by == 8 && fits<8>()) || (by == 16 && fits<16>());
  }
  template <int BY, int MODE, int VAR> static cudaError_t go(const KArgs& a, dim3 grid, cudaStream_t st) {
    if constexpr (!fits<BY>()) {
      return cudaErrorInvalidConfiguration;
    } else {
      lb_fused_kernel<S, BY, MODE, VAR><<<grid, dim3(BX, BY), smem<BY>(), st>>>(a);
      return cudaGetLastError();
    }
  }
  template <int BY> static cudaError_t go_by(const KArgs& a, int mode, dim3 grid, cudaStream_t st) {
    const int var = variant_of(a.forcing, a.psi_kind);
    // the fused step + Nu sample exists for the paper's scheme only (the caller checks)
    if (mode == MODE_STEP_DIAG) return var == 0 ? go<BY, MODE_STEP_DIAG, 0>(a, grid, st) : cudaErrorInvalidValue;
    if (mode == MODE_STEP) {
      switch (var) {
        case 0: return go<BY, MODE_STEP, 0>(a, grid, st);
        case VAR_GUO: return go<BY, MODE_STEP, VAR_GUO>(a, grid, st);
        case VAR_VDW: return go<BY, MODE_STEP, VAR_VDW>(a, grid, st);
        default: return go<BY, MODE_STEP, VAR_GUO | VAR_VDW>(a, grid, st);
      }
    }
    // the moments pass has no collision: only the pseudopotential matters
    if (var & VAR_VDW) return go<BY, MODE_MOMENTS, VAR_VDW>(a, grid, st);
    return go<BY, MODE_MOMENTS, 0>(a, grid, st);
  }
  static cudaError_t fused(const KArgs& a, int mode, int by, dim3 grid, cudaStream_t st) {
    if constexpr (std::is_same<S, double>::value) {
      // FP64: the ring's moments and psi of the state read, once per node, before the step
      if (a.pre == nullptr) return cudaErrorInvalidValue;
      const unsigned blocks = ((unsigned)a.N + 255u) / 256u;
      if (a.psi_kind == PSI_VDW) lb_fields_kernel<true><<<blocks, 256, 0, st>>>(a);
      else lb_fields_kernel<false><<<blocks, 256, 0, st>>>(a);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    if (by == 4) return go_by<4>(a, mode, grid, st);
    if (by == 8) return go_by<8>(a, mode, grid, st);
    if (by == 16) return go_by<16>(a, mode, grid, st);
    return cudaErrorInvalidValue;
  }
  static int blocks_for(int N) {
    long long b = ((long long)N + 255) / 256;
    return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
  }
  static cudaError_t init(const KArgs& a, const double* rho, const double* T, cudaStream_t st) {
    lb_init_kernel<S><<<blocks_for(a.N), 256, 0, st>>>(a, rho, T);
    return cudaGetLastError();
  }
  static cudaError_t setpops(const KArgs& a, const double* f, const double* g, cudaStream_t st) {
    lb_setpops_kernel<S><<<blocks_for(a.N), 256, 0, st>>>(a, f, g);
    return cudaGetLastError();
  }
  static cudaError_t pops(const KArgs& a, double* f, double* g, cudaStream_t st) {
    lb_pops_kernel<S><<<blocks_for(a.N), 256, 0, st>>>(a, f, g);
    return cudaGetLastError();
  }
};

}  // namespace tlbm
