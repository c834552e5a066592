// lb_ctx.h -- the context behind the opaque lb_ctx of include/lb.h (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/lb.h"
#include "lb_launch.cuh"

struct lb_ctx {
  lb_params p;
  int device = 0;
  cudaStream_t stream = nullptr;
  const tlbm::PrecOps* ops = nullptr;
  void* f[2] = {nullptr, nullptr};
  void* g[2] = {nullptr, nullptr};
  int cur = 0;
  int N = 0, plane = 0;
  int by = 8, zc = 0, tiles_x = 0, tiles_y = 0, ntiles = 0, nchunks = 0;
  double lam = 0.0, rho0 = 0.0, T0 = 0.0;
  double* part = nullptr;    // [nz][ntiles][NPART]
  double* diag = nullptr;    // [nz + 8]
  double* nu_acc = nullptr;  // [2]
  double* fields = nullptr;  // [5][N] staging for host-bound lb_moments
  double* pops = nullptr;    // [38][N] staging for host-bound lb_populations
  double* pre = nullptr;     // FP64 form: [6][N] rho, 1/rho, j, psi of the state a step reads
  long long step = 0;
  // the current state is due for a Nu sample (nu_every) that the next step's launch takes in
  // passing (fused step + diagnostics); lb_nusselt, lb_diagnostics, lb_save and
  // lb_adjoint_step take it first with a separate moments pass
  bool sample_pending = false;
  // the state is lb_init's equilibrium of its fields (or its successors by lb_step); false once
  // lb_set_populations replaced it (dJ/dT0 of lb_adjoint_step needs the former)
  bool from_init = true;
  std::string err;
};

inline int lb_fail(lb_ctx* c, int code, const std::string& what) {
  if (c) c->err = what;
  return code;
}
inline int lb_cuda_fail(lb_ctx* c, const char* where, cudaError_t e) {
  return lb_fail(c, LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define LB_CU(ctx, call)                                           \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return lb_cuda_fail((ctx), #call, e_);  \
  } while (0)

// shared host helpers (lb_api.cu)
tlbm::KArgs make_args(const lb_ctx* c);
dim3 fused_grid(const lb_ctx* c);
int run_diag(lb_ctx* c, bool accumulate);
int run_diag_acc(lb_ctx* c, double* acc);
int finalize_diag(lb_ctx* c, double* acc);   // Nu(z) and health values from the partials
int flush_sample(lb_ctx* c);                 // take a pending Nu sample (moments pass)
