// Launch table of the __nv_bfloat16 population storage (see lb_launch.cuh).
#include "lb_launch.cuh"

namespace tlbm {
const PrecOps kOpsBF16 = {sizeof(__nv_bfloat16), 1, &OpsImpl<__nv_bfloat16>::prepare, &OpsImpl<__nv_bfloat16>::fused,
                    &OpsImpl<__nv_bfloat16>::init, &OpsImpl<__nv_bfloat16>::pops,
                    &OpsImpl<__nv_bfloat16>::tile_ok, &OpsImpl<__nv_bfloat16>::info,
                    &OpsImpl<__nv_bfloat16>::setpops, slots<__nv_bfloat16>()};
}  // namespace tlbm
