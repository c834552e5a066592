// Launch table of the __half population storage (see lb_launch.cuh).
#include "lb_launch.cuh"

namespace tlbm {
const PrecOps kOpsF16 = {sizeof(__half), 1, &OpsImpl<__half>::prepare, &OpsImpl<__half>::fused,
                    &OpsImpl<__half>::init, &OpsImpl<__half>::pops,
                    &OpsImpl<__half>::tile_ok, &OpsImpl<__half>::info,
                    &OpsImpl<__half>::setpops, slots<__half>()};
}  // namespace tlbm
