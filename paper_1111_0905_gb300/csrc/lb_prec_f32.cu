// Launch table of the float population storage (see lb_launch.cuh).
#include "lb_launch.cuh"

namespace tlbm {
const PrecOps kOpsF32 = {sizeof(float), 0, &OpsImpl<float>::prepare, &OpsImpl<float>::fused,
                    &OpsImpl<float>::init, &OpsImpl<float>::pops,
                    &OpsImpl<float>::tile_ok, &OpsImpl<float>::info,
                    &OpsImpl<float>::setpops, slots<float>()};
}  // namespace tlbm
