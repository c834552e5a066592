// Launch table of the double population storage (see lb_launch.cuh).
#include "lb_launch.cuh"

namespace tlbm {
const PrecOps kOpsF64 = {sizeof(double), 0, &OpsImpl<double>::prepare, &OpsImpl<double>::fused,
                    &OpsImpl<double>::init, &OpsImpl<double>::pops,
                    &OpsImpl<double>::tile_ok, &OpsImpl<double>::info,
                    &OpsImpl<double>::setpops, slots<double>()};
}  // namespace tlbm
