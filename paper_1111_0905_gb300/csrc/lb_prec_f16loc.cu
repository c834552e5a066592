// Launch table of the float16 storage against local references (see lb_launch.cuh).
#include "lb_launch.cuh"

namespace tlbm {
const PrecOps kOpsF16Loc = {sizeof(half_loc), 1, &OpsImpl<half_loc>::prepare, &OpsImpl<half_loc>::fused,
                    &OpsImpl<half_loc>::init, &OpsImpl<half_loc>::pops,
                    &OpsImpl<half_loc>::tile_ok, &OpsImpl<half_loc>::info,
                    &OpsImpl<half_loc>::setpops, slots<half_loc>()};
}  // namespace tlbm
