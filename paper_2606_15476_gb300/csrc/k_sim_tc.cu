// k_sim_tc.cu -- tensor-core similarity (placeholder until the tcgen05 kernel lands).
#include "farm_internal.h"

namespace farm {

bool sim_tc_available() { return false; }

cudaError_t launch_sim_tc_tf32x3(const float *, const float *, const float *, const float *, float *, int64_t,
                                 int64_t, int32_t, int64_t, int, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace farm
