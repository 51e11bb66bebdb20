// Tensor-core contraction path for large fused gates (placeholder until the tcgen05 kernel lands).
#include "sv_internal.h"

namespace svg {

int build_tc_operands(sv_fused *f)
{
    f->tc_offset.assign(f->gates.size(), SIZE_MAX);
    for (const FusedGate &g : f->gates)
        if (g.path == SV_PATH_TC_TF32 || g.path == SV_PATH_TC_BF16X3) {
            set_error("tensor-core path is not available in this build");
            return SV_EINVAL;
        }
    return SV_OK;
}

int launch_tc_gate(float *, int, const FusedGate &, const void *, cudaStream_t, int)
{
    set_error("tensor-core path is not available in this build");
    return SV_EINVAL;
}

}  // namespace svg
