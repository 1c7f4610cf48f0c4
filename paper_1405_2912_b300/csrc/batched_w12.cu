// batched_w12.cu -- the batched voter kernels with 12 warps per CTA: the
// plan's persistent kernel with and without the L2 prefetch.
#include "batched_kernels.cuh"

namespace ftv {

template <>
const void *group_fn_w<12>(int kind, int R, bool pf, bool small)
{
    if (small) return nullptr;
    return pf ? group_fn_shape<12, true, false>(kind, R) : group_fn_shape<12, false, false>(kind, R);
}

}  // namespace ftv
