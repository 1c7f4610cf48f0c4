// batched_w8.cu -- the batched voter kernels with 8 warps per CTA: the
// plan's persistent kernel with and without the L2 prefetch, and the small-batch kernel.
#include "batched_kernels.cuh"

namespace ftv {

template <>
const void *group_fn_w<8>(int kind, int R, bool pf, bool small)
{
    if (small) return group_fn_shape<8, false, true>(kind, R);
    return pf ? group_fn_shape<8, true, false>(kind, R) : group_fn_shape<8, false, false>(kind, R);
}

}  // namespace ftv
