// vote_flag.cu -- the single-task voter's default shapes built with a
// completion flag (vote_kernel<..., FLAG = true>): the server's lone requests
// and large ones vote through these, and the last CTA writes the request's
// flag to host-mapped memory after its statistics.  They live in a
// translation unit of their own so that the library's build stays parallel.
#include "runtime.h"
#include "vote_kernel.cuh"

namespace ftv {

template <int K, int R, int W, bool PF, int JB, bool SMALL>
const void *flagged_vote_kernel()
{
    static_assert(kDefaultShape<K, R, W, PF, JB, SMALL>, "only the default shapes are built with the flag");
    return reinterpret_cast<const void *>(vote_kernel<K, R, W, PF, JB, SMALL, true>);
}

// Each (K, R): the 8-warp and 16-warp SMALL forms and 16 warps without the
// prefetch (also the policy shape of every (K, R) but f32 R = 3).
#define FTV_FLAGGED_KR(K, R)                                                        \
    template const void *flagged_vote_kernel<K, R, kTinyWarps, false, kSubBatch<K, R>, true>(); \
    template const void *flagged_vote_kernel<K, R, 16, false, kSubBatch<K, R>, true>();         \
    template const void *flagged_vote_kernel<K, R, 16, false, kSubBatch<K, R>, false>();
#define FTV_FLAGGED_K(K)                                                            \
    FTV_FLAGGED_KR(K, 2) FTV_FLAGGED_KR(K, 3) FTV_FLAGGED_KR(K, 4) FTV_FLAGGED_KR(K, 5) \
    FTV_FLAGGED_KR(K, 6) FTV_FLAGGED_KR(K, 7) FTV_FLAGGED_KR(K, 8)
FTV_FLAGGED_K(K_F32)
FTV_FLAGGED_K(K_F64)
FTV_FLAGGED_K(K_B1)
FTV_FLAGGED_K(K_B4)
FTV_FLAGGED_K(K_B8)
// the policy shape of f32 R = 3: 12 warps with the L2 prefetch
template const void *flagged_vote_kernel<K_F32, 3, 12, true, kSubBatch<K_F32, 3>, false>();
#undef FTV_FLAGGED_K
#undef FTV_FLAGGED_KR

template <int K, int R>
static int preload_flagged_kr()
{
    constexpr int JB = kSubBatch<K, R>;
    using P = VotePolicy<K, R>;
    const void *fns[] = {flagged_vote_kernel<K, R, kTinyWarps, false, JB, true>(),
                         flagged_vote_kernel<K, R, 16, false, JB, true>(),
                         flagged_vote_kernel<K, R, 16, false, JB, false>(),
                         flagged_vote_kernel<K, R, P::kWarps, P::kPrefetch, JB, false>()};
    const int warps[] = {kTinyWarps, 16, 16, P::kWarps};
    for (int i = 0; i < 4; ++i) {
        int sms = 0, per_sm = 0;
        const int rc = occupancy(fns[i], warps[i] * 32, kSmemBytes, &sms, &per_sm);
        if (rc != FT_OK) return rc;
    }
    return FT_OK;
}

template <int K>
static int preload_flagged_k()
{
    int rc;
    if ((rc = preload_flagged_kr<K, 2>()) != FT_OK || (rc = preload_flagged_kr<K, 3>()) != FT_OK ||
        (rc = preload_flagged_kr<K, 4>()) != FT_OK || (rc = preload_flagged_kr<K, 5>()) != FT_OK ||
        (rc = preload_flagged_kr<K, 6>()) != FT_OK || (rc = preload_flagged_kr<K, 7>()) != FT_OK)
        return rc;
    return preload_flagged_kr<K, 8>();
}

int preload_flagged_vote_kernels()
{
    int rc;
    if ((rc = preload_flagged_k<K_F32>()) != FT_OK || (rc = preload_flagged_k<K_F64>()) != FT_OK ||
        (rc = preload_flagged_k<K_B1>()) != FT_OK || (rc = preload_flagged_k<K_B4>()) != FT_OK)
        return rc;
    return preload_flagged_k<K_B8>();
}

}  // namespace ftv
