// knn_launch.cuh -- launcher of the traversal kernel for one padded width DP;
// explicit instantiations live in knn_lo.cu (DP 2, 3, 4) and knn_hi.cu
// (DP 8, 10, 16) so the translation units compile in parallel.
#pragma once

#include "query.cuh"
#include "runtime.h"

namespace panda {

template <int DP, int KC>
static panda_status launch_knn_t(const KnnArgs& a, cudaStream_t s)
{
    const long long warps = (a.m + 31) / 32;
    const long long blocks = (warps + 3) / 4;
    k_knn<DP, KC><<<(unsigned)blocks, 128, 0, s>>>(a);
    PANDA_LAUNCHED("k_knn");
    return PANDA_OK;
}

// Top-k capacity classes: the smallest class >= k is used (unused slots hold
// sentinels below every key, so results do not depend on the class).
template <int DP>
panda_status launch_knn_dp(const KnnArgs& a, int kc, cudaStream_t s)
{
    switch (kc) {
        case 4: return launch_knn_t<DP, 4>(a, s);
        case 8: return launch_knn_t<DP, 8>(a, s);
        case 12: return launch_knn_t<DP, 12>(a, s);
        case 16: return launch_knn_t<DP, 16>(a, s);
        case 24: return launch_knn_t<DP, 24>(a, s);
        case 32: return launch_knn_t<DP, 32>(a, s);
        case 48: return launch_knn_t<DP, 48>(a, s);
        default: return launch_knn_t<DP, 64>(a, s);
    }
}

}  // namespace panda
