// knn_launch.cuh -- launcher of the traversal kernel for one padded width DP;
// explicit instantiations live in knn_lo.cu (DP 2, 3, 4) and knn_hi.cu
// (DP 8, 10, 16) so the translation units compile in parallel.
#pragma once

#include "query.cuh"
#include "runtime.h"

namespace panda {

template <int DP>
panda_status configure_knn()
{
    static bool configured = false;
    if (!configured) {
        PANDA_CUDA(cudaFuncSetAttribute(k_knn<DP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kMaxK * kKnnThreads * 8),
                   "configure k_knn");
        PANDA_CUDA(cudaFuncSetAttribute(k_knn<DP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kMaxK * kKnnThreads * 8),
                   "configure k_knn");
        configured = true;
    }
    return PANDA_OK;
}

template <int DP>
panda_status launch_knn_dp(const KnnArgs& a, cudaStream_t s)
{
    panda_status st = configure_knn<DP>();
    if (st != PANDA_OK) return st;
    // one launch per tree: one warp per 32 queries; many sets: persistent
    // warps (8 blocks per SM) draining the job queue
    const long long warps = (a.m + 31) / 32;
    const long long blocks = a.jobs ? (long long)num_sms() * 8
                                    : (warps + kKnnThreads / 32 - 1) / (kKnnThreads / 32);
    if (blocks <= 0) return PANDA_OK;
    const size_t heap_bytes = (size_t)a.k * kKnnThreads * 8;
    if (a.jobs || a.solo)
        k_knn<DP, true><<<(unsigned)blocks, kKnnThreads, heap_bytes, s>>>(a);
    else
        k_knn<DP, false><<<(unsigned)blocks, kKnnThreads, heap_bytes, s>>>(a);
    PANDA_LAUNCHED("k_knn");
    return PANDA_OK;
}

}  // namespace panda
