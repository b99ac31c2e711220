// knn_launch.cuh -- launcher of the traversal kernel for one padded width DP;
// explicit instantiations live in knn_lo.cu (DP 2, 3, 4) and knn_hi.cu
// (DP 8, 10, 16) so the translation units compile in parallel.
#pragma once

#include "query.cuh"
#include "runtime.h"

namespace panda {

template <int DP, int MODE, bool SOLO>
panda_status configure_knn_variant()
{
    PANDA_CUDA(cudaFuncSetAttribute(k_knn<DP, MODE, SOLO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (kMaxK + 1) * kKnnThreads * 8),
               "configure k_knn");
    return PANDA_OK;
}

// Resident blocks per SM of the multi-set kernel, [solo][k], filled by
// configure_knn (before any graph capture, so a captured launch needs no query).
template <int DP>
int (&multi_blocks_per_sm())[2][kMaxK + 1]
{
    static int t[2][kMaxK + 1];
    return t;
}

template <int DP, bool SOLO>
panda_status fill_multi_blocks()
{
    for (int k = 1; k <= kMaxK; k++) {
        int v = 0;
        PANDA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_knn<DP, kKnnManySets, SOLO>, kKnnThreads,
                                                                 (size_t)(k + 1) * kKnnThreads * 8),
                   "k_knn occupancy");
        multi_blocks_per_sm<DP>()[SOLO ? 1 : 0][k] = v > 0 ? v : 1;
    }
    return PANDA_OK;
}

template <int DP>
panda_status configure_knn()
{
    static PerDeviceOnce once;
    return once_per_device(once, [] {
        panda_status st = configure_knn_variant<DP, kKnnOneSet, false>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnOneSet, true>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnOneTreeReqs, false>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnOneTreeReqs, true>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnManySets, false>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnManySets, true>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnStats, false>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnStats, true>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnRadius, false>();
        if (st == PANDA_OK) st = configure_knn_variant<DP, kKnnRadius, true>();
        if (st == PANDA_OK) st = fill_multi_blocks<DP, false>();
        if (st == PANDA_OK) st = fill_multi_blocks<DP, true>();
        return st;
    });
}

// Persistent launch of the multi-set kernel: as many blocks as can be resident.
template <int DP, bool SOLO>
panda_status launch_knn_multi(const KnnArgs& a, size_t heap_bytes, cudaStream_t s)
{
    const int per_sm = multi_blocks_per_sm<DP>()[SOLO ? 1 : 0][std::min(std::max(a.k, 1), kMaxK)];
    const long long blocks = (long long)num_sms() * per_sm;
    PANDA_LAUNCH((k_knn<DP, kKnnManySets, SOLO>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
    return PANDA_OK;
}

// a.jobs selects the multi-set kernel, a.reqs the one-tree kernel with the
// per-lane request lookup; a.solo = 1 compiles in the per-query traversal
// (for a multi-set launch: some set has its solo flag set).
template <int DP>
panda_status launch_knn_dp(const KnnArgs& a, cudaStream_t s)
{
    panda_status st = configure_knn<DP>();
    if (st != PANDA_OK) return st;
    const size_t heap_bytes = (size_t)(a.k + 1) * kKnnThreads * 8;   // heap + sentinel row
    if (a.jobs) {
        if (a.njobs <= 0) return PANDA_OK;
        return a.solo ? launch_knn_multi<DP, true>(a, heap_bytes, s) : launch_knn_multi<DP, false>(a, heap_bytes, s);
    }
    // one launch per tree: one warp per 32 queries (all-points query: per job)
    const long long warps = a.pos_jobs ? a.pos_jobs_cap : (a.m + 31) / 32;
    const long long blocks = (warps + kKnnThreads / 32 - 1) / (kKnnThreads / 32);
    if (blocks <= 0) return PANDA_OK;
    if (a.rkey) {
        if (a.solo)
            PANDA_LAUNCH((k_knn<DP, kKnnRadius, true>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
        else
            PANDA_LAUNCH((k_knn<DP, kKnnRadius, false>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
    } else if (a.stats || a.visits) {
        if (a.solo)
            PANDA_LAUNCH((k_knn<DP, kKnnStats, true>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
        else
            PANDA_LAUNCH((k_knn<DP, kKnnStats, false>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
    } else if (a.reqs) {
        if (a.solo)
            PANDA_LAUNCH((k_knn<DP, kKnnOneTreeReqs, true>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
        else
            PANDA_LAUNCH((k_knn<DP, kKnnOneTreeReqs, false>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
    } else if (a.solo) {
        PANDA_LAUNCH((k_knn<DP, kKnnOneSet, true>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
    } else {
        PANDA_LAUNCH((k_knn<DP, kKnnOneSet, false>), (unsigned)blocks, kKnnThreads, heap_bytes, s, a);
    }
    return PANDA_OK;
}

}  // namespace panda
