// tune.cu -- autotuner for the knobs that change speed but never results.
//
// Knobs: the bucket size B (the paper found 32 best on its CPUs, Sec.
// III-A1 "Choice of bucket size"), the query ordering (none, Morton, leaf)
// and the leaf-scan shape switch (how many of a warp's 32 queries must need a
// bucket before the warp scans it lanes=queries instead of lanes=points, i.e.
// how a warp's query group shares the scan).  Every candidate is timed with
// CUDA events on the caller's points and a sample of its queries; the score
// is build time + query time scaled to the expected number of queries per
// build.  Results are cached per (d, ceil(log2 n), k, log2 of the queries per
// build) for the life of the process.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace panda {
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, panda_tune_result> g_tune_cache;

std::tuple<int, int, int, int> tune_key(int d, int64_t n, int k, int64_t m_total)
{
    const int ln = (int)ceil(log2((double)std::max<int64_t>(n, 1)));
    const int lm = (int)ceil(log2((double)std::max<int64_t>(m_total, 1)));
    return std::make_tuple(d, ln, k, lm);
}

panda_status time_ms(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms)
{
    PANDA_CUDA(cudaEventSynchronize(e1), "tune: sync");
    PANDA_CUDA(cudaEventElapsedTime(ms, e0, e1), "tune: elapsed");
    (void)s;
    return PANDA_OK;
}

}  // namespace
}  // namespace panda

using namespace panda;

extern "C" {

panda_status panda_tune(const float* points, int64_t n, int32_t d, const float* queries, int64_t m_sample,
                        int64_t m_total, int32_t k, void* stream, panda_tune_result* out)
{
    clear_error();
    if (!points || !queries || !out || n < 1 || d < 1 || m_sample < 1 || m_total < 1 || k < 1) {
        set_error("panda_tune: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (d > kMaxDim || k > kMaxK) {
        set_error("panda_tune: unsupported d or k");
        return PANDA_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int buckets[] = {16, 32, 64};
    const int orders[] = {PANDA_ORDER_NONE, PANDA_ORDER_MORTON, PANDA_ORDER_LEAF};
    // scan-shape switches of the packet traversal, then the per-query traversal
    const int shapes[] = {-1, 4, 8, 12, 16, 32, 0};
    void *ids = nullptr, *d2 = nullptr;
    panda_status st = ws_alloc(&ids, (size_t)m_sample * k * 4, s, "tune ids");
    if (st == PANDA_OK) st = ws_alloc(&d2, (size_t)m_sample * k * 4, s, "tune distances");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == PANDA_OK) {
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) st = cuda_fail(e, "tune: events");
    }
    panda_tune_result best;
    memset(&best, 0, sizeof(best));
    best.score_ms = INFINITY;
    const double scale = (double)m_total / (double)m_sample;
    for (int bi = 0; st == PANDA_OK && bi < 3; bi++) {
        panda_tree* t = nullptr;
        // warm the allocator and caches with one build, then time another
        st = build_tree(points, n, d, buckets[bi], s, &t);
        if (st != PANDA_OK) break;
        panda_free(t);
        t = nullptr;
        cudaEventRecord(e0, s);
        st = build_tree(points, n, d, buckets[bi], s, &t);
        cudaEventRecord(e1, s);
        float bms = 0.0f;
        if (st == PANDA_OK) st = time_ms(s, e0, e1, &bms);
        for (int oi = 0; st == PANDA_OK && oi < 3; oi++) {
            for (int si = 0; st == PANDA_OK && si < 7; si++) {
                panda_query_params prm;
                memset(&prm, 0, sizeof(prm));
                prm.order = orders[oi];
                prm.transpose_max = shapes[si];
                prm.traversal = si == 6 ? PANDA_TRAVERSAL_PER_QUERY : PANDA_TRAVERSAL_PACKET;
                float qms = 0.0f;
                for (int rep = 0; rep < 2 && st == PANDA_OK; rep++) {   // second run is timed
                    cudaEventRecord(e0, s);
                    st = knn_query(t, queries, m_sample, k, (int32_t*)ids, (float*)d2, &prm, s, nullptr);
                    cudaEventRecord(e1, s);
                    if (st == PANDA_OK) st = time_ms(s, e0, e1, &qms);
                }
                if (st != PANDA_OK) break;
                const double score = bms + qms * scale;
                if (score < best.score_ms) {
                    best.bucket = buckets[bi];
                    best.order = orders[oi];
                    best.transpose_max = shapes[si];
                    best.traversal = prm.traversal;
                    best.build_ms = bms;
                    best.query_ms = (float)(qms * scale);
                    best.score_ms = (float)score;
                }
            }
        }
        panda_free(t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ws_free(ids, s);
    ws_free(d2, s);
    if (st != PANDA_OK) return st;
    *out = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(d, n, k, m_total)] = best;
    return PANDA_OK;
}

panda_status panda_tune_lookup(int32_t d, int64_t n, int32_t k, int64_t m_total, panda_tune_result* out)
{
    if (!out) return PANDA_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(d, n, k, m_total));
    if (it == g_tune_cache.end()) {
        set_error("panda_tune_lookup: no tuned entry for d=%d n=%lld k=%d", d, (long long)n, k);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    *out = it->second;
    return PANDA_OK;
}

}  // extern "C"
