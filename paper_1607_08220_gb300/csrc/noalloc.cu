// noalloc.cu -- a KNN query entry point that allocates no memory.
//
// Some callers cannot allocate device memory while they query: code that runs
// under an allocator it does not own (a host runtime that has reserved the
// whole device, or a framework whose memory pool must not be bypassed), or
// code that must never wait on, or fail in, an allocation on a latency path.
// panda_knn_noalloc serves them.  It orders the queries by leaf and runs the
// same traversal kernel as panda_knn_async, but the ordering's scratch space
// (query keys, permutation, histogram, error word) is one file-scope device
// array of fixed size, so the call performs no cudaMalloc, cudaMallocAsync or
// cudaFree and calls no allocating library routine.  The caller still passes
// the queries and the output buffers.  What it leaves out of
// panda_knn_async's path (no result depends on it): the histogram has at most
// 2^20 - 1 bins (2^22 there), and dense query sets (2m >= n) keep 32-query
// packets instead of the job list that gives each warp one bin's queries, so
// large batches against small trees run somewhat slower than through
// panda_knn_async.
//
// Limits and sharing:
//   * at most kNoAllocMaxQueries queries per call; larger m is rejected with
//     PANDA_ERR_UNSUPPORTED;
//   * the array lives on every device that loads the library, until exit;
//   * all calls share it and it keeps the last call's contents, so calls that
//     overlap on the GPU (concurrent streams, or two threads) race: the caller
//     must serialise them (one stream is enough);
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress, once per device with that device current); make
//     that first call before any stream capture.  The address is cached for
//     the life of the process: it does not survive cudaDeviceReset.
#include <string.h>

#include <mutex>

#include "order.cuh"
#include "query.cuh"
#include "runtime.h"

namespace panda {

constexpr long long kNoAllocMaxQueries = 1LL << 20;
constexpr int kNoAllocBins = 1 << 20;   // histogram bins (multiple of 4096)
constexpr size_t kNoAllocInts = 2 * (size_t)kNoAllocMaxQueries   // keys, permutation
                                + kNoAllocBins                    // histogram
                                + kNoAllocBins / 4096             // block sums
                                + 64;                             // error word (+ padding)

// The scratch space.  In host code this name is a host-side stand-in, not a
// device address: only the pointer from cudaGetSymbolAddress is passed to kernels.
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocInts];

template <int DP>
panda_status launch_knn_dp(const KnnArgs& a, cudaStream_t s);

namespace {

std::mutex g_scratch_mu;
int* g_scratch_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
panda_status scratch_on_current_device(int** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "panda_knn_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("panda_knn_noalloc: device %d out of range", dev);
        return PANDA_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "panda_knn_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = static_cast<int*>(p);
    }
    *out = g_scratch_ptr[dev];
    return PANDA_OK;
}

panda_status launch_traversal(const KnnArgs& a, int dp, cudaStream_t s)
{
    switch (dp) {
        case 2: return launch_knn_dp<2>(a, s);
        case 3: return launch_knn_dp<3>(a, s);
        case 4: return launch_knn_dp<4>(a, s);
        case 8: return launch_knn_dp<8>(a, s);
        case 10: return launch_knn_dp<10>(a, s);
        default: return launch_knn_dp<16>(a, s);
    }
}

}  // namespace
}  // namespace panda

using namespace panda;

static panda_status knn_noalloc_impl(const panda_tree* t, const float* queries, int64_t m, int32_t k,
                                     int32_t* out_ids, float* out_d2, void* stream)
{
    if (!t || m < 0 || k < 1 || (m > 0 && (!queries || !out_ids || !out_d2))) {
        set_error("panda_knn_noalloc: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (k > kMaxK) {
        set_error("panda_knn_noalloc: k=%d above the maximum %d", k, kMaxK);
        return PANDA_ERR_UNSUPPORTED;
    }
    if (m > kNoAllocMaxQueries) {
        set_error("panda_knn_noalloc: m=%lld exceeds the limit of %lld queries per call "
                  "(fixed scratch array; split the batch or use panda_knn_async)",
                  (long long)m, kNoAllocMaxQueries);
        return PANDA_ERR_UNSUPPORTED;
    }
    if (m == 0) return PANDA_OK;
    if (!is_device_ptr(queries) || !is_device_ptr(out_ids) || !is_device_ptr(out_d2)) {
        set_error("panda_knn_noalloc: queries and outputs must be device pointers");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    int* scratch = nullptr;
    panda_status st = scratch_on_current_device(&scratch);
    if (st != PANDA_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* keys = reinterpret_cast<unsigned*>(scratch);
    int* perm = scratch + kNoAllocMaxQueries;
    int* hist = perm + kNoAllocMaxQueries;
    int* bsum = hist + kNoAllocBins;
    unsigned* err = reinterpret_cast<unsigned*>(bsum + kNoAllocBins / 4096);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "panda_knn_noalloc: clear error word");
    const int* order = nullptr;
    if (m > 32) {
        // group queries by the leaf bucket they fall in (as panda_knn's default),
        // with the bucket key shifted so the bins fit the fixed histogram
        OrderArgs oa;
        memset(&oa, 0, sizeof(oa));
        oa.nodes = t->nodes;
        oa.num_nodes = t->node_slots;
        oa.queries = queries;
        oa.m = m;
        oa.d = t->d;
        oa.ns = t->ns;
        oa.mode = PANDA_ORDER_LEAF;
        const long long want = std::max<long long>(4096, std::min<long long>(kNoAllocBins - 1, 4 * m));
        int sh = 0;
        while (((long long)t->n >> sh) > want) sh++;
        oa.shift = sh;
        const int nb = (int)(((long long)t->n >> sh) + 1);
        const int nblk = (nb + 4095) / 4096;
        oa.keys = keys;
        oa.hist = hist;
        e = cudaMemsetAsync(hist, 0, (size_t)nb * sizeof(int), s);
        if (e != cudaSuccess) return cuda_fail(e, "panda_knn_noalloc: clear histogram");
        const unsigned gb = (unsigned)((m + 255) / 256);
        k_order_keys<<<gb, 256, 0, s>>>(oa);
        if ((st = note_launch("k_order_keys")) != PANDA_OK) return st;
        k_scan_blocks<<<nblk, 1024, 0, s>>>(hist, nb, bsum);
        if ((st = note_launch("k_scan_blocks")) != PANDA_OK) return st;
        k_scan_sums<<<1, 1024, 0, s>>>(bsum, nblk);
        if ((st = note_launch("k_scan_sums")) != PANDA_OK) return st;
        k_order_scatter<<<gb, 256, 0, s>>>(keys, m, hist, bsum, perm);
        if ((st = note_launch("k_order_scatter")) != PANDA_OK) return st;
        order = perm;
    }
    KnnArgs ka;
    memset(&ka, 0, sizeof(ka));
    ka.nodes = t->nodes;
    ka.pts = t->points;
    ka.queries = queries;
    ka.perm = order;
    ka.ids = out_ids;
    ka.d2 = out_d2;
    ka.err = err;
    ka.m = m;
    ka.num_nodes = t->node_slots;
    ka.npts = t->n;
    ka.d = t->d;
    ka.k = k;
    ka.transpose_max = kTransposeMaxDefault;
    ka.solo = prefer_per_query(m, t->n, t->d);
    return launch_traversal(ka, t->dp, s);
}

extern "C" panda_status panda_knn_noalloc(const panda_tree* t, const float* queries, int64_t m, int32_t k,
                                          int32_t* out_ids, float* out_d2, void* stream)
{
    clear_error();
    try {
        return knn_noalloc_impl(t, queries, m, k, out_ids, out_d2, stream);
    } catch (...) {   // e.g. std::system_error from the lock: no exception crosses the C ABI
        set_error("panda_knn_noalloc: host exception");
        return PANDA_ERR_OUT_OF_MEMORY;
    }
}
