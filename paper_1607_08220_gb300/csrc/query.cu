// query.cu -- KNN query host path: query ordering and traversal dispatch.
//
// Algorithm 1 is run for many queries at once (the paper parallelises over
// queries, Sec. V-B2).  To make the 32 queries of a warp traverse nearly the
// same nodes, queries are first grouped by a spatial key with one counting
// sort: either the leaf bucket the query falls into (descending the tree by
// its split planes) or a 30-bit Morton code over the tree's root box.  The
// order only changes which queries share a warp, never a result.  Dense
// leaf-ordered sets (m >= n/2) then hand each warp one bin's queries (a job
// list), and the all-points query (knn_self) takes the tree's own packed
// points, one leaf per warp, with no ordering pass at all.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "order.cuh"
#include "query.cuh"
#include "runtime.h"

namespace panda {

__device__ __forceinline__ unsigned morton_key(const OrderArgs& a, const float* q)
{
    unsigned code = 0;
    unsigned cell[kMaxDim];
    const unsigned top = (1u << a.bits) - 1u;
    for (int k = 0; k < a.d; k++) {
        float u = (q[k] - a.lo[k]) * a.inv[k];
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        unsigned c = (unsigned)(u * (float)top);
        cell[k] = c > top ? top : c;
    }
    for (int b = a.bits - 1; b >= 0; b--)
        for (int k = 0; k < a.d; k++) code = (code << 1) | ((cell[k] >> b) & 1u);
    return code;
}

__global__ void k_order_keys(OrderArgs a)
{
    griddep_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    const float* q = a.queries + i * a.d;
    unsigned key;
    if (a.mode == PANDA_ORDER_MORTON) {
        key = morton_key(a, q) >> a.shift;
    } else {
        int node = 0, set = 0;
        if (a.qset_off) {
            int lo = 0, hi = a.nsets - 1;        // last set whose first row <= i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.qset_off[mid] <= i) lo = mid; else hi = mid - 1;
            }
            set = lo;
            node = set;
        }
        for (int step = 0; step <= kMaxDepth + 1; step++) {
            if ((unsigned)node >= (unsigned)a.num_nodes) {
                node = 0;
                break;
            }
            const int4 h = __ldg(reinterpret_cast<const int4*>(a.nodes + (long long)node * a.ns));
            const unsigned meta = (unsigned)h.w;
            if (meta & kMetaLeaf) break;
            if (meta & kMetaIndex) {
                node = h.x;
            } else {
                const float s = __int_as_float(h.z);
                node = h.x + (q[meta & kMetaDimMask] >= s ? 1 : 0);
            }
        }
        const int4 h = __ldg(reinterpret_cast<const int4*>(a.nodes + (long long)node * a.ns));
        key = a.qset_off ? (unsigned)a.set_bin[set] + ((unsigned)(h.x - a.set_poff[set]) >> a.shift)
                         : (unsigned)h.x >> a.shift;
    }
    a.keys[i] = key;
    atomicAdd(&a.hist[key], 1);
}

// Exclusive scan of hist[0..nb) in blocks of 4096; block sums to bsum.
__global__ void k_scan_blocks(int* hist, int nb, int* bsum)
{
    griddep_enter();
    __shared__ int sh[33];
    const int base = blockIdx.x * 4096 + threadIdx.x * 4;
    int v[4], t = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        v[e] = base + e < nb ? hist[base + e] : 0;
        t += v[e];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = warp_incl_scan(t);
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = sh[lane];
        int wi = warp_incl_scan(w);
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    int run = sh[warp] + incl - t;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        if (base + e < nb) hist[base + e] = run;
        run += v[e];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = sh[32];
}

__global__ void k_scan_sums(int* bsum, int nblocks)
{
    griddep_enter();
    __shared__ int sh[33];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nblocks; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int v = i < nblocks ? bsum[i] : 0;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int incl = warp_incl_scan(v);
        if (lane == 31) sh[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
            int wi = warp_incl_scan(w);
            sh[lane] = wi - w;
            if (lane == 31) sh[32] = wi;
        }
        __syncthreads();
        if (i < nblocks) bsum[i] = carry + sh[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += sh[32];
        __syncthreads();
    }
}

__global__ void k_order_scatter(const unsigned* keys, long long m, int* cursor, const int* bsum, int* perm)
{
    griddep_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const unsigned key = keys[i];
    const int p = atomicAdd(&cursor[key], 1) + bsum[key >> 12];
    perm[p] = (int)i;
}

// Jobs of a leaf-ordered query set: the queries of each bin (after the
// counting sort, bin b holds positions [end(b - 1), end(b)), end(b) =
// bsum[b >> 12] + cursor[b]), in pieces of at most 32.  One atomic per warp.
__global__ void k_bin_jobs(const int* cursor, const int* bsum, int nb, int2* jobs, int* njobs, long long cap,
                           unsigned* err)
{
    griddep_enter();
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int start = 0, count = 0;
    if (b < nb) {
        const int end = bsum[b >> 12] + cursor[b];
        start = b > 0 ? bsum[(b - 1) >> 12] + cursor[b - 1] : 0;
        count = end - start;
    }
    const int nj = (count + 31) >> 5;
    const int incl = warp_incl_scan(nj);
    int base = 0;
    if (lane == 31 && incl > 0) base = atomicAdd(njobs, incl);
    base = __shfl_sync(kFull, base, 31) + incl - nj;
    if (base + nj > cap) {
        atomicOr(err, kErrInternal);
        return;
    }
    for (int j = 0; j < nj; j++) jobs[base + j] = make_int2(start + 32 * j, min(32, count - 32 * j));
}

// Key of the search radius: (max_d2 bits, 0xffffffff) -- every point with
// d2 <= max_d2 has a smaller key (ids < 2^31); 0 when the query is unbounded.
static unsigned long long radius_key(const panda_query_params* params)
{
    if (!params || !params->bounded) return 0ull;
    unsigned bits;
    const float r2 = params->max_d2 + 0.0f;   // -0 -> +0
    memcpy(&bits, &r2, 4);
    return ((unsigned long long)bits << 32) | 0xffffffffull;
}

// Radius parameters are valid: unbounded, or max_d2 >= 0 (not NaN).
static panda_status check_radius(const panda_query_params* params, bool counters, const char* what)
{
    if (!params || !params->bounded) return PANDA_OK;
    if (!(params->max_d2 >= 0.0f)) {
        set_error("%s: max_d2 must be >= 0", what);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (counters) {
        set_error("%s: work counters are not kept for radius-bounded queries", what);
        return PANDA_ERR_UNSUPPORTED;
    }
    return PANDA_OK;
}

template <int DP>
panda_status launch_knn_dp(const KnnArgs& a, cudaStream_t s);

static panda_status launch_knn(const KnnArgs& a, int dp, cudaStream_t s)
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

panda_status knn_query(const panda_tree* t, const float* queries, int64_t m, int32_t k, int32_t* ids,
                       float* d2, const panda_query_params* params, cudaStream_t stream,
                       unsigned* host_err, int32_t* visits, unsigned long long* stats)
{
    if (host_err) *host_err = 0;
    if (!t || m < 0 || k < 1 || (m > 0 && (!queries || !ids || !d2))) {
        set_error("panda_knn: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (k > kMaxK) {
        set_error("panda_knn: k=%d above the maximum %d", k, kMaxK);
        return PANDA_ERR_UNSUPPORTED;
    }
    if (m >= (1LL << 31)) {
        set_error("panda_knn: m=%lld too large", (long long)m);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (m == 0) return PANDA_OK;
    if (!is_device_ptr(queries) || !is_device_ptr(ids) || !is_device_ptr(d2)) {
        set_error("panda_knn: queries and outputs must be device pointers");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    {
        const panda_status rs = check_radius(params, visits || stats, "panda_knn");
        if (rs != PANDA_OK) return rs;
    }
    const int order = params ? params->order : PANDA_ORDER_LEAF;
    if (order < PANDA_ORDER_NONE || order > PANDA_ORDER_LEAF) {
        set_error("panda_knn: unknown order %d", order);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    PhaseTimer timer(stream);
    std::vector<void*> ws;
    auto cleanup = [&]() {
        for (void* p : ws) ws_free(p, stream);
    };
    panda_status st;
    auto get = [&](void** p, size_t bytes, const char* what) -> panda_status {
        panda_status r = ws_alloc(p, bytes, stream, what);
        if (r == PANDA_OK) ws.push_back(*p);
        return r;
    };
    unsigned* err = nullptr;
    if ((st = get((void**)&err, sizeof(unsigned), "query error word")) != PANDA_OK) return cleanup(), st;
    cudaError_t ce = cudaMemsetAsync(err, 0, sizeof(unsigned), stream);
    if (ce != cudaSuccess) return cleanup(), cuda_fail(ce, "clear query error");
    int* perm = nullptr;
    const int traversal = params ? params->traversal : PANDA_TRAVERSAL_AUTO;
    const int solo = traversal == PANDA_TRAVERSAL_PER_QUERY ? 1
                     : traversal == PANDA_TRAVERSAL_PACKET  ? 0
                                                            : prefer_per_query(m, t->n, t->d);
    // dense leaf-ordered packets: one leaf's queries per warp (as the
    // all-points query), so no packet straddles two leaves
    int2* jobs = nullptr;
    int* njobs = nullptr;
    long long jobs_cap = 0;
    if (order != PANDA_ORDER_NONE && m > 32) {
        timer.begin("query.order");
        OrderArgs oa;
        memset(&oa, 0, sizeof(oa));
        oa.nodes = t->nodes;
        oa.num_nodes = t->node_slots;
        oa.queries = queries;
        oa.m = m;
        oa.d = t->d;
        oa.ns = t->ns;
        oa.mode = order;
        int nb;
        if (order == PANDA_ORDER_MORTON) {
            oa.bits = std::max(1, std::min(10, 30 / t->d));
            const int total = oa.bits * t->d;
            oa.shift = std::max(0, total - 20);
            nb = 1 << (total - oa.shift);
            for (int j = 0; j < t->d; j++) {
                oa.lo[j] = t->root_lo[j];
                float w = t->root_hi[j] - t->root_lo[j];
                oa.inv[j] = w > 0.0f ? 1.0f / w : 0.0f;
            }
        } else {
            // about four bins per query (at least 4096, at most 2^22): the
            // histogram scan then costs no more than the queries themselves
            const long long want = std::max<long long>(4096, std::min<long long>(1LL << 22, 4 * m));
            int sh = 0;
            while (((long long)t->n >> sh) > want) sh++;
            oa.shift = sh;
            nb = (int)(((long long)t->n >> sh) + 1);
        }
        const int nblk = (nb + 4095) / 4096;
        unsigned* keys = nullptr;
        int *hist = nullptr, *bsum = nullptr;
        if ((st = get((void**)&keys, (size_t)m * 4, "order keys")) != PANDA_OK) return cleanup(), st;
        if ((st = get((void**)&perm, (size_t)m * 4, "order permutation")) != PANDA_OK) return cleanup(), st;
        if ((st = get((void**)&hist, (size_t)nblk * 4096 * 4, "order histogram")) != PANDA_OK) return cleanup(), st;
        if ((st = get((void**)&bsum, (size_t)nblk * 4, "order block sums")) != PANDA_OK) return cleanup(), st;
        oa.keys = keys;
        oa.hist = hist;
        ce = cudaMemsetAsync(hist, 0, (size_t)nb * 4, stream);
        if (ce != cudaSuccess) return cleanup(), cuda_fail(ce, "clear order histogram");
        const unsigned gb = (unsigned)((m + 255) / 256);
        if ((st = launch_k("k_order_keys", k_order_keys, gb, 256, 0, stream, oa)) != PANDA_OK) return cleanup(), st;
        if ((st = launch_k("k_scan_blocks", k_scan_blocks, nblk, 1024, 0, stream, hist, nb, bsum)) != PANDA_OK)
            return cleanup(), st;
        if ((st = launch_k("k_scan_sums", k_scan_sums, 1, 1024, 0, stream, bsum, nblk)) != PANDA_OK)
            return cleanup(), st;
        if ((st = launch_k("k_order_scatter", k_order_scatter, gb, 256, 0, stream, (const unsigned*)keys, (long long)m,
                           hist, (const int*)bsum, perm)) != PANDA_OK)
            return cleanup(), st;
        if (order == PANDA_ORDER_LEAF && !solo && 2 * m >= t->n) {
            jobs_cap = nb + m / 32 + 1;
            void* jp = nullptr;
            if ((st = get(&jp, 16 + (size_t)jobs_cap * sizeof(int2), "query jobs")) != PANDA_OK) return cleanup(), st;
            njobs = static_cast<int*>(jp);
            jobs = reinterpret_cast<int2*>(static_cast<char*>(jp) + 16);
            ce = cudaMemsetAsync(njobs, 0, sizeof(int), stream);
            if (ce != cudaSuccess) return cleanup(), cuda_fail(ce, "clear query jobs");
            if ((st = launch_k("k_bin_jobs", k_bin_jobs, (unsigned)((nb + 255) / 256), 256, 0, stream,
                               (const int*)hist, (const int*)bsum, nb, jobs, njobs, jobs_cap, err)) != PANDA_OK)
                return cleanup(), st;
        }
    }
    timer.begin("query.traverse");
    KnnArgs ka;
    memset(&ka, 0, sizeof(ka));
    ka.nodes = t->nodes;
    ka.pts = t->points;
    ka.queries = queries;
    ka.perm = perm;
    ka.ids = ids;
    ka.d2 = d2;
    ka.err = err;
    ka.m = m;
    ka.num_nodes = t->node_slots;
    ka.npts = t->n;
    ka.visits = visits;
    ka.stats = stats;
    ka.transpose_max = (params && params->transpose_max != 0) ? params->transpose_max : kTransposeMaxDefault;
    ka.solo = solo;
    ka.rkey = radius_key(params);
    ka.pos_jobs = jobs;
    ka.pos_njobs = njobs;
    ka.pos_jobs_cap = jobs_cap;
    ka.d = t->d;
    ka.k = k;
    st = launch_knn(ka, t->dp, stream);
    if (st != PANDA_OK) return cleanup(), st;
    note_tree_use(t, stream);
    timer.end();
    if (host_err) {
        ce = cudaMemcpyAsync(host_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) return cleanup(), cuda_fail(ce, "query");
    }
    cleanup();
    timer.finish();
    return PANDA_OK;
}

// Jobs of the all-points query: every leaf, in pieces of at most 32 points
// (one warp each), listed in position order to 1,024-point granularity so the
// warps in flight at any time work on one region of the tree (L2 reuse): a
// counting sort of the leaves by start >> 10.  Node slots that are not leaves
// (inner nodes, holes with an all-zero header) are skipped.
__device__ __forceinline__ bool leaf_of_slot(const float4* nodes, long long i, int ns, int& start, int& count)
{
    const int4 h = __ldg(reinterpret_cast<const int4*>(nodes + i * ns));
    start = h.x;
    count = h.y;
    return ((unsigned)h.w & kMetaLeaf) && h.y > 0;
}

// Pass 1: jobs per 1,024-position bin, and the total (one atomic per warp).
__global__ void k_pos_jobs_count(const float4* nodes, long long slots, int ns, int* hist, int* njobs)
{
    griddep_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int start = 0, count = 0, nj = 0;
    if (i < slots && leaf_of_slot(nodes, i, ns, start, count)) {
        nj = (count + 31) >> 5;
        atomicAdd(&hist[start >> 10], nj);
    }
    const int tot = warp_sum(nj);
    if ((threadIdx.x & 31) == 0 && tot > 0) atomicAdd(njobs, tot);
}

// Pass 2 (after the scan of hist into cursor offsets + bsum): place each
// leaf's jobs at its bin's next free slots.
__global__ void k_pos_jobs_place(const float4* nodes, long long slots, int ns, int* cursor, const int* bsum,
                                 int2* jobs, long long cap, unsigned* err)
{
    griddep_enter();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int start = 0, count = 0;
    if (i >= slots || !leaf_of_slot(nodes, i, ns, start, count)) return;
    const int nj = (count + 31) >> 5;
    const int key = start >> 10;
    const long long base = (long long)atomicAdd(&cursor[key], nj) + bsum[key >> 12];
    if (base + nj > cap) {
        atomicOr(err, kErrInternal);
        return;
    }
    for (int j = 0; j < nj; j++) jobs[base + j] = make_int2(start + 32 * j, min(32, count - 32 * j));
}

panda_status knn_self(const panda_tree* t, int32_t k, int32_t* ids, float* d2, const panda_query_params* params,
                      cudaStream_t stream, unsigned* host_err, int32_t* visits, unsigned long long* stats)
{
    if (host_err) *host_err = 0;
    if (!t || k < 1 || !ids || !d2) {
        set_error("panda_knn_self: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (k > kMaxK) {
        set_error("panda_knn_self: k=%d above the maximum %d", k, kMaxK);
        return PANDA_ERR_UNSUPPORTED;
    }
    if (!is_device_ptr(ids) || !is_device_ptr(d2)) {
        set_error("panda_knn_self: outputs must be device pointers");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    {
        const panda_status rs = check_radius(params, visits || stats, "panda_knn_self");
        if (rs != PANDA_OK) return rs;
    }
    PhaseTimer timer(stream);
    // scratch: error word, job counter, jobs (at most one per leaf plus one per
    // 32 points), the bin histogram (bins of 1,024 positions) and its block sums
    const long long cap = t->num_leaves + t->n / 32 + 1;
    const int nb = (int)(t->n >> 10) + 1;
    const int nblk = (nb + 4095) / 4096;
    const size_t hist_off = 16 + (size_t)cap * sizeof(int2);
    const size_t bytes = hist_off + ((size_t)nblk * 4096 + nblk) * sizeof(int);
    void* scratch = nullptr;
    panda_status st = ws_alloc(&scratch, bytes, stream, "self-query jobs");
    if (st != PANDA_OK) return st;
    unsigned* err = static_cast<unsigned*>(scratch);
    int* njobs = reinterpret_cast<int*>(static_cast<char*>(scratch) + 4);
    int2* jobs = reinterpret_cast<int2*>(static_cast<char*>(scratch) + 16);
    int* hist = reinterpret_cast<int*>(static_cast<char*>(scratch) + hist_off);
    int* bsum = hist + (size_t)nblk * 4096;
    cudaError_t ce = cudaMemsetAsync(scratch, 0, 16, stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(hist, 0, (size_t)nb * sizeof(int), stream);
    if (ce != cudaSuccess) {
        ws_free(scratch, stream);
        return cuda_fail(ce, "clear query error");
    }
    timer.begin("query.jobs");
    const unsigned gs = (unsigned)((t->node_slots + 255) / 256);
    st = launch_k("k_pos_jobs_count", k_pos_jobs_count, gs, 256, 0, stream, (const float4*)t->nodes,
                  (long long)t->node_slots, t->ns, hist, njobs);
    if (st == PANDA_OK) st = launch_k("k_scan_blocks", k_scan_blocks, nblk, 1024, 0, stream, hist, nb, bsum);
    if (st == PANDA_OK) st = launch_k("k_scan_sums", k_scan_sums, 1, 1024, 0, stream, bsum, nblk);
    if (st == PANDA_OK)
        st = launch_k("k_pos_jobs_place", k_pos_jobs_place, gs, 256, 0, stream, (const float4*)t->nodes,
                      (long long)t->node_slots, t->ns, hist, (const int*)bsum, jobs, cap, err);
    if (st != PANDA_OK) {
        ws_free(scratch, stream);
        return st;
    }
    timer.begin("query.traverse");
    KnnArgs ka;
    memset(&ka, 0, sizeof(ka));
    ka.nodes = t->nodes;
    ka.pts = t->points;
    ka.ids = ids;
    ka.d2 = d2;
    ka.err = err;
    ka.m = t->n;
    ka.num_nodes = t->node_slots;
    ka.npts = t->n;
    ka.self_q = 1;
    ka.pos_jobs = jobs;
    ka.pos_njobs = njobs;
    ka.pos_jobs_cap = cap;
    ka.visits = visits;
    ka.stats = stats;
    ka.transpose_max = (params && params->transpose_max != 0) ? params->transpose_max : kTransposeMaxDefault;
    ka.solo = (params && params->traversal == PANDA_TRAVERSAL_PER_QUERY) ? 1 : 0;
    ka.rkey = radius_key(params);
    ka.d = t->d;
    ka.k = k;
    st = launch_knn(ka, t->dp, stream);
    if (st == PANDA_OK) note_tree_use(t, stream);
    timer.end();
    if (st == PANDA_OK && host_err) {
        ce = cudaMemcpyAsync(host_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) st = cuda_fail(ce, "query");
    }
    ws_free(scratch, stream);
    if (st == PANDA_OK) timer.finish();
    return st;
}

}  // namespace panda
