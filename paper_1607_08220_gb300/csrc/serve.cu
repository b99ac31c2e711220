// serve.cu -- served form: resident trees and continuous batching of KNN
// requests (the paper pipelines query batches across stages, Sec. III-B).
//
// Trees stay resident in device memory; a tree is admitted only if the
// server's memory budget and the device's free memory hold it, and it is
// built on its own stream so queries keep running.  A scheduler thread forms
// batches from the request queue in arrival order -- requests of different
// trees, sizes and k -- and runs each batch as one ordering pass (one counting
// sort over all its queries, each request keyed by the leaves of its own
// tree) and one traversal launch; requests on the same tree are ordered
// together, so a warp's 32 queries may belong to several requests.  Up to four
// batches are in flight, each on its own stream (a small batch leaves most of
// the GPU idle, so batches overlap); requests that arrive while batches run
// join the next one as soon as a slot frees.  Each request records its submit
// and completion times.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "order.cuh"
#include "query.cuh"
#include "runtime.h"

namespace panda {
template <int DP>
panda_status launch_knn_dp(const KnnArgs& a, cudaStream_t s);

// Ordering of one request of a served batch against its own tree.
struct OrderSet {
    const float4* nodes;
    long long num_nodes;
    const float* queries;
    int root, bin_base, shift, ns, row_begin, d;
};

// Keys of all queries of a batch: row i belongs to the request whose rows start
// at row_begin[s] <= i; key = the request's first bin + (leaf start >> shift).
__global__ void k_order_keys_multi(const OrderSet* sets, const int* row_begin, int nsets, long long m,
                                   unsigned* keys, int* hist)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_begin[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const OrderSet S = sets[lo];
    const float* q = S.queries + (i - S.row_begin) * S.d;
    int node = S.root;
    for (int step = 0; step <= kMaxDepth + 1; step++) {
        if ((unsigned)node >= (unsigned)S.num_nodes) {
            node = S.root;
            break;
        }
        const int4 h = __ldg(reinterpret_cast<const int4*>(S.nodes + (long long)node * S.ns));
        const unsigned meta = (unsigned)h.w;
        if (meta & kMetaLeaf) break;
        node = (meta & kMetaIndex) ? h.x : h.x + (q[meta & kMetaDimMask] >= __int_as_float(h.z) ? 1 : 0);
    }
    const int4 h = __ldg(reinterpret_cast<const int4*>(S.nodes + (long long)node * S.ns));
    const unsigned key = (unsigned)S.bin_base + ((unsigned)h.x >> S.shift);
    keys[i] = key;
    atomicAdd(&hist[key], 1);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    int tree = 0;
    const float* queries = nullptr;
    int64_t m = 0;
    int k = 0;
    int32_t* ids = nullptr;
    float* d2 = nullptr;
    int64_t t_submit = 0, t_done = -1;
    int64_t batch = -1;
    panda_status status = PANDA_OK;
    bool done = false;
    bool waited = false;   // deferred at least once because its batch's scratch did not fit
};

struct InFlight {
    int64_t batch_id = 0;
    std::vector<int64_t> reqs;   // request ids; entry r owns error word 1 + r of the slot
    int slot = 0;                // pinned error region of this batch
    cudaEvent_t done = nullptr;
    std::vector<void*> scratch;
    int64_t reserved = 0;        // scratch bytes reserved for this batch
};

// Upper bound of the device scratch enqueue_batch allocates for a batch of m
// queries in nr requests over ng trees: keys and permutation (8 B a query),
// the counting-sort histogram (at most 4 bins a query + 64 per tree, rounded
// to whole 4,096-bin blocks) and its block sums, per-request descriptors and
// error words, and the job queue of the multi-tree launch; each allocation
// rounded up to the pool's 512-byte granularity.
int64_t batch_scratch_bound(int64_t m, int64_t nr, int64_t ng)
{
    const int64_t bins = std::min<int64_t>(4 * m + 64 * ng, (int64_t)ng << 20) + 4096;
    const int64_t bytes = 8 * m + 4 * bins + 4 * (bins / 4096 + 1) + nr * (int64_t)(sizeof(OrderSet) + sizeof(KnnReq) + 8) +
                          ng * (int64_t)sizeof(KnnSet) + 8 * (m / 32 + ng + 1) + 64;
    return bytes + 16 * 512;
}

}  // namespace

struct Server {
    int device = 0;
    int64_t budget = 0, used = 0;
    int64_t max_batch_queries = 0;
    // Batches in flight at most, each on its own stream: a small batch does
    // not fill the GPU, so batches run concurrently.
    static constexpr int kSlots = 4;
    int max_inflight = kSlots;
    // Pinned host copies of each in-flight batch's error words: [0] the
    // batch's (internal errors), [1 + r] request r's (non-finite query).
    unsigned* h_err[kSlots] = {};
    int h_err_cap[kSlots] = {};
    bool slot_busy[kSlots] = {};
    cudaStream_t qstream[kSlots] = {};
    cudaStream_t bstream = nullptr;
    std::vector<panda_tree*> trees;
    std::vector<int64_t> tree_bytes;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int64_t> pending;
    std::unordered_map<int64_t, Request> reqs;
    std::vector<InFlight> inflight;
    int64_t next_id = 1, next_batch = 0;
    int64_t batches = 0, batched_requests = 0;
    // Query batches are admitted by memory: each in-flight batch reserves an
    // upper bound of its device scratch; a batch starts only if that bound fits
    // both the budget left by the resident trees and the device's free memory
    // (memory the stream-ordered pool holds for reuse included).
    int64_t scratch_reserved = 0;
    int64_t deferred = 0;            // requests that waited for memory at least once
    int64_t pending_queries = 0;     // queries of requests not yet in a batch
    int64_t max_pending_queries = 0; // submit refuses beyond this (0: no limit)
    bool stop = false;
    std::thread sched;
    Clock::time_point t0;
    std::mutex build_mu;

    int64_t now_ns() const
    {
        return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
    }
};

namespace {

panda_status enqueue_batch(Server* S, const std::vector<Request*>& batch_in, InFlight& fl)
{
    cudaStream_t s = S->qstream[fl.slot];
    const int nr = (int)batch_in.size();
    // Requests on the same tree form one query set: their queries are sorted
    // together by the tree's leaves, so a warp's 32 queries may come from
    // several requests (each lane finds its own request by batch row).  Rows
    // are numbered group by group, so each group's sorted positions are one
    // contiguous range, and each group is one traversal launch.
    std::vector<int> group_tree;
    std::vector<std::vector<const Request*>> groups;
    for (const Request* R : batch_in) {
        size_t g = 0;
        while (g < group_tree.size() && group_tree[g] != R->tree) g++;
        if (g == group_tree.size()) {
            group_tree.push_back(R->tree);
            groups.emplace_back();
        }
        groups[g].push_back(R);
    }
    const int ng = (int)groups.size();
    fl.reqs.clear();
    for (int g = 0; g < ng; g++)
        for (const Request* R : groups[g]) fl.reqs.push_back(R->id);
    if (S->h_err_cap[fl.slot] < nr + 1) {
        if (S->h_err[fl.slot]) cudaFreeHost(S->h_err[fl.slot]);
        S->h_err[fl.slot] = nullptr;
        S->h_err_cap[fl.slot] = 0;
        const int cap = std::max(nr + 1, 1024);
        PANDA_CUDA(cudaHostAlloc((void**)&S->h_err[fl.slot], (size_t)cap * sizeof(unsigned), cudaHostAllocDefault),
                   "served error words");
        S->h_err_cap[fl.slot] = cap;
    }
    long long m_total = 0;
    std::vector<int> row_begin;
    std::vector<OrderSet> os;
    std::vector<KnnReq> kr;
    std::vector<long long> group_begin(ng + 1, 0), group_m(ng, 0);
    std::vector<int> group_req0(ng, 0), group_kmax(ng, 1);
    long long bins = 0;
    for (int g = 0; g < ng; g++) {
        const panda_tree* t = S->trees[group_tree[g]];
        long long mg = 0;
        for (const Request* R : groups[g]) mg += R->m;
        // bins of this tree: about 4 per query, at most 2^20, no finer than a point
        const long long want = std::min<long long>(1LL << 20, std::max<long long>(64, 4 * mg));
        int sh = 0;
        while ((t->n >> sh) + 1 > want) sh++;
        group_begin[g] = m_total;
        group_m[g] = mg;
        group_req0[g] = (int)kr.size();
        for (const Request* R : groups[g]) {
            row_begin.push_back((int)m_total);
            OrderSet o;
            o.nodes = t->nodes;
            o.num_nodes = t->node_slots;
            o.queries = R->queries;
            o.root = 0;
            o.bin_base = (int)bins;
            o.shift = sh;
            o.ns = t->ns;
            o.row_begin = (int)m_total;
            o.d = t->d;
            os.push_back(o);
            kr.push_back(KnnReq{R->queries, R->ids, R->d2, nullptr, R->k, (int)m_total});
            m_total += R->m;
            group_kmax[g] = std::max(group_kmax[g], R->k);
        }
        bins += (t->n >> sh) + 1;
    }
    group_begin[ng] = m_total;
    row_begin.push_back((int)m_total);
    const int nb = (int)bins;
    const int nblk = (nb + 4095) / 4096;
    auto get = [&](void** p, size_t bytes, const char* what) -> panda_status {
        panda_status st = ws_alloc(p, std::max<size_t>(bytes, 16), s, what);
        if (st == PANDA_OK) fl.scratch.push_back(*p);
        return st;
    };
    unsigned* keys;
    int *perm, *hist, *bsum, *rb;
    unsigned* err;
    OrderSet* d_os;
    KnnReq* d_kr;
    panda_status st;
    if ((st = get((void**)&keys, m_total * 4, "served keys")) != PANDA_OK) return st;
    if ((st = get((void**)&perm, m_total * 4, "served permutation")) != PANDA_OK) return st;
    if ((st = get((void**)&hist, (size_t)nblk * 4096 * 4, "served histogram")) != PANDA_OK) return st;
    if ((st = get((void**)&bsum, (size_t)nblk * 4, "served block sums")) != PANDA_OK) return st;
    if ((st = get((void**)&rb, (size_t)(nr + 1) * 4, "served row offsets")) != PANDA_OK) return st;
    if ((st = get((void**)&err, (size_t)(nr + 1) * 4, "served error words")) != PANDA_OK) return st;
    for (int r = 0; r < nr; r++) kr[r].err = err + 1 + r;
    if ((st = get((void**)&d_os, nr * sizeof(OrderSet), "served order sets")) != PANDA_OK) return st;
    if ((st = get((void**)&d_kr, nr * sizeof(KnnReq), "served requests")) != PANDA_OK) return st;
    PANDA_CUDA(cudaMemcpyAsync(rb, row_begin.data(), (nr + 1) * 4, cudaMemcpyHostToDevice, s), "served copy");
    PANDA_CUDA(cudaMemcpyAsync(d_os, os.data(), nr * sizeof(OrderSet), cudaMemcpyHostToDevice, s), "served copy");
    PANDA_CUDA(cudaMemcpyAsync(d_kr, kr.data(), nr * sizeof(KnnReq), cudaMemcpyHostToDevice, s), "served copy");
    PANDA_CUDA(cudaMemsetAsync(hist, 0, (size_t)nb * 4, s), "served clear");
    PANDA_CUDA(cudaMemsetAsync(err, 0, (size_t)(nr + 1) * 4, s), "served clear");
    if (m_total > 0) {
        const unsigned gb = (unsigned)((m_total + 255) / 256);
        k_order_keys_multi<<<gb, 256, 0, s>>>(d_os, rb, nr, m_total, keys, hist);
        PANDA_LAUNCHED("k_order_keys_multi");
        k_scan_blocks<<<nblk, 1024, 0, s>>>(hist, nb, bsum);
        PANDA_LAUNCHED("k_scan_blocks");
        k_scan_sums<<<1, 1024, 0, s>>>(bsum, nblk);
        PANDA_LAUNCHED("k_scan_sums");
        k_order_scatter<<<gb, 256, 0, s>>>(keys, m_total, hist, bsum, perm);
        PANDA_LAUNCHED("k_order_scatter");
        int any_solo = 0, kmax = 1;
        for (int g = 0; g < ng; g++) {
            const panda_tree* t = S->trees[group_tree[g]];
            any_solo |= prefer_per_query(group_m[g], t->n, t->d);
            kmax = std::max(kmax, group_kmax[g]);
        }
        if (ng > 1 || any_solo) {
            // several trees, or per-query traversal (lanes of very uneven
            // work): one persistent launch whose warps take (tree, 32 queries)
            // jobs from a device queue, so no launch waits on another's tail
            std::vector<KnnSet> ks(ng);
            std::vector<KnnJob> jobs;
            for (int g = 0; g < ng; g++) {
                const panda_tree* t = S->trees[group_tree[g]];
                KnnSet& K = ks[g];
                memset(&K, 0, sizeof(K));
                K.nodes = t->nodes;
                K.pts = t->points;
                K.num_nodes = t->node_slots;
                K.npts = t->n;
                K.perm = perm + group_begin[g];
                K.m = group_m[g];
                K.k = group_kmax[g];
                K.solo = prefer_per_query(group_m[g], t->n, t->d);
                K.nreq = (int)groups[g].size();
                K.reqs = d_kr + group_req0[g];
                for (long long p = 0; p < group_m[g]; p += 32) jobs.push_back(KnnJob{g, (int)p});
            }
            KnnSet* d_ks;
            KnnJob* d_jobs;
            int* head;
            if ((st = get((void**)&d_ks, ng * sizeof(KnnSet), "served query sets")) != PANDA_OK) return st;
            if ((st = get((void**)&d_jobs, std::max<size_t>(jobs.size(), 1) * sizeof(KnnJob), "served jobs")) !=
                PANDA_OK)
                return st;
            if ((st = get((void**)&head, 4, "served queue head")) != PANDA_OK) return st;
            PANDA_CUDA(cudaMemcpyAsync(d_ks, ks.data(), ng * sizeof(KnnSet), cudaMemcpyHostToDevice, s),
                       "served copy");
            PANDA_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(KnnJob), cudaMemcpyHostToDevice,
                                       s),
                       "served copy");
            PANDA_CUDA(cudaMemsetAsync(head, 0, 4, s), "served clear");
            KnnArgs ka;
            memset(&ka, 0, sizeof(ka));
            ka.sets = d_ks;
            ka.jobs = d_jobs;
            ka.njobs = (int)jobs.size();
            ka.job_head = head;
            ka.err = err;
            ka.m = m_total;
            ka.d = S->trees[group_tree[0]]->d;
            ka.k = kmax;
            ka.transpose_max = kTransposeMaxDefault;
            ka.solo = any_solo;
            switch (S->trees[group_tree[0]]->dp) {
                case 2: st = launch_knn_dp<2>(ka, s); break;
                case 3: st = launch_knn_dp<3>(ka, s); break;
                case 4: st = launch_knn_dp<4>(ka, s); break;
                case 8: st = launch_knn_dp<8>(ka, s); break;
                case 10: st = launch_knn_dp<10>(ka, s); break;
                default: st = launch_knn_dp<16>(ka, s); break;
            }
        }
        for (int g = 0; g < ng && st == PANDA_OK && !(ng > 1 || any_solo); g++) {
            // one tree, packet traversal: tree fields as kernel parameters
            if (group_m[g] == 0) continue;
            const panda_tree* t = S->trees[group_tree[g]];
            KnnArgs ka;
            memset(&ka, 0, sizeof(ka));
            ka.nodes = t->nodes;
            ka.pts = t->points;
            ka.num_nodes = t->node_slots;
            ka.npts = t->n;
            ka.perm = perm + group_begin[g];
            ka.err = err;
            ka.m = group_m[g];
            ka.d = t->d;
            ka.k = group_kmax[g];
            ka.transpose_max = kTransposeMaxDefault;
            ka.solo = prefer_per_query(group_m[g], t->n, t->d);
            ka.reqs = d_kr + group_req0[g];
            ka.nreq = (int)groups[g].size();
            switch (t->dp) {
                case 2: st = launch_knn_dp<2>(ka, s); break;
                case 3: st = launch_knn_dp<3>(ka, s); break;
                case 4: st = launch_knn_dp<4>(ka, s); break;
                case 8: st = launch_knn_dp<8>(ka, s); break;
                case 10: st = launch_knn_dp<10>(ka, s); break;
                default: st = launch_knn_dp<16>(ka, s); break;
            }
        }
        if (st != PANDA_OK) return st;
    }
    PANDA_CUDA(cudaMemcpyAsync(S->h_err[fl.slot], err, (size_t)(nr + 1) * 4, cudaMemcpyDeviceToHost, s),
               "served error words");
    PANDA_CUDA(cudaEventCreateWithFlags(&fl.done, cudaEventDisableTiming), "served event");
    PANDA_CUDA(cudaEventRecord(fl.done, s), "served event");
    return PANDA_OK;
}

void release(Server* S, InFlight& fl)
{
    for (void* p : fl.scratch) ws_free(p, S->qstream[fl.slot]);
    fl.scratch.clear();
    S->scratch_reserved -= fl.reserved;
    fl.reserved = 0;
    if (fl.done) cudaEventDestroy(fl.done);
    fl.done = nullptr;
    S->slot_busy[fl.slot] = false;
}

// Status of request r of a finished batch from its slot's error words.
panda_status request_status(const Server* S, const InFlight& fl, size_t r)
{
    const volatile unsigned* h = S->h_err[fl.slot];
    if (h[0] != 0) return PANDA_ERR_CUDA;
    if (h[1 + r] & kErrNonfinite) return PANDA_ERR_NONFINITE_INPUT;
    return h[1 + r] ? PANDA_ERR_CUDA : PANDA_OK;
}

// Bytes a new batch may reserve: the budget left by the resident trees and the
// batches in flight (no budget: unbounded), and the device's free memory plus
// what the stream-ordered pool holds unused, less what the batches in flight
// reserved and have not allocated yet (a bound: they may have allocated some).
int64_t scratch_available(Server* S)
{
    int64_t avail = INT64_MAX;
    if (S->budget > 0) avail = S->budget - S->used - S->scratch_reserved;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        int64_t dev = (int64_t)free_b;
        cudaMemPool_t pool;
        uint64_t reserved = 0, used = 0;
        if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            dev += (int64_t)(reserved - used);
        avail = std::min(avail, dev - S->scratch_reserved);
    }
    cudaGetLastError();
    return avail;
}

void scheduler(Server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // completions
        bool finished = false;
        for (size_t i = 0; i < S->inflight.size();) {
            InFlight& fl = S->inflight[i];
            const cudaError_t q = cudaEventQuery(fl.done);
            if (q == cudaErrorNotReady) {
                i++;
                continue;
            }
            const int64_t t = S->now_ns();
            for (size_t r = 0; r < fl.reqs.size(); r++) {
                Request& R = S->reqs[fl.reqs[r]];
                R.t_done = t;
                R.status = q == cudaSuccess ? request_status(S, fl, r) : PANDA_ERR_CUDA;
                R.done = true;
            }
            release(S, fl);
            S->inflight.erase(S->inflight.begin() + i);
            finished = true;
        }
        if (finished) S->cv.notify_all();
        if (S->stop && S->pending.empty() && S->inflight.empty()) break;
        bool start = !S->pending.empty() && (int)S->inflight.size() < S->max_inflight;
        std::vector<Request*> batch;
        std::vector<int64_t> ids;
        int64_t reserve = 0;
        if (start) {
            // next batch: requests in arrival order, same padded width, up to the
            // query cap, while the batch's scratch fits the memory available
            const int64_t avail = scratch_available(S);
            int64_t qsum = 0;
            std::vector<int> trees_in;
            const int dp = S->trees[S->reqs[S->pending.front()].tree]->dp;
            for (int64_t rid : S->pending) {
                Request& R = S->reqs[rid];
                if (S->trees[R.tree]->dp != dp) break;
                if (!batch.empty() && qsum + R.m > S->max_batch_queries) break;
                const bool new_tree = std::find(trees_in.begin(), trees_in.end(), R.tree) == trees_in.end();
                const int64_t need = batch_scratch_bound(qsum + R.m, (int64_t)batch.size() + 1,
                                                         (int64_t)trees_in.size() + (new_tree ? 1 : 0));
                if (need > avail) {
                    if (!R.waited) {
                        R.waited = true;
                        S->deferred++;
                    }
                    break;
                }
                batch.push_back(&R);
                ids.push_back(R.id);
                qsum += R.m;
                reserve = need;
                if (new_tree) trees_in.push_back(R.tree);
            }
            if (batch.empty()) {
                start = false;
                if (S->inflight.empty()) {
                    // nothing runs, so nothing will free memory: the first request
                    // can never fit; it fails instead of waiting forever
                    Request& R = S->reqs[S->pending.front()];
                    S->pending.pop_front();
                    S->pending_queries -= R.m;
                    R.status = PANDA_ERR_OUT_OF_MEMORY;
                    R.t_done = S->now_ns();
                    R.done = true;
                    S->cv.notify_all();
                    continue;
                }
            } else {
                for (size_t i = 0; i < batch.size(); i++) S->pending.pop_front();
                S->pending_queries -= qsum;
            }
        }
        if (start) {
            InFlight fl;
            fl.reserved = reserve;
            S->scratch_reserved += reserve;
            fl.batch_id = S->next_batch++;
            fl.reqs = ids;
            while (S->slot_busy[fl.slot]) fl.slot++;   // a slot is free: fewer than kSlots in flight
            S->slot_busy[fl.slot] = true;
            for (Request* R : batch) R->batch = fl.batch_id;
            lk.unlock();
            const panda_status st = enqueue_batch(S, batch, fl);
            lk.lock();
            S->batches++;
            S->batched_requests += (int64_t)batch.size();
            if (st != PANDA_OK) {
                const int64_t t = S->now_ns();
                release(S, fl);
                for (int64_t id : ids) {
                    Request& R = S->reqs[id];
                    R.status = st;
                    R.t_done = t;
                    R.done = true;
                }
                S->cv.notify_all();
            } else {
                S->inflight.push_back(fl);
            }
            continue;
        }
        if (!S->inflight.empty())
            S->cv.wait_for(lk, std::chrono::microseconds(20));
        else
            S->cv.wait(lk, [S] { return S->stop || !S->pending.empty(); });
    }
}

}  // namespace
}  // namespace panda

struct panda_server : panda::Server {};

using namespace panda;

extern "C" {

panda_status panda_server_create(int64_t mem_budget_bytes, int64_t max_batch_queries, panda_server** out)
{
    clear_error();
    if (!out || mem_budget_bytes < 0 || max_batch_queries < 1) {
        set_error("panda_server_create: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    *out = nullptr;
    panda_server* S = new panda_server();
    cudaGetDevice(&S->device);
    S->budget = mem_budget_bytes;
    S->max_batch_queries = max_batch_queries;
    S->t0 = Clock::now();
    auto destroy_streams = [S] {
        for (cudaStream_t& q : S->qstream)
            if (q) cudaStreamDestroy(q);
        if (S->bstream) cudaStreamDestroy(S->bstream);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&S->bstream, cudaStreamNonBlocking);
    for (int i = 0; i < Server::kSlots && e == cudaSuccess; i++)
        e = cudaStreamCreateWithFlags(&S->qstream[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        destroy_streams();
        delete S;
        return cuda_fail(e, "panda_server_create: streams");
    }
    panda_status st = configure_knn_lo();
    if (st == PANDA_OK) st = configure_knn_hi();
    if (st != PANDA_OK) {
        destroy_streams();
        delete S;
        return st;
    }
    S->sched = std::thread(scheduler, S);
    *out = S;
    return PANDA_OK;
}

panda_status panda_server_add_tree(panda_server* S, const float* points, int64_t n, int32_t d, int32_t bucket,
                                   int32_t* tree_id)
{
    clear_error();
    if (!S || !tree_id || !points || n < 1 || d < 1 || bucket < 1) {
        set_error("panda_server_add_tree: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    // admission: the resident tree plus the build's transient buffers must fit
    const int dp = padded_dim(d);
    const int64_t tree_est = n * point_float4s(dp) * 16 + (4 * n / bucket + 200000) * node_float4s(dp) * 16;
    const int64_t build_est = n * (2LL * (4 * d + 4)) + tree_est;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->budget > 0 && S->used + tree_est > S->budget) {
            set_error("panda_server_add_tree: memory budget of %lld bytes would be exceeded (%lld used, %lld needed)",
                      (long long)S->budget, (long long)S->used, (long long)tree_est);
            return PANDA_ERR_OUT_OF_MEMORY;
        }
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    if ((int64_t)free_b < build_est) {
        set_error("panda_server_add_tree: %zu bytes free on the device, about %lld needed", free_b,
                  (long long)build_est);
        return PANDA_ERR_OUT_OF_MEMORY;
    }
    std::lock_guard<std::mutex> blk(S->build_mu);   // one build at a time, on the build stream
    panda_tree* t = nullptr;
    panda_status st = build_tree(points, n, d, bucket, S->bstream, &t);
    if (st != PANDA_OK) return st;
    cudaError_t e = cudaStreamSynchronize(S->bstream);
    if (e != cudaSuccess) {
        panda_free(t);
        return cuda_fail(e, "panda_server_add_tree: build");
    }
    const int64_t bytes = (int64_t)t->node_cap * t->ns * 16 + t->n * t->nv * 16;
    std::lock_guard<std::mutex> lk(S->mu);
    S->trees.push_back(t);
    S->tree_bytes.push_back(bytes);
    S->used += bytes;
    *tree_id = (int32_t)S->trees.size() - 1;
    return PANDA_OK;
}

panda_status panda_server_submit(panda_server* S, int32_t tree_id, const float* queries, int64_t m, int32_t k,
                                 int32_t* out_ids, float* out_d2, int64_t* request_id)
{
    clear_error();
    if (!S || !request_id || m < 0 || k < 1 || (m > 0 && (!queries || !out_ids || !out_d2))) {
        set_error("panda_server_submit: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (k > kMaxK) {
        set_error("panda_server_submit: k=%d above %d", k, kMaxK);
        return PANDA_ERR_UNSUPPORTED;
    }
    if (m >= (1LL << 31)) {
        set_error("panda_server_submit: m too large");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (tree_id < 0 || tree_id >= (int32_t)S->trees.size()) {
        set_error("panda_server_submit: unknown tree %d", tree_id);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (S->stop) {
        set_error("panda_server_submit: server is shutting down");
        return PANDA_ERR_QUEUE_FULL;
    }
    if (S->max_pending_queries > 0 && S->pending_queries + m > S->max_pending_queries) {
        set_error("panda_server_submit: %lld queries waiting, %lld more exceed the queue limit of %lld",
                  (long long)S->pending_queries, (long long)m, (long long)S->max_pending_queries);
        return PANDA_ERR_QUEUE_FULL;
    }
    Request R;
    R.id = S->next_id++;
    R.tree = tree_id;
    R.queries = queries;
    R.m = m;
    R.k = k;
    R.ids = out_ids;
    R.d2 = out_d2;
    R.t_submit = S->now_ns();
    if (m == 0) {
        R.done = true;
        R.t_done = R.t_submit;
    }
    S->reqs[R.id] = R;
    if (m > 0) {
        S->pending.push_back(R.id);
        S->pending_queries += m;
    }
    *request_id = R.id;
    S->cv.notify_all();
    return PANDA_OK;
}

panda_status panda_server_poll(panda_server* S, int64_t request_id, int32_t* done)
{
    if (!S || !done) return PANDA_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) {
        set_error("panda_server_poll: unknown request %lld", (long long)request_id);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    *done = it->second.done ? 1 : 0;
    const panda_status st = it->second.done ? it->second.status : PANDA_OK;
    if (st != PANDA_OK)
        set_error("panda_server_poll: request %lld failed: %s", (long long)request_id, panda_status_string(st));
    return st;
}

panda_status panda_server_wait(panda_server* S, int64_t request_id, int64_t timeout_us)
{
    if (!S) return PANDA_ERR_INVALID_ARGUMENT;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) {
        set_error("panda_server_wait: unknown request %lld", (long long)request_id);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    const bool ok = S->cv.wait_for(lk, std::chrono::microseconds(std::max<int64_t>(timeout_us, 0)),
                                   [&] { return S->reqs[request_id].done; });
    if (!ok) {
        set_error("panda_server_wait: request %lld not done after %lld us", (long long)request_id,
                  (long long)timeout_us);
        return PANDA_ERR_TIMEOUT;
    }
    const panda_status st = S->reqs[request_id].status;
    if (st != PANDA_OK)
        set_error("panda_server_wait: request %lld failed: %s", (long long)request_id, panda_status_string(st));
    return st;
}

panda_status panda_server_request_info(panda_server* S, int64_t request_id, int64_t* t_submit_ns,
                                       int64_t* t_done_ns, int64_t* batch_id)
{
    if (!S) return PANDA_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return PANDA_ERR_INVALID_ARGUMENT;
    if (t_submit_ns) *t_submit_ns = it->second.t_submit;
    if (t_done_ns) *t_done_ns = it->second.t_done;
    if (batch_id) *batch_id = it->second.batch;
    return PANDA_OK;
}

int64_t panda_server_now_ns(panda_server* S) { return S ? S->now_ns() : -1; }

panda_status panda_server_stats(panda_server* S, int64_t* batches, int64_t* requests, int64_t* pending,
                                int64_t* bytes_used)
{
    if (!S) return PANDA_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(S->mu);
    if (batches) *batches = S->batches;
    if (requests) *requests = S->batched_requests;
    if (pending) *pending = (int64_t)S->pending.size();
    if (bytes_used) *bytes_used = S->used;
    return PANDA_OK;
}

panda_status panda_server_set_queue_limit(panda_server* S, int64_t max_pending_queries)
{
    if (!S || max_pending_queries < 0) {
        set_error("panda_server_set_queue_limit: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->max_pending_queries = max_pending_queries;
    return PANDA_OK;
}

panda_status panda_server_admission(panda_server* S, int64_t* scratch_reserved, int64_t* deferred_requests,
                                    int64_t* pending_queries)
{
    if (!S) return PANDA_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(S->mu);
    if (scratch_reserved) *scratch_reserved = S->scratch_reserved;
    if (deferred_requests) *deferred_requests = S->deferred;
    if (pending_queries) *pending_queries = S->pending_queries;
    return PANDA_OK;
}

void panda_server_destroy(panda_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->sched.joinable()) S->sched.join();
    for (cudaStream_t q : S->qstream) cudaStreamSynchronize(q);
    for (panda_tree* t : S->trees) panda_free(t);
    for (int i = 0; i < Server::kSlots; i++) {
        if (S->h_err[i]) cudaFreeHost(S->h_err[i]);
        cudaStreamDestroy(S->qstream[i]);
    }
    cudaStreamDestroy(S->bstream);
    delete S;
}

}  // extern "C"
