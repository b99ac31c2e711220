// batch.cu -- batched form: many independent point sets built and queried
// together (the paper batches queries to balance load, Sec. III-B).
//
// All sets are concatenated; one forest build (one root per set, the level
// passes and the subtree stage serving every set at once) is followed by one
// query ordering over all queries (keys keep each set's queries contiguous)
// and one persistent traversal launch whose warps take (set, 32 queries) jobs
// from a device work queue, so sets of very different sizes share the GPU.
// Buffers belong to the batch, so the first run captures the whole sequence
// in a CUDA graph and later runs replay it with one launch.
#include <string.h>

#include <algorithm>
#include <vector>

#include "order.cuh"
#include "query.cuh"
#include "runtime.h"

namespace panda {
template <int DP>
panda_status launch_knn_dp(const KnnArgs& a, cudaStream_t s);
}

struct panda_batch {
    int nsets = 0, d = 0, bucket = 0, kmax = 0, device = 0;
    long long n_total = 0, m_total = 0, out_total = 0;
    std::vector<long long> np, nq, poff, qoff, ooff;
    std::vector<int> ks;
    panda_tree forest;
    panda::BuildState* bs = nullptr;
    float* points = nullptr;
    float* queries = nullptr;
    int32_t* ids = nullptr;
    float* d2 = nullptr;
    unsigned* keys = nullptr;
    int* perm = nullptr;
    int* hist = nullptr;
    int* bsum = nullptr;
    int nb = 0, nblk = 0, shift = 0;
    int* d_qoff = nullptr;
    int* d_poff = nullptr;
    int* d_bin = nullptr;
    panda::KnnSet* d_sets = nullptr;
    panda::KnnJob* d_jobs = nullptr;
    int njobs = 0;
    int* d_head = nullptr;
    unsigned* d_err = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels_per_run = 0;
    int transpose_max = panda::kTransposeMaxDefault;
    int traversal = PANDA_TRAVERSAL_AUTO;
    int any_solo = 0;   // some set takes the per-query traversal
    std::vector<void*> owned;
};

namespace panda {
namespace {

panda_status batch_alloc(panda_batch* b, void** p, size_t bytes, const char* what)
{
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("panda_batch: allocating %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? PANDA_ERR_OUT_OF_MEMORY : PANDA_ERR_CUDA;
    }
    b->owned.push_back(*p);
    return PANDA_OK;
}

panda_status launch_multi(const KnnArgs& a, int dp, cudaStream_t s)
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

// Every step of one batch run, enqueued on `s` (no host synchronisation).
panda_status batch_enqueue(panda_batch* b, cudaStream_t s)
{
    panda_status st = forest_enqueue(b->bs, s);
    if (st != PANDA_OK) return st;
    PANDA_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), s), "batch: clear error");
    PANDA_CUDA(cudaMemsetAsync(b->d_head, 0, sizeof(int), s), "batch: clear queue head");
    PANDA_CUDA(cudaMemsetAsync(b->hist, 0, (size_t)b->nb * sizeof(int), s), "batch: clear histogram");
    if (b->m_total == 0) return PANDA_OK;
    OrderArgs oa;
    memset(&oa, 0, sizeof(oa));
    oa.nodes = b->forest.nodes;
    oa.num_nodes = b->forest.node_cap;
    oa.queries = b->queries;
    oa.m = b->m_total;
    oa.d = b->d;
    oa.ns = b->forest.ns;
    oa.mode = PANDA_ORDER_LEAF;
    oa.shift = b->shift;
    oa.keys = b->keys;
    oa.hist = b->hist;
    oa.qset_off = b->d_qoff;
    oa.set_poff = b->d_poff;
    oa.set_bin = b->d_bin;
    oa.nsets = b->nsets;
    const unsigned gb = (unsigned)((b->m_total + 255) / 256);
    k_order_keys<<<gb, 256, 0, s>>>(oa);
    PANDA_LAUNCHED("k_order_keys");
    k_scan_blocks<<<b->nblk, 1024, 0, s>>>(b->hist, b->nb, b->bsum);
    PANDA_LAUNCHED("k_scan_blocks");
    k_scan_sums<<<1, 1024, 0, s>>>(b->bsum, b->nblk);
    PANDA_LAUNCHED("k_scan_sums");
    k_order_scatter<<<gb, 256, 0, s>>>(b->keys, b->m_total, b->hist, b->bsum, b->perm);
    PANDA_LAUNCHED("k_order_scatter");
    KnnArgs ka;
    memset(&ka, 0, sizeof(ka));
    ka.sets = b->d_sets;
    ka.jobs = b->d_jobs;
    ka.njobs = b->njobs;
    ka.job_head = b->d_head;
    ka.err = b->d_err;
    ka.m = b->m_total;
    ka.d = b->d;
    ka.k = b->kmax;
    ka.transpose_max = b->transpose_max;
    ka.solo = b->any_solo;
    return launch_multi(ka, padded_dim(b->d), s);
}

}  // namespace
}  // namespace panda

using namespace panda;

extern "C" {

panda_status panda_batch_create(const panda_set_desc* sets, int32_t nsets, int32_t d, int32_t bucket,
                                panda_batch** out)
{
    clear_error();
    if (!out) return PANDA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (!sets || nsets < 1 || d < 1 || bucket < 1) {
        set_error("panda_batch_create: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (d > kMaxDim || bucket > kMaxBucket) {
        set_error("panda_batch_create: unsupported d=%d or bucket=%d", d, bucket);
        return PANDA_ERR_UNSUPPORTED;
    }
    panda_batch* b = new panda_batch();
    b->nsets = nsets;
    b->d = d;
    b->bucket = bucket;
    cudaGetDevice(&b->device);
    b->np.resize(nsets);
    b->nq.resize(nsets);
    b->ks.resize(nsets);
    b->poff.resize(nsets + 1);
    b->qoff.resize(nsets + 1);
    b->ooff.resize(nsets + 1);
    for (int s = 0; s < nsets; s++) {
        if (sets[s].n_points < 1 || sets[s].n_queries < 0 || sets[s].k < 1) {
            set_error("panda_batch_create: set %d needs n_points >= 1, n_queries >= 0, k >= 1", s);
            delete b;
            return PANDA_ERR_INVALID_ARGUMENT;
        }
        if (sets[s].k > kMaxK) {
            set_error("panda_batch_create: set %d has k=%d above %d", s, sets[s].k, kMaxK);
            delete b;
            return PANDA_ERR_UNSUPPORTED;
        }
        b->np[s] = sets[s].n_points;
        b->nq[s] = sets[s].n_queries;
        b->ks[s] = sets[s].k;
        b->poff[s] = b->n_total;
        b->qoff[s] = b->m_total;
        b->ooff[s] = b->out_total;
        b->n_total += b->np[s];
        b->m_total += b->nq[s];
        b->out_total += b->nq[s] * b->ks[s];
        b->kmax = std::max(b->kmax, b->ks[s]);
    }
    b->poff[nsets] = b->n_total;
    b->qoff[nsets] = b->m_total;
    b->ooff[nsets] = b->out_total;
    if (b->n_total >= (1LL << 31) - 4 || b->m_total >= (1LL << 31)) {
        set_error("panda_batch_create: more than 2^31 points or queries");
        delete b;
        return PANDA_ERR_UNSUPPORTED;
    }
    panda_status st;
#define BALLOC(ptr, bytes, what)                                                         \
    if ((st = batch_alloc(b, (void**)&(ptr), (bytes), what)) != PANDA_OK) {             \
        panda_batch_free(b);                                                              \
        return st;                                                                        \
    }
    BALLOC(b->points, (size_t)b->n_total * d * sizeof(float), "points");
    BALLOC(b->queries, (size_t)std::max<long long>(b->m_total, 1) * d * sizeof(float), "queries");
    BALLOC(b->ids, (size_t)std::max<long long>(b->out_total, 1) * sizeof(int32_t), "ids");
    BALLOC(b->d2, (size_t)std::max<long long>(b->out_total, 1) * sizeof(float), "distances");
    st = forest_create(b->np.data(), nsets, d, bucket, b->points, nullptr, &b->forest, &b->bs);
    if (st != PANDA_OK) {
        panda_batch_free(b);
        return st;
    }
    // ordering bins: set s owns bins [bin[s], bin[s] + (n_s >> shift) + 1)
    int sh = 0;
    for (;;) {
        long long tot = 0;
        for (int s = 0; s < nsets; s++) tot += (b->np[s] >> sh) + 1;
        if (tot <= (1LL << 22) || sh >= 30) {
            b->nb = (int)tot;
            break;
        }
        sh++;
    }
    b->shift = sh;
    b->nblk = (b->nb + 4095) / 4096;
    std::vector<int> hq(nsets + 1), hp(nsets), hb(nsets);
    long long acc = 0;
    for (int s = 0; s < nsets; s++) {
        hq[s] = (int)b->qoff[s];
        hp[s] = (int)b->poff[s];
        hb[s] = (int)acc;
        acc += (b->np[s] >> sh) + 1;
    }
    hq[nsets] = (int)b->m_total;
    std::vector<KnnSet> hs(nsets);
    std::vector<KnnJob> hj;
    for (int s = 0; s < nsets; s++) {
        KnnSet& S = hs[s];
        memset(&S, 0, sizeof(S));
        S.nodes = b->forest.nodes;
        S.pts = b->forest.points;
        S.num_nodes = b->forest.node_cap;
        S.npts = b->n_total;
        S.queries = b->queries + b->qoff[s] * d;
        S.perm = nullptr;   // set below (device pointer arithmetic)
        S.ids = b->ids + b->ooff[s];
        S.d2 = b->d2 + b->ooff[s];
        S.m = b->nq[s];
        S.root = s;
        S.id_base = (int)b->poff[s];
        S.k = b->ks[s];
        S.row_base = (int)b->qoff[s];
        S.solo = prefer_per_query(b->nq[s], b->np[s], d);
        b->any_solo |= S.solo;
        for (long long p = 0; p < b->nq[s]; p += 32) hj.push_back(KnnJob{s, (int)p});
    }
    b->njobs = (int)hj.size();
    BALLOC(b->keys, (size_t)std::max<long long>(b->m_total, 1) * 4, "order keys");
    BALLOC(b->perm, (size_t)std::max<long long>(b->m_total, 1) * 4, "order permutation");
    BALLOC(b->hist, (size_t)b->nblk * 4096 * 4, "order histogram");
    BALLOC(b->bsum, (size_t)b->nblk * 4, "order block sums");
    BALLOC(b->d_qoff, (size_t)(nsets + 1) * 4, "query offsets");
    BALLOC(b->d_poff, (size_t)nsets * 4, "point offsets");
    BALLOC(b->d_bin, (size_t)nsets * 4, "bin offsets");
    BALLOC(b->d_sets, (size_t)nsets * sizeof(KnnSet), "set descriptors");
    BALLOC(b->d_jobs, (size_t)std::max(b->njobs, 1) * sizeof(KnnJob), "jobs");
    BALLOC(b->d_head, sizeof(int), "queue head");
    BALLOC(b->d_err, sizeof(unsigned), "error word");
#undef BALLOC
    for (int s = 0; s < nsets; s++) hs[s].perm = b->perm + b->qoff[s];
    cudaError_t e = cudaMemcpy(b->d_qoff, hq.data(), (nsets + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_poff, hp.data(), nsets * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_bin, hb.data(), nsets * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_sets, hs.data(), nsets * sizeof(KnnSet), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b->njobs)
        e = cudaMemcpy(b->d_jobs, hj.data(), b->njobs * sizeof(KnnJob), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "panda_batch_create: descriptors");
        panda_batch_free(b);
        return st;
    }
    *out = b;
    return PANDA_OK;
}

panda_status panda_batch_buffers(panda_batch* b, float** points, float** queries, int32_t** out_ids,
                                 float** out_d2)
{
    if (!b) return PANDA_ERR_INVALID_ARGUMENT;
    if (points) *points = b->points;
    if (queries) *queries = b->queries;
    if (out_ids) *out_ids = b->ids;
    if (out_d2) *out_d2 = b->d2;
    return PANDA_OK;
}

panda_status panda_batch_offsets(const panda_batch* b, int64_t* point_off, int64_t* query_off,
                                 int64_t* out_off)
{
    if (!b) return PANDA_ERR_INVALID_ARGUMENT;
    for (int s = 0; s <= b->nsets; s++) {
        if (point_off) point_off[s] = b->poff[s];
        if (query_off) query_off[s] = b->qoff[s];
        if (out_off) out_off[s] = b->ooff[s];
    }
    return PANDA_OK;
}

panda_status panda_batch_set_query_params(panda_batch* b, const panda_query_params* params)
{
    if (!b) return PANDA_ERR_INVALID_ARGUMENT;
    if (params && params->order != PANDA_ORDER_LEAF) {
        set_error("panda_batch_set_query_params: a batch orders queries by leaf");
        return PANDA_ERR_UNSUPPORTED;
    }
    if (params && params->bounded) {
        set_error("panda_batch_set_query_params: a batch answers unbounded queries");
        return PANDA_ERR_UNSUPPORTED;
    }
    if (b->exec) {
        // the parameters are baked into the captured graph: wait for every run
        // in flight, drop the graph, and capture again at the next run
        PANDA_CUDA(cudaDeviceSynchronize(), "panda_batch_set_query_params: wait for runs in flight");
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->transpose_max = (params && params->transpose_max != 0) ? params->transpose_max : panda::kTransposeMaxDefault;
    b->traversal = params ? params->traversal : PANDA_TRAVERSAL_AUTO;
    // rewrite the set descriptors with the requested traversal shape
    std::vector<KnnSet> hs(b->nsets);
    PANDA_CUDA(cudaMemcpy(hs.data(), b->d_sets, b->nsets * sizeof(KnnSet), cudaMemcpyDeviceToHost),
               "panda_batch_set_query_params");
    b->any_solo = 0;
    for (int s = 0; s < b->nsets; s++) {
        hs[s].solo = b->traversal == PANDA_TRAVERSAL_PER_QUERY ? 1
                     : b->traversal == PANDA_TRAVERSAL_PACKET  ? 0
                                                               : prefer_per_query(b->nq[s], b->np[s], b->d);
        b->any_solo |= hs[s].solo;
    }
    PANDA_CUDA(cudaMemcpy(b->d_sets, hs.data(), b->nsets * sizeof(KnnSet), cudaMemcpyHostToDevice),
               "panda_batch_set_query_params");
    return PANDA_OK;
}

panda_status panda_batch_run(panda_batch* b, void* stream)
{
    clear_error();
    if (!b) {
        set_error("panda_batch_run: NULL batch");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->exec) {
        // the launch configuration of the traversal is set before capture
        panda_status cst = configure_knn_lo();
        if (cst == PANDA_OK) cst = configure_knn_hi();
        if (cst != PANDA_OK) return cst;
        const int64_t l0 = launches_so_far();
        set_phase_timing_suppressed(true);
        cudaStream_t cap = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            set_phase_timing_suppressed(false);
            return cuda_fail(e, "panda_batch_run: capture stream");
        }
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        panda_status st = PANDA_OK;
        if (e == cudaSuccess) st = batch_enqueue(b, cap);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        set_phase_timing_suppressed(false);
        b->kernels_per_run = launches_so_far() - l0;
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return cuda_fail(e, "panda_batch_run: begin capture");
        if (st != PANDA_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "panda_batch_run: end capture");
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(e, "panda_batch_run: instantiate");
        }
    }
    PANDA_CUDA(cudaGraphLaunch(b->exec, s), "panda_batch_run: launch");
    return PANDA_OK;
}

panda_status panda_batch_status(panda_batch* b, void* stream)
{
    clear_error();
    if (!b) return PANDA_ERR_INVALID_ARGUMENT;
    unsigned e1 = 0, e2 = 0;
    panda_status st = forest_collect(b->bs, &b->forest, &e1, (cudaStream_t)stream);
    if (st != PANDA_OK) return st;
    PANDA_CUDA(cudaMemcpy(&e2, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "panda_batch_status");
    const unsigned e = e1 | e2;
    if (e & kErrNonfinite) {
        set_error("panda_batch: non-finite point or query coordinate");
        return PANDA_ERR_NONFINITE_INPUT;
    }
    if (e & (kErrDepth | kErrLevels)) {
        set_error("panda_batch: a tree needed more levels than planned (0x%x)", e);
        return PANDA_ERR_DEPTH;
    }
    if (e) {
        set_error("panda_batch: internal consistency check failed (0x%x)", e);
        return PANDA_ERR_CUDA;
    }
    return PANDA_OK;
}

panda_status panda_batch_info(const panda_batch* b, panda_tree_info* info, int64_t* kernels_per_run)
{
    if (!b || !info) return PANDA_ERR_INVALID_ARGUMENT;
    if (kernels_per_run) *kernels_per_run = b->kernels_per_run;
    return panda_tree_get_info(&b->forest, info);
}

void panda_batch_free(panda_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    forest_destroy(b->bs, nullptr);
    cudaDeviceSynchronize();
    // the forest's tables come from the stream-ordered pool
    ws_free(b->forest.nodes, nullptr);
    ws_free(b->forest.points, nullptr);
    cudaStreamSynchronize(0);
    b->forest.nodes = nullptr;
    b->forest.points = nullptr;
    for (void* p : b->owned) cudaFree(p);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
