// api.cu -- the C ABI declared in include/panda.h and the host runtime
// (errors, launch accounting, phase timing, stream-ordered workspace).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace panda {

namespace {
thread_local char g_err[512] = "";
thread_local int64_t g_launches = 0;
int g_timing = 0;   // 0 off, 1 every phase, 2 the traversal phase only
thread_local bool g_timing_suppressed = false;

struct PhaseRow {
    const char* name;
    float ms;
    int32_t launches;
};
thread_local std::vector<PhaseRow> g_phases;

std::once_flag g_pool_once[64];
// Fault injection for the host-side error paths: workspace allocations left
// before the next one fails (-1: none fails).
std::atomic<long long> g_fail_after{-1};
int g_sms[64] = {0};
// Live workspace and tree allocations of the library: pointer -> bytes.
std::mutex g_ws_mu;
std::unordered_map<void*, size_t> g_ws_live;
long long g_ws_bytes = 0;
// Guards the use-event lists of every tree.
std::mutex g_use_mu;
}  // namespace

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

panda_status cuda_fail(cudaError_t e, const char* what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PANDA_ERR_OUT_OF_MEMORY : PANDA_ERR_CUDA;
}

panda_status note_launch(const char* what)
{
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return PANDA_OK;
}

int64_t launches_so_far() { return g_launches; }
bool phase_timing_enabled() { return g_timing != 0; }
void set_phase_timing_suppressed(bool on) { g_timing_suppressed = on; }

PhaseTimer::PhaseTimer(cudaStream_t s) : stream_(s), on_(g_timing != 0 && !g_timing_suppressed) {}

PhaseTimer::~PhaseTimer()
{
    for (cudaEvent_t e : ev_) cudaEventDestroy(e);
}

void PhaseTimer::mark(const char* name)
{
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        on_ = false;
        return;
    }
    cudaEventRecord(e, stream_);
    ev_.push_back(e);
    names_.push_back(name);
    launches_at_.push_back(g_launches);
}

void PhaseTimer::begin(const char* name)
{
    if (!on_) return;
    if (g_timing == 2 && strcmp(name, "query.traverse") != 0) {
        end();   // traversal-only mode: no event between the other kernels
        return;
    }
    mark(name);
}

void PhaseTimer::end()
{
    if (on_ && !names_.empty() && names_.back() != nullptr) mark(nullptr);
}

void PhaseTimer::finish()
{
    if (!on_) return;
    end();
    g_phases.clear();
    if (ev_.size() < 2) return;
    cudaEventSynchronize(ev_.back());
    for (size_t i = 0; i + 1 < ev_.size(); i++) {
        if (!names_[i]) continue;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev_[i], ev_[i + 1]);
        int32_t l = (int32_t)(launches_at_[i + 1] - launches_at_[i]);
        bool merged = false;
        for (auto& r : g_phases)
            if (strcmp(r.name, names_[i]) == 0) {
                r.ms += ms;
                r.launches += l;
                merged = true;
                break;
            }
        if (!merged) g_phases.push_back({names_[i], ms, l});
    }
    cudaGetLastError();
}

int num_sms()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!g_sms[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = v > 0 ? v : 152;
    }
    return g_sms[dev];
}

panda_status ws_alloc(void** p, size_t bytes, cudaStream_t s, const char* what)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64) {
        std::call_once(g_pool_once[dev], [dev]() {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t keep = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
            cudaGetLastError();
        });
    }
    *p = nullptr;
    long long f = g_fail_after.load();
    while (f >= 0 && !g_fail_after.compare_exchange_weak(f, f - 1)) {
    }
    if (f == 0) {
        set_error("allocating %zu bytes for %s: injected allocation failure", bytes, what);
        return PANDA_ERR_OUT_OF_MEMORY;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("allocating %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? PANDA_ERR_OUT_OF_MEMORY : PANDA_ERR_CUDA;
    }
    try {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        g_ws_live[*p] = bytes;
        g_ws_bytes += (long long)bytes;
    } catch (...) {
        cudaFreeAsync(*p, s);
        *p = nullptr;
        set_error("allocating %zu bytes for %s: host bookkeeping failed", bytes, what);
        return PANDA_ERR_OUT_OF_MEMORY;
    }
    return PANDA_OK;
}

void ws_free(void* p, cudaStream_t s)
{
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        auto it = g_ws_live.find(p);
        if (it != g_ws_live.end()) {
            g_ws_bytes -= (long long)it->second;
            g_ws_live.erase(it);
        }
    }
    cudaFreeAsync(p, s);
}

long long ws_bytes_held()
{
    std::lock_guard<std::mutex> lk(g_ws_mu);
    return g_ws_bytes;
}

void note_tree_use(const panda_tree* ct, cudaStream_t s)
{
    if (!ct) return;
    panda_tree* t = const_cast<panda_tree*>(ct);
    std::lock_guard<std::mutex> lk(g_use_mu);
    // drop the uses that have finished
    int w = 0;
    for (int i = 0; i < t->nuses; i++) {
        if (cudaEventQuery(t->uses[i]) == cudaSuccess) cudaEventDestroy(t->uses[i]);
        else t->uses[w++] = t->uses[i];
    }
    cudaGetLastError();
    t->nuses = w;
    if (t->nuses == panda_tree::kMaxUses) {
        // list full: wait for the oldest on the host (rare: kMaxUses uses still in flight)
        cudaEventSynchronize(t->uses[0]);
        cudaEventDestroy(t->uses[0]);
        for (int i = 1; i < t->nuses; i++) t->uses[i - 1] = t->uses[i];
        t->nuses--;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(e, s) != cudaSuccess) {
        // no event: fall back to waiting for the stream now
        if (e) cudaEventDestroy(e);
        cudaGetLastError();
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return;
    }
    t->uses[t->nuses++] = e;
}

void wait_tree_uses(const panda_tree* ct, cudaStream_t s)
{
    panda_tree* t = const_cast<panda_tree*>(ct);
    std::lock_guard<std::mutex> lk(g_use_mu);
    for (int i = 0; i < t->nuses; i++) {
        if (cudaStreamWaitEvent(s, t->uses[i], 0) != cudaSuccess) {
            cudaGetLastError();
            cudaEventSynchronize(t->uses[i]);
        }
        cudaEventDestroy(t->uses[i]);
    }
    cudaGetLastError();
    t->nuses = 0;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Overwrite a failed query's device outputs with the padding row (-1, +inf),
// so a blocking call that reports an error never leaves partial results.
__global__ void k_fill_failed(int32_t* ids, float* d2, long long count)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        ids[i] = -1;
        d2[i] = __int_as_float(0x7f800000);
    }
}

void clear_failed_outputs(int32_t* ids, float* d2, long long count)
{
    if (!ids || !d2 || count <= 0) return;
    const unsigned blocks = (unsigned)std::min<long long>((count + 255) / 256, 4LL * num_sms());
    k_fill_failed<<<blocks, 256>>>(ids, d2, count);
    cudaStreamSynchronize(nullptr);
    cudaGetLastError();
}

}  // namespace panda

using namespace panda;

extern "C" {

const char* panda_version(void) { return "panda-gb300 0.1 (sm_103a)"; }

const char* panda_status_string(panda_status s)
{
    switch (s) {
        case PANDA_OK: return "ok";
        case PANDA_ERR_INVALID_ARGUMENT: return "invalid argument";
        case PANDA_ERR_NONFINITE_INPUT: return "non-finite input";
        case PANDA_ERR_UNSUPPORTED: return "unsupported";
        case PANDA_ERR_OUT_OF_MEMORY: return "out of memory";
        case PANDA_ERR_CUDA: return "cuda error";
        case PANDA_ERR_TIMEOUT: return "timeout";
        case PANDA_ERR_QUEUE_FULL: return "queue full";
        case PANDA_ERR_DEPTH: return "depth limit exceeded";
    }
    return "unknown status";
}

const char* panda_last_error(void) { return g_err; }

void panda_set_phase_timing(int32_t enable) { g_timing = enable == 2 ? 2 : (enable != 0 ? 1 : 0); }

int32_t panda_phase_times(const char** names, float* ms, int32_t* launches, int32_t cap)
{
    int32_t n = (int32_t)g_phases.size();
    for (int32_t i = 0; i < n && i < cap; i++) {
        if (names) names[i] = g_phases[i].name;
        if (ms) ms[i] = g_phases[i].ms;
        if (launches) launches[i] = g_phases[i].launches;
    }
    return n;
}

int64_t panda_kernel_launches(void) { return g_launches; }

panda_status panda_build_async(const float* points, int64_t n, int32_t d, int32_t bucket, void* stream,
                               panda_tree** out)
{
    if (!out) {
        set_error("panda_build: out is NULL");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    clear_error();
    try {
        return build_tree(points, n, d, bucket, (cudaStream_t)stream, out);
    } catch (...) {
        set_error("panda_build: host exception");
        return PANDA_ERR_OUT_OF_MEMORY;
    }
}

panda_status panda_debug_fail_alloc(int64_t after)
{
    g_fail_after.store(after < 0 ? -1 : (long long)after);
    return PANDA_OK;
}

panda_status panda_debug_pool_used(int64_t* bytes)
{
    clear_error();
    if (!bytes) {
        set_error("panda_debug_pool_used: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    *bytes = (int64_t)ws_bytes_held();
    return PANDA_OK;
}

panda_status panda_build(const float* points, int64_t n, int32_t d, int32_t bucket, panda_tree** out)
{
    panda_status s = panda_build_async(points, n, d, bucket, nullptr, out);
    if (s == PANDA_OK) {
        cudaError_t e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) {
            panda_free(*out);
            *out = nullptr;
            return cuda_fail(e, "panda_build");
        }
    }
    return s;
}

panda_status panda_build_host(const float* points, int64_t n, int32_t d, int32_t bucket, void* stream,
                              panda_tree** out)
{
    if (!out || !points || n < 1 || d < 1 || d > kMaxDim) {
        if (out) *out = nullptr;
        set_error("panda_build_host: invalid argument");
        return (d > kMaxDim) ? PANDA_ERR_UNSUPPORTED : PANDA_ERR_INVALID_ARGUMENT;
    }
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    void* dev = nullptr;
    const size_t bytes = (size_t)n * d * sizeof(float);
    panda_status st = ws_alloc(&dev, bytes, s, "host points staging");
    if (st != PANDA_OK) return st;
    cudaError_t e = cudaMemcpyAsync(dev, points, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        ws_free(dev, s);
        return cuda_fail(e, "panda_build_host copy");
    }
    try {
        st = build_tree(static_cast<const float*>(dev), n, d, bucket, s, out);
    } catch (...) {
        st = PANDA_ERR_OUT_OF_MEMORY;
    }
    ws_free(dev, s);
    return st;
}

panda_status panda_knn_async(const panda_tree* tree, const float* queries, int64_t m, int32_t k,
                             int32_t* out_ids, float* out_d2, const panda_query_params* params, void* stream)
{
    clear_error();
    try {
        return knn_query(tree, queries, m, k, out_ids, out_d2, params, (cudaStream_t)stream, nullptr);
    } catch (...) {
        set_error("panda_knn: host exception");
        return PANDA_ERR_OUT_OF_MEMORY;
    }
}

panda_status panda_knn(const panda_tree* tree, const float* queries, int64_t m, int32_t k, int32_t* out_ids,
                       float* out_d2)
{
    clear_error();
    unsigned herr = 0;
    panda_status s;
    try {
        s = knn_query(tree, queries, m, k, out_ids, out_d2, nullptr, nullptr, &herr);
    } catch (...) {
        set_error("panda_knn: host exception");
        return PANDA_ERR_OUT_OF_MEMORY;
    }
    if (s == PANDA_OK && herr) clear_failed_outputs(out_ids, out_d2, m * (long long)k);
    if (s == PANDA_OK && (herr & kErrNonfinite)) {
        set_error("panda_knn: non-finite query coordinate");
        return PANDA_ERR_NONFINITE_INPUT;
    }
    if (s == PANDA_OK && herr) {
        set_error("panda_knn: internal consistency check failed (0x%x)", herr);
        return PANDA_ERR_CUDA;
    }
    return s;
}

panda_status panda_knn_self_async(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2,
                                  const panda_query_params* params, void* stream)
{
    clear_error();
    try {
        return knn_self(tree, k, out_ids, out_d2, params, (cudaStream_t)stream, nullptr);
    } catch (...) {
        set_error("panda_knn_self: host exception");
        return PANDA_ERR_OUT_OF_MEMORY;
    }
}

panda_status panda_knn_self(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2)
{
    clear_error();
    unsigned herr = 0;
    panda_status s;
    try {
        s = knn_self(tree, k, out_ids, out_d2, nullptr, nullptr, &herr);
    } catch (...) {
        set_error("panda_knn_self: host exception");
        return PANDA_ERR_OUT_OF_MEMORY;
    }
    if (s == PANDA_OK && herr) {
        clear_failed_outputs(out_ids, out_d2, tree->n * (long long)k);
        set_error("panda_knn_self: internal consistency check failed (0x%x)", herr);
        return PANDA_ERR_CUDA;
    }
    return s;
}

// Shared by the blocking and the enqueue-only host variants of the all-points query.
static panda_status knn_self_host_impl(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2,
                                       const panda_query_params* params, void* stream, bool wait)
{
    clear_error();
    if (!tree || k < 1 || !out_ids || !out_d2) {
        set_error("panda_knn_self_host: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (k > kMaxK) {
        set_error("panda_knn_self_host: k=%d above the maximum %d", k, kMaxK);
        return PANDA_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void *di = nullptr, *dd = nullptr;
    const size_t ob = (size_t)tree->n * k * 4;
    panda_status st = ws_alloc(&di, ob, s, "id staging");
    if (st == PANDA_OK) st = ws_alloc(&dd, ob, s, "distance staging");
    unsigned herr = 0;
    if (st == PANDA_OK) {
        try {
            st = knn_self(tree, k, static_cast<int32_t*>(di), static_cast<float*>(dd), params, s,
                          wait ? &herr : nullptr);
        } catch (...) {
            st = PANDA_ERR_OUT_OF_MEMORY;
        }
    }
    if (st == PANDA_OK && !herr) {   // a failed query leaves the host outputs untouched
        cudaError_t e = cudaMemcpyAsync(out_ids, di, ob, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_d2, dd, ob, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && wait) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "panda_knn_self_host copy out");
    }
    ws_free(di, s);
    ws_free(dd, s);
    if (st == PANDA_OK && herr) {
        set_error("panda_knn_self_host: internal consistency check failed (0x%x)", herr);
        return PANDA_ERR_CUDA;
    }
    return st;
}

panda_status panda_knn_self_host(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2,
                                 const panda_query_params* params, void* stream)
{
    return knn_self_host_impl(tree, k, out_ids, out_d2, params, stream, true);
}

panda_status panda_knn_self_host_async(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2,
                                       const panda_query_params* params, void* stream)
{
    return knn_self_host_impl(tree, k, out_ids, out_d2, params, stream, false);
}

panda_status panda_knn_host(const panda_tree* tree, const float* queries, int64_t m, int32_t k, int32_t* out_ids,
                            float* out_d2, const panda_query_params* params, void* stream)
{
    clear_error();
    if (!tree || m < 0 || k < 1 || (m > 0 && (!queries || !out_ids || !out_d2))) {
        set_error("panda_knn_host: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (k > kMaxK) {
        set_error("panda_knn_host: k=%d above the maximum %d", k, kMaxK);
        return PANDA_ERR_UNSUPPORTED;
    }
    if (m == 0) return PANDA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    void *dq = nullptr, *di = nullptr, *dd = nullptr;
    const size_t qb = (size_t)m * tree->d * sizeof(float), ob = (size_t)m * k * 4;
    panda_status st = ws_alloc(&dq, qb, s, "query staging");
    if (st == PANDA_OK) st = ws_alloc(&di, ob, s, "id staging");
    if (st == PANDA_OK) st = ws_alloc(&dd, ob, s, "distance staging");
    cudaError_t e = cudaSuccess;
    unsigned herr = 0;
    if (st == PANDA_OK) {
        e = cudaMemcpyAsync(dq, queries, qb, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = cuda_fail(e, "panda_knn_host copy in");
    }
    if (st == PANDA_OK) {
        try {
            st = knn_query(tree, static_cast<const float*>(dq), m, k, static_cast<int32_t*>(di),
                           static_cast<float*>(dd), params, s, &herr);
        } catch (...) {
            st = PANDA_ERR_OUT_OF_MEMORY;
        }
    }
    if (st == PANDA_OK && !herr) {   // a failed query leaves the host outputs untouched
        e = cudaMemcpyAsync(out_ids, di, ob, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_d2, dd, ob, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "panda_knn_host copy out");
    }
    ws_free(dq, s);
    ws_free(di, s);
    ws_free(dd, s);
    if (st == PANDA_OK && (herr & kErrNonfinite)) {
        set_error("panda_knn_host: non-finite query coordinate");
        return PANDA_ERR_NONFINITE_INPUT;
    }
    if (st == PANDA_OK && herr) {
        set_error("panda_knn_host: internal consistency check failed (0x%x)", herr);
        return PANDA_ERR_CUDA;
    }
    return st;
}

panda_status panda_knn_visits(const panda_tree* tree, const float* queries, int64_t m, int32_t k,
                              int32_t* out_ids, float* out_d2, int32_t* out_visits,
                              uint64_t* out_stats, const panda_query_params* params, void* stream)
{
    clear_error();
    if ((out_visits && m > 0 && !is_device_ptr(out_visits)) || (out_stats && !is_device_ptr(out_stats))) {
        set_error("panda_knn_visits: out_visits and out_stats must be device pointers");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    try {
        if (!queries) {   // the all-points query of panda_knn_self
            if (!tree || m != tree->n) {
                set_error("panda_knn_visits: queries NULL needs m = the tree's n");
                return PANDA_ERR_INVALID_ARGUMENT;
            }
            return knn_self(tree, k, out_ids, out_d2, params, (cudaStream_t)stream, nullptr, out_visits,
                            reinterpret_cast<unsigned long long*>(out_stats));
        }
        return knn_query(tree, queries, m, k, out_ids, out_d2, params, (cudaStream_t)stream, nullptr,
                         out_visits, reinterpret_cast<unsigned long long*>(out_stats));
    } catch (...) {
        set_error("panda_knn_visits: host exception");
        return PANDA_ERR_OUT_OF_MEMORY;
    }
}

// Frees wait, on the GPU, for every recorded use of the tree (the build, each
// query and refit), then return the memory to the pool in stream order; the
// host does not wait.
static void free_tree_on(panda_tree* tree, cudaStream_t s)
{
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != tree->device) cudaSetDevice(tree->device);
    if (tree->pooled) {
        wait_tree_uses(tree, s);
        ws_free(tree->nodes, s);
        ws_free(tree->points, s);
    } else {
        // cudaMalloc'd tables (a loaded checkpoint): cudaFree waits for the device
        wait_tree_uses(tree, s);
        if (tree->nodes) cudaFree(tree->nodes);
        if (tree->points) cudaFree(tree->points);
    }
    cudaGetLastError();
    if (cur != tree->device) cudaSetDevice(cur);
    delete tree;
}

void panda_free(panda_tree* tree)
{
    if (!tree) return;
    free_tree_on(tree, nullptr);
}

void panda_free_async(panda_tree* tree, void* stream)
{
    if (!tree) return;
    free_tree_on(tree, (cudaStream_t)stream);
}

panda_status panda_tree_get_info(const panda_tree* t, panda_tree_info* info)
{
    if (!t || !info) {
        set_error("panda_tree_get_info: NULL argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    info->n = t->n;
    info->d = t->d;
    info->bucket = t->bucket;
    info->num_nodes = t->num_nodes;
    info->node_slots = t->node_slots;
    info->num_leaves = t->num_leaves;
    info->depth = t->depth;
    info->node_floats = 4 * t->ns;
    info->point_floats = 4 * t->nv;
    info->subtree_threshold = t->threshold;
    info->device_bytes = (int64_t)t->node_cap * t->ns * 16 + t->n * t->nv * 16;
    return PANDA_OK;
}

panda_status panda_tree_copy(const panda_tree* t, float* host_nodes, float* host_points)
{
    if (!t) {
        set_error("panda_tree_copy: NULL tree");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (host_nodes)
        PANDA_CUDA(cudaMemcpy(host_nodes, t->nodes, (size_t)t->node_slots * t->ns * 16, cudaMemcpyDeviceToHost),
                   "panda_tree_copy nodes");
    if (host_points)
        PANDA_CUDA(cudaMemcpy(host_points, t->points, (size_t)t->n * t->nv * 16, cudaMemcpyDeviceToHost),
                   "panda_tree_copy points");
    return PANDA_OK;
}

}  // extern "C"
