// runtime.h -- host-side runtime of the library: tree object, error state,
// launch accounting, phase timing, stream-ordered workspace.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <atomic>
#include <utility>
#include <mutex>
#include <vector>

#include "panda.h"

struct panda_tree {
    int64_t n = 0;
    int32_t d = 0, dp = 0, bucket = 0;
    int32_t nv = 0;           // float4 per packed point
    int32_t ns = 0;           // float4 per node record
    int32_t threshold = 0;    // subtree-stage threshold T
    int device = 0;
    float4* points = nullptr; // [n][nv], leaf order
    float4* nodes = nullptr;  // [node_cap][ns]
    int64_t node_cap = 0;
    int64_t num_nodes = 0, num_leaves = 0;
    int64_t node_slots = 0;   // records in use in the node table (holes included)
    int32_t depth = 0;
    float root_lo[16] = {0}, root_hi[16] = {0};
    bool pooled = true;       // nodes/points from the stream-ordered pool (cudaMallocAsync)
    // Work that may still read or write the tree: one event per call that
    // used it, recorded on that call's stream (completed events are dropped
    // at the next use).  Freeing the tree waits for these events on the GPU,
    // not on the host.
    static constexpr int kMaxUses = 8;
    cudaEvent_t uses[kMaxUses] = {};
    int nuses = 0;
};

namespace panda {

// Thread-local last error text.
void set_error(const char* fmt, ...);
void clear_error();

// Count one kernel launch (thread-local) and check the launch status.
panda_status note_launch(const char* what);

// Phase timing (CUDA events on the launching stream).  begin(name) starts a
// phase (ending the previous one), end() closes the open phase; finish()
// waits for the last event and adds every phase's time to the thread-local
// table read by panda_phase_times (merged by name).
struct PhaseTimer {
    explicit PhaseTimer(cudaStream_t s);
    ~PhaseTimer();
    void begin(const char* name);
    void end();
    void finish();
  private:
    void mark(const char* name);
    cudaStream_t stream_;
    bool on_;
    std::vector<cudaEvent_t> ev_;
    std::vector<const char*> names_;     // names_[i] = phase started by ev_[i] (nullptr: gap)
    std::vector<int64_t> launches_at_;
};

bool phase_timing_enabled();
// While set on this thread, PhaseTimers record nothing (used around graph capture).
void set_phase_timing_suppressed(bool on);
// Runs fn once for the current device (kernel attributes are per device);
// thread-safe.  A failed fn is retried on the next call.
constexpr int kMaxDevices = 64;
struct PerDeviceOnce {
    std::mutex mu;
    std::atomic<bool> done[kMaxDevices] = {};
};
template <class F>
panda_status once_per_device(PerDeviceOnce& o, F fn)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fn();
    if (o.done[dev].load(std::memory_order_acquire)) return PANDA_OK;
    std::lock_guard<std::mutex> lk(o.mu);
    if (o.done[dev].load(std::memory_order_relaxed)) return PANDA_OK;
    const panda_status st = fn();
    if (st == PANDA_OK) o.done[dev].store(true, std::memory_order_release);
    return st;
}

// Launch attributes of the traversal kernels (set before any graph capture).
panda_status configure_knn_lo();
panda_status configure_knn_hi();
int64_t launches_so_far();

// Convert a CUDA error into a status with a message.
panda_status cuda_fail(cudaError_t e, const char* what);

// Stream-ordered allocation from the device's default pool (cached across
// calls: the pool keeps freed memory for reuse).  The library counts the bytes
// it holds through these two calls (ws_bytes_held): allocations that are live
// now, whatever the pool caches.
panda_status ws_alloc(void** p, size_t bytes, cudaStream_t s, const char* what);
void ws_free(void* p, cudaStream_t s);
long long ws_bytes_held();

// Record that work enqueued on stream s uses tree t (reads its tables, or
// writes them: build, refit).  Thread-safe.
void note_tree_use(const panda_tree* t, cudaStream_t s);
// Make stream s wait for every recorded use of t, then forget them.
void wait_tree_uses(const panda_tree* t, cudaStream_t s);

// Device pointer check: true if p is device memory (or managed) usable by kernels.
bool is_device_ptr(const void* p);

int num_sms();

// Build and query entry points implemented in build.cu / query.cu.
panda_status build_tree(const float* points, int64_t n, int32_t d, int32_t bucket,
                        cudaStream_t stream, panda_tree** out);
// Automatic traversal shape: each lane walks its own query when the queries
// are sparse (fewer than a quarter of the points) in low dimension (d <= 4).
// At d = 10 the search regions of even distant queries overlap, and the
// packet traversal was faster at every query count measured.
inline bool prefer_per_query(long long m, long long n, int d) { return d <= 4 && 4 * m < n; }

panda_status knn_query(const panda_tree* t, const float* queries, int64_t m, int32_t k,
                       int32_t* ids, float* d2, const panda_query_params* params,
                       cudaStream_t stream, unsigned* host_err, int32_t* visits = nullptr,
                       unsigned long long* stats = nullptr);
// All-points query: every point of the tree as a query, output row = its id.
panda_status knn_self(const panda_tree* t, int32_t k, int32_t* ids, float* d2, const panda_query_params* params,
                      cudaStream_t stream, unsigned* host_err, int32_t* visits = nullptr,
                      unsigned long long* stats = nullptr);

// Forests of independent trees (batched form), in build.cu.
struct BuildState;
panda_status forest_create(const long long* set_sizes, int nsets, int d, int bucket, const float* points,
                           cudaStream_t stream, panda_tree* t, BuildState** out);
panda_status forest_enqueue(BuildState* S, cudaStream_t stream);
panda_status forest_collect(BuildState* S, panda_tree* t, unsigned* err, cudaStream_t stream);
void forest_destroy(BuildState* S, cudaStream_t stream);
int forest_levels(const BuildState* S);

}  // namespace panda

#define PANDA_CUDA(call, what)                                  \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return panda::cuda_fail(_e, what); \
    } while (0)

namespace panda {
// Launch with programmatic stream serialization (the kernel calls
// griddep_enter() first): the launch latency between consecutive kernels of one
// stream overlaps the predecessor's last blocks.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// launch_pdl, counted and checked: PANDA_OK or the launch error as a status.
template <typename... KArgs, typename... Args>
panda_status launch_k(const char* what, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                      cudaStream_t stream, Args&&... args)
{
    const cudaError_t e = launch_pdl(kernel, grid, block, smem, stream, std::forward<Args>(args)...);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return note_launch(what);
}
}  // namespace panda

// Launch `kernel` with programmatic dependent launch, count it and check it;
// return the status from the enclosing function on failure.
#define PANDA_LAUNCH(kernel, grid, block, smem, stream, ...)                                              \
    do {                                                                                                   \
        panda_status _ls = panda::launch_k(#kernel, kernel, dim3(grid), dim3(block), (size_t)(smem), (stream), \
                                           __VA_ARGS__);                                                   \
        if (_ls != PANDA_OK) return _ls;                                                                   \
    } while (0)

#define PANDA_LAUNCHED(what)                                    \
    do {                                                        \
        panda_status _s = panda::note_launch(what);             \
        if (_s != PANDA_OK) return _s;                          \
    } while (0)
