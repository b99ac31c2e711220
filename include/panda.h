/*
 * panda.h -- C ABI of the GB300 (sm_103a) kd-tree build and exact KNN library.
 *
 * The method is PANDA's local kd-tree construction and k-nearest-neighbour
 * query (Patwary et al., arXiv 1607.08220): Sec. III-A (steps ii-iv: split
 * levels, bucket stop, leaf packing), Sec. III-A1 (split dimension by maximum
 * sample variance, split value by a sampled histogram, bucket size B) and
 * Algorithm 1 in Sec. III-B/III-C (stack traversal with a top-k heap and
 * bound pruning).  The problem statement followed here is Algorithm 1's
 * signature FINDKNN(T, q, k, r) with r = infinity.
 *
 * Result contract (every entry point that returns neighbours):
 *   - d2(q, x) is the FP32 sum over dimensions 0..d-1, in that order, of
 *     fl(fl(q_i - x_i) * fl(q_i - x_i)), every operation rounded to nearest
 *     even, no fused multiply-add, denormals kept;
 *   - row r of the output lists the k points with the smallest keys
 *     (d2, point index), ascending; ids are the 0-based row indices of the
 *     points given to the build; the answer is unique;
 *   - when the tree holds n < k points, entries n..k-1 of a row are
 *     (id -1, d2 +inf).
 *
 * Conventions:
 *   - Functions without the _host suffix take DEVICE pointers (CUDA global
 *     memory of the current device); a host pointer is rejected with
 *     PANDA_ERR_INVALID_ARGUMENT.  _host variants take host pointers
 *     (pinned or pageable) and copy in and out themselves.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL is
 *     the legacy default stream.
 *   - Outputs are caller-allocated.  No exception crosses this ABI.  No
 *     partial output survives an error: argument errors are found before
 *     anything is enqueued and leave every output untouched; a blocking
 *     device-pointer query (panda_knn, panda_knn_self) that finds a
 *     non-finite query or fails a consistency check after its kernels ran
 *     overwrites every output row with (id -1, d2 +inf); the _host variants
 *     then leave the host outputs untouched; a failed build creates no
 *     handle.  The _async variants return once their work is enqueued and
 *     report no data error.
 *   - Every CUDA failure is reported as PANDA_ERR_CUDA; panda_last_error()
 *     returns the message of the last failure on the calling thread.
 *   - A tree is immutable after its build: concurrent panda_knn calls on one
 *     tree from several streams are allowed.  Every call that enqueues work
 *     on a tree records it (one CUDA event per call); panda_free and
 *     panda_free_async make the GPU wait for that work before the memory goes
 *     back to the pool, so the host never waits in a free.
 *   - Valid ranges: 1 <= n < 2^31, 1 <= d <= 16, 1 <= bucket <= 256,
 *     1 <= k <= 64, m >= 0 (m = 0 does nothing).  Out-of-range values give
 *     PANDA_ERR_INVALID_ARGUMENT (or PANDA_ERR_UNSUPPORTED for d > 16,
 *     k > 64, bucket > 256).  Coordinates must be finite
 *     (PANDA_ERR_NONFINITE_INPUT otherwise).
 */
#ifndef PANDA_H
#define PANDA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct panda_tree panda_tree; /* opaque; owns its device memory */

typedef enum panda_status {
    PANDA_OK = 0,
    PANDA_ERR_INVALID_ARGUMENT = 1,
    PANDA_ERR_NONFINITE_INPUT = 2,
    PANDA_ERR_UNSUPPORTED = 3,
    PANDA_ERR_OUT_OF_MEMORY = 4,
    PANDA_ERR_CUDA = 5,
    PANDA_ERR_TIMEOUT = 6,
    PANDA_ERR_QUEUE_FULL = 7,
    PANDA_ERR_DEPTH = 8 /* a node deeper than 64 levels would still hold > bucket points */
} panda_status;

/* Query point ordering before the traversal (does not change results). */
typedef enum panda_order {
    PANDA_ORDER_NONE = 0,   /* queries traversed in input order */
    PANDA_ORDER_MORTON = 1, /* grouped by a 30-bit Morton code over the tree's root box */
    PANDA_ORDER_LEAF = 2    /* grouped by the leaf bucket each query falls in */
} panda_order;

typedef struct panda_query_params {
    int32_t order;          /* panda_order; default PANDA_ORDER_LEAF */
    int32_t transpose_max;  /* scan shape: a leaf bucket needed by at most this many of
                               a warp's 32 queries is scanned with lanes holding points
                               (queries broadcast in turn), otherwise with lanes holding
                               queries; 0 = default (16), 32 = always the former,
                               -1 = always the latter.  Never changes results. */
    int32_t traversal;      /* PANDA_TRAVERSAL_*: 0 = automatic (per-query when the
                               queries are sparse, fewer than n/4, and d <= 4), never
                               changes results */
    int32_t bounded;        /* 1: Algorithm 1's search radius r applies -- only points
                               with d2 <= max_d2 (= r^2, FP32) are neighbours; rows
                               with fewer than k pad with (-1, +inf).  Not with
                               panda_knn_visits (PANDA_ERR_UNSUPPORTED). */
    float max_d2;           /* >= 0 (NaN is invalid); used when bounded = 1 */
    int32_t reserved;
} panda_query_params;

/* Traversal shape of the KNN kernel. */
enum {
    PANDA_TRAVERSAL_AUTO = 0,
    PANDA_TRAVERSAL_PACKET = 1,   /* a warp's 32 spatially grouped queries share one stack */
    PANDA_TRAVERSAL_PER_QUERY = 2 /* each lane walks its own query with its own stack */
};

typedef struct panda_tree_info {
    int64_t n;          /* points */
    int32_t d;          /* dimensions */
    int32_t bucket;     /* B: maximum points per leaf */
    int64_t num_nodes;  /* inner + leaf nodes */
    int64_t num_leaves;
    int32_t depth;      /* deepest node (root = 0) */
    int32_t node_floats;  /* floats per node record (header + box, padded to 4) */
    int32_t point_floats; /* floats per packed point (coordinates + id, padded to 4) */
    int32_t subtree_threshold; /* nodes of at most this many points were built in shared memory */
    int64_t device_bytes;      /* device memory held by the tree */
    int64_t node_slots;        /* records in the node table: num_nodes plus unused
                                  records no node refers to */
} panda_tree_info;

/* ---- construction: Sec. III-A (ii)-(iv) and Sec. III-A1 --------------------
 * points: device, row-major [n][d] FP32.  Copied into the tree (leaf order,
 * one packed record per point), so the caller may free it once the call
 * returns (for _async: once `stream` has passed the build).
 * bucket: B, the leaf capacity (the paper's best value is 32).
 * The build synchronises `stream` once, between its data-parallel levels and
 * its shared-memory subtree stage, to size the latter. */
panda_status panda_build(const float* points, int64_t n, int32_t d, int32_t bucket,
                         panda_tree** out);
panda_status panda_build_async(const float* points, int64_t n, int32_t d, int32_t bucket,
                               void* stream, panda_tree** out);
/* Same with host `points`; copies host->device inside the call. */
panda_status panda_build_host(const float* points, int64_t n, int32_t d, int32_t bucket,
                              void* stream, panda_tree** out);

/* ---- query: Algorithm 1 (corrected), Sec. III-B/III-C ------------------------
 * queries: device [m][d] FP32 (d = the tree's d); out_ids: device [m][k] int32;
 * out_d2: device [m][k] FP32.  panda_knn blocks until the results are written;
 * panda_knn_async only enqueues on `stream` (params may be NULL for defaults).
 * The query uses a temporary device workspace of about 12*m bytes for the
 * query ordering (from the stream-ordered pool; freed in stream order). */
panda_status panda_knn(const panda_tree* tree, const float* queries, int64_t m, int32_t k,
                       int32_t* out_ids, float* out_d2);
panda_status panda_knn_async(const panda_tree* tree, const float* queries, int64_t m, int32_t k,
                             int32_t* out_ids, float* out_d2,
                             const panda_query_params* params, void* stream);
/* Same with host queries/outputs; copies in and out inside the call and returns
 * after the results are on the host. */
panda_status panda_knn_host(const panda_tree* tree, const float* queries, int64_t m, int32_t k,
                            int32_t* out_ids, float* out_d2, const panda_query_params* params,
                            void* stream);

/* All-points query (the self-KNN of the paper's particle workloads): every
 * point of the tree is a query, so no query buffer is read -- the queries are
 * the tree's own packed points, taken in leaf order, which also makes the
 * query ordering pass unnecessary.  Row i of out_ids / out_d2 (device,
 * [n][k]) holds the neighbours of input point i, exactly what panda_knn gives
 * with queries = the points the tree was built from (a point is its own
 * rank-0 neighbour unless an exact duplicate has a smaller id).  params:
 * order is ignored, traversal PER_QUERY is honoured (AUTO means packet),
 * transpose_max as for panda_knn_async.  panda_knn_self blocks until the
 * results are written; _async only enqueues; _host writes host outputs and
 * returns after they are on the host. */
panda_status panda_knn_self(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2);
panda_status panda_knn_self_async(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2,
                                  const panda_query_params* params, void* stream);
panda_status panda_knn_self_host(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2,
                                 const panda_query_params* params, void* stream);
/* Enqueue-only host variant: the copy into out_ids / out_d2 (pinned host
 * memory, or the copy blocks) is queued on `stream` and the call returns;
 * the results are there once the stream has passed it.  Queries of the next
 * batch can then run on another stream while this one's results travel.
 * Device-side consistency checks are not read back (the blocking variants
 * report them). */
panda_status panda_knn_self_host_async(const panda_tree* tree, int32_t k, int32_t* out_ids, float* out_d2,
                                       const panda_query_params* params, void* stream);

/* ---- refit: particles moved (Sec. II: the tree is rebuilt every few steps of a
 * simulation; in between it can be refitted) ---------------------------------
 * points: device [n][d] FP32, the new coordinates of the tree's points in the
 * original id order.  Every point keeps its leaf; leaf boxes become the exact
 * boxes of the new coordinates and inner boxes the union of their children's,
 * so later queries are exact for the new positions (they slow down as the
 * split planes drift away from the points).  Synchronises `stream`; a
 * non-finite coordinate returns PANDA_ERR_NONFINITE_INPUT and changes nothing.
 * Trees of the batched or served forms are not refitted. */
panda_status panda_refit(panda_tree* tree, const float* points, void* stream);

/* ---- prediction from a KNN result (Sec. I: majority vote for classification,
 * average for regression) ----------------------------------------------------
 * ids: device [m][k] int32 as written by a query on a tree of n points (entries
 * outside [0, n), such as the -1 padding, are ignored).  labels / values:
 * device [n], indexed by point id.  Per row: panda_knn_vote writes the label
 * with the largest count among the valid neighbours (the smallest label among
 * equal counts; -1 when there is none); panda_knn_mean writes the FP32 sum of
 * their values in rank order (nearest first, from +0) divided in FP32 by their
 * number (NaN when there is none).  Both only enqueue on `stream`.  No
 * counterpart in the paper's code: it names these uses of the neighbours. */
panda_status panda_knn_vote(const int32_t* ids, int64_t m, int32_t k, const int32_t* labels, int64_t n,
                            int32_t* out_labels, void* stream);
panda_status panda_knn_mean(const int32_t* ids, int64_t m, int32_t k, const float* values, int64_t n,
                            float* out_values, void* stream);

/* The same answers as panda_knn_async (default parameters) for callers that
 * cannot allocate device memory while they query.  No counterpart in the
 * paper: the query ordering's scratch space is a fixed file-scope device array
 * (12.6 MB, present on every device that loads the library until exit)
 * instead of stream-ordered allocations, so the call makes no
 * cudaMalloc/cudaFree and calls no allocating library routine.  m is limited
 * to 1048576 (2^20) queries per call; larger m returns PANDA_ERR_UNSUPPORTED.
 * All calls share the array: calls that overlap on the GPU race, so serialise
 * them (one stream).  The first call on a device looks up the array's address;
 * make it before any stream capture.  The address is cached per device for the
 * life of the process and does not survive cudaDeviceReset.  Differences from
 * panda_knn_async, none of which changes a result: the leaf-ordering histogram
 * has at most 2^20 - 1 bins (2^22 there), dense query sets (2m >= n) keep
 * 32-query packets instead of one bin's queries per warp (panda_knn_async's
 * job list), non-finite queries are not reported, and the call records no use
 * of the tree (that takes an event): free the tree only once `stream` has
 * passed this call. */
panda_status panda_knn_noalloc(const panda_tree* tree, const float* queries, int64_t m, int32_t k,
                               int32_t* out_ids, float* out_d2, void* stream);

/* Releases the tree (NULL-safe).  The handle is gone at once; the device
 * memory returns to the stream-ordered pool, in the order of the legacy
 * default stream, after every recorded use of the tree (its build, each query
 * and refit, on whatever stream they ran) has finished on the GPU.  The host
 * does not wait.  Trees read by panda_tree_load (cudaMalloc'd tables) are
 * released with cudaFree, which waits for the device. */
void panda_free(panda_tree* tree);
/* The same, in the order of `stream`: the memory returns to the pool after
 * the work queued on `stream` before the call and every recorded use of the
 * tree have run. */
void panda_free_async(panda_tree* tree, void* stream);

/* ---- batched form: many independent point sets, Sec. III-B (query batching) ---
 * A batch owns device buffers for nsets sets of fixed sizes: all points
 * (set s = rows point_off[s] .. point_off[s+1]-1 of a [sum n_points][d]
 * array), all queries (likewise), and the outputs (set s's [n_queries][k]
 * block starts at out_off[s] elements).  panda_batch_run enqueues, with no host
 * synchronisation, one build of every set's kd-tree (a forest) and the exact
 * KNN of every set's queries against its own tree; the first run captures the
 * sequence in a CUDA graph, later runs replay it (write new inputs into the
 * same buffers between runs).  Ids in the outputs are row indices within the
 * set.  panda_batch_status reports the last run's errors once `stream` has
 * passed it (it synchronises `stream`). */
typedef struct panda_batch panda_batch;
typedef struct panda_set_desc {
    int64_t n_points;   /* >= 1 */
    int64_t n_queries;  /* >= 0 */
    int32_t k;          /* 1 .. 64 */
    int32_t reserved;
} panda_set_desc;
panda_status panda_batch_create(const panda_set_desc* sets, int32_t nsets, int32_t d, int32_t bucket,
                                panda_batch** out);
panda_status panda_batch_buffers(panda_batch* batch, float** points, float** queries, int32_t** out_ids,
                                 float** out_d2);
/* point_off, query_off, out_off: host arrays of nsets + 1 entries (each may be NULL). */
panda_status panda_batch_offsets(const panda_batch* batch, int64_t* point_off, int64_t* query_off,
                                 int64_t* out_off);
/* Query parameters of the batch's traversal (order must be PANDA_ORDER_LEAF
 * or params NULL for defaults).  traversal AUTO chooses per set (per-query
 * when the set has fewer than n/4 queries and d <= 4); PACKET or PER_QUERY applies to
 * every set.  After a run this waits for the whole device and drops the
 * captured graph; the next panda_batch_run captures it again. */
panda_status panda_batch_set_query_params(panda_batch* batch, const panda_query_params* params);
panda_status panda_batch_run(panda_batch* batch, void* stream);
panda_status panda_batch_status(panda_batch* batch, void* stream);
/* Forest statistics of the last run; *kernels_per_run = kernels in the captured graph. */
panda_status panda_batch_info(const panda_batch* batch, panda_tree_info* info, int64_t* kernels_per_run);
void panda_batch_free(panda_batch* batch);

/* ---- served form: resident trees, continuous batching (Sec. III-B pipelining) --
 * A server keeps trees resident and answers KNN requests asynchronously.  A
 * scheduler thread takes queued requests in arrival order -- any tree, size
 * and k (1..64) -- into batches of at most max_batch_queries queries (a larger
 * request runs alone) and runs each batch as one query-ordering pass (the
 * queries of all requests on one tree sorted together by its leaves) and one
 * traversal launch; up to four batches are in flight, each on its own
 * stream, so requests arriving while batches run join the next one and small
 * batches overlap.  Results equal panda_knn's.  A
 * request with a non-finite query coordinate finishes with
 * PANDA_ERR_NONFINITE_INPUT (its output rows are then unspecified); the other
 * requests of its batch are unaffected.
 * panda_server_add_tree builds on the server's own stream (queries continue)
 * and is refused with PANDA_ERR_OUT_OF_MEMORY if mem_budget_bytes (0 = no
 * budget) or the device's free memory cannot hold it.  Requests reference
 * caller-owned device buffers, which must stay valid until the request is
 * done.  Times are nanoseconds since the server was created. */
typedef struct panda_server panda_server;
panda_status panda_server_create(int64_t mem_budget_bytes, int64_t max_batch_queries, panda_server** out);
panda_status panda_server_add_tree(panda_server* server, const float* points, int64_t n, int32_t d,
                                   int32_t bucket, int32_t* tree_id);
panda_status panda_server_submit(panda_server* server, int32_t tree_id, const float* queries, int64_t m,
                                 int32_t k, int32_t* out_ids, float* out_d2, int64_t* request_id);
/* *done = 1 once the request finished; returns the request's status. */
panda_status panda_server_poll(panda_server* server, int64_t request_id, int32_t* done);
/* Waits at most timeout_us; PANDA_ERR_TIMEOUT if the request is not done by then. */
panda_status panda_server_wait(panda_server* server, int64_t request_id, int64_t timeout_us);
panda_status panda_server_request_info(panda_server* server, int64_t request_id, int64_t* t_submit_ns,
                                       int64_t* t_done_ns, int64_t* batch_id);
int64_t panda_server_now_ns(panda_server* server);
panda_status panda_server_stats(panda_server* server, int64_t* batches, int64_t* requests, int64_t* pending,
                                int64_t* bytes_used);
/* Query batches are admitted by memory as well: before a batch starts, the
 * scheduler reserves an upper bound of its device scratch (query keys and
 * permutation, the counting-sort histogram, request descriptors, the job
 * queue), and the batch starts only if the reservation fits both what
 * mem_budget_bytes leaves after the resident trees and the batches in flight,
 * and the device's free memory (plus what the stream-ordered pool holds
 * unused).  Requests that do not fit wait in the queue, in arrival order,
 * until batches in flight finish; a request that cannot fit even with nothing
 * in flight finishes with PANDA_ERR_OUT_OF_MEMORY.
 * panda_server_set_queue_limit caps the queries waiting to be batched (0: no
 * cap, the default): a submit that would exceed it returns
 * PANDA_ERR_QUEUE_FULL and queues nothing.  panda_server_admission reports
 * the scratch bytes reserved by the batches in flight, how many requests
 * have waited for memory so far, and the queries waiting now. */
panda_status panda_server_set_queue_limit(panda_server* server, int64_t max_pending_queries);
panda_status panda_server_admission(panda_server* server, int64_t* scratch_reserved, int64_t* deferred_requests,
                                    int64_t* pending_queries);
/* Finishes queued and running requests, then releases every tree and the server. */
void panda_server_destroy(panda_server* server);

/* ---- autotuner ------------------------------------------------------------------
 * Times every combination of bucket size {16, 32, 64}, query order {none,
 * Morton, leaf}, traversal shape {packet with scan-shape switch -1, 4, 8, 12,
 * 16, 32 (see panda_query_params.transpose_max), per-query} on the given
 * device points and a device
 * sample of queries ([m_sample][d]), and returns the combination with the
 * smallest build time + query time scaled to m_total queries per build.  None
 * of these knobs changes a result.  The choice is also cached per (d,
 * ceil(log2 n), k, ceil(log2 m_total)) for panda_tune_lookup.  Builds 6 trees. */
typedef struct panda_tune_result {
    int32_t bucket;
    int32_t order;          /* panda_order */
    int32_t transpose_max;  /* for panda_query_params */
    int32_t traversal;      /* PANDA_TRAVERSAL_PACKET or _PER_QUERY */
    float build_ms;         /* timed build with this bucket */
    float query_ms;         /* query time scaled to m_total queries */
    float score_ms;         /* build_ms + query_ms */
    float reserved2;
} panda_tune_result;
panda_status panda_tune(const float* points, int64_t n, int32_t d, const float* queries, int64_t m_sample,
                        int64_t m_total, int32_t k, void* stream, panda_tune_result* out);
panda_status panda_tune_lookup(int32_t d, int64_t n, int32_t k, int64_t m_total, panda_tune_result* out);

/* ---- inspection -------------------------------------------------------------
 * panda_tree_get_info fills *info.  panda_tree_copy copies the tree's node
 * table ([node_slots][node_floats] floats) and packed points
 * ([n][point_floats] floats) to host buffers of those sizes (either may be
 * NULL).  Let dp be d rounded up to the padded width (2, 3, 4, 8, 10 or 16);
 * padded coordinates are 0.  Node record: int32 a, int32 b, float split,
 * uint32 meta, then lo[dp], hi[dp], zero padding to a multiple of 4 floats;
 * meta bit 31 = leaf, bit 30 = index split, bits 0..4 = split dimension; an
 * inner node's children are nodes a and a+1 and b is the right child's first
 * packed position (the all-points query walks down to a leaf by it; a table
 * with other b values still answers exactly, only slower); a leaf holds the
 * packed points a .. a+b-1.  Packed point: dp coordinates, then the point's id as int32
 * bits in float slot dp, zero padding to a multiple of 4 floats. */
panda_status panda_tree_get_info(const panda_tree* tree, panda_tree_info* info);
panda_status panda_tree_copy(const panda_tree* tree, float* host_nodes, float* host_points);
/* Checkpoint: panda_tree_save writes the tree (header, root box, node table,
 * packed points) to the file at `path`; panda_tree_load reads one back onto
 * the current device as a new tree (free it with panda_free).  Loading checks
 * the header, that the stored ids are a permutation of 0..n-1 and that every
 * node record stays inside the tables (PANDA_ERR_INVALID_ARGUMENT otherwise).
 * Queries on a loaded tree return what they return on the saved one.  The
 * paper has no counterpart: it rebuilds trees. */
panda_status panda_tree_save(const panda_tree* tree, const char* path);
panda_status panda_tree_load(const char* path, panda_tree** out);

/* ---- diagnostics --------------------------------------------------------------
 * Phase timing: enable = 1 records CUDA events on the launching stream around
 * each phase of the next builds/queries; enable = 2 records only the
 * traversal phase ("query.traverse"), so no event separates the other kernels
 * (consecutive kernels then overlap their launches: programmatic dependent
 * launch); 0 turns it off.  panda_phase_times writes up to `cap` (name,
 * milliseconds, launches) triples of the last call that finished on this
 * thread and returns how many there were. */
void panda_set_phase_timing(int32_t enable);
int32_t panda_phase_times(const char** names, float* ms, int32_t* launches, int32_t cap);
/* Same as panda_knn_async (queries NULL and m = the tree's n: the all-points
 * query of panda_knn_self_async), and also writes (each optional, device memory):
 * out_visits [m][2] int32: per query, the tree nodes whose bound did not
 * exceed its k-th distance when popped, and the bucket points it scanned in
 * those nodes -- the work Algorithm 1 needs for that query, used to state
 * algorithmic FLOPs; out_stats [12] uint64, ADDED to (zero it first): warps,
 * inner nodes, bucket chunks, chunks scanned with lanes = queries, query
 * broadcasts of the lanes = points scan, insertion rounds (lanes = points
 * scans; the lanes = queries scan inserts as it goes), candidates,
 * insertions, pops no lane needed, and the insertion rounds, candidates and
 * insertions of the lanes = points scans alone (per-warp event counts of the
 * packet traversal kernel). */
panda_status panda_knn_visits(const panda_tree* tree, const float* queries, int64_t m, int32_t k,
                              int32_t* out_ids, float* out_d2, int32_t* out_visits,
                              uint64_t* out_stats, const panda_query_params* params, void* stream);
/* Number of kernels this library launched on this thread so far. */
int64_t panda_kernel_launches(void);
/* Fault injection for tests of the host-side error paths (no GPU fault is
 * involved): after `after` >= 0 further device workspace allocations (the
 * stream-ordered pool: scratch, staging buffers, tree tables) succeed, the
 * next one fails as if the device were out of memory -- the call returns
 * PANDA_ERR_OUT_OF_MEMORY, frees what it held and launches nothing on the
 * missing buffer -- and injection is off again; `after` < 0 turns it off.
 * Process-wide.  panda_debug_pool_used writes the bytes the library holds in
 * the stream-ordered pool right now (its own count of live allocations:
 * trees, the batched form's forest and every call's workspace, on all
 * devices; memory the pool caches for reuse and other users' allocations
 * are not counted), so a test can check that a failed call leaked nothing. */
panda_status panda_debug_fail_alloc(int64_t after);
panda_status panda_debug_pool_used(int64_t* bytes);

const char* panda_status_string(panda_status status);
const char* panda_last_error(void); /* thread-local; "" if none */
const char* panda_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PANDA_H */
