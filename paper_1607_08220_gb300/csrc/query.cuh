// query.cuh -- exact KNN traversal kernel (Algorithm 1, corrected) for sm_103a.
//
// One warp serves up to 32 queries (one per lane) that were grouped by spatial
// key, so they traverse nearly the same nodes: 32 consecutive queries in leaf
// or Morton order, or -- for the all-points query and dense leaf-ordered
// query sets -- the queries of one leaf (a job list), so that no packet
// straddles two leaves.  The warp walks one shared stack
// (Algorithm 1's S): at every popped node each lane computes its own bound,
// the squared distance from its query to the node's tight box, and the node
// is skipped only when every lane's bound is strictly greater than its current
// k-th distance (corrections C1, C3).  Inner nodes push the far child first
// and the near child last, as Algorithm 1 does; the near side is the one the
// majority of the lanes that need the node fall on.
//
// Sparse query sets (fewer queries than a quarter of the points) leave the 32
// queries of a warp far apart, and a shared stack would walk the union of
// their paths; there each lane walks its own query instead (knn_lane_solo).
//
// A leaf bucket is staged once into shared memory, structure-of-arrays, and
// scanned (Sec. III-C: the bucket scan is the SIMD-friendly part) in one of
// two shapes, chosen per bucket by how many lanes need it:
//   * many lanes: every lane computes its distance to all staged points
//     (four at a time over the 32 staging slots, padded with far sentinels)
//     and inserts each candidate at once, so its radius tightens within
//     the bucket (measured 7% faster than marking candidates first);
//   * few lanes: the warp turns around -- lane j holds point j and the
//     needing queries are broadcast one at a time -- so idle lanes do not
//     pay for the scan; each needing lane then inserts the candidates
//     marked for it.
// Candidates are points whose distance does not exceed the lane's current
// k-th distance; they enter with the exact key (d2 bits << 32 | id) into the
// lane's heap H of the k best keys: a max-heap in shared memory (interleaved
// by lane, so the lanes of a warp hit distinct banks), whose root is the
// radius r' (correction C2; with a search radius r, r' never exceeds r^2).
// At the end the heap is emptied in order into the output row.
#pragma once

#include "common.cuh"

namespace panda {

// One request of a served batch: its queries are batch rows
// [row_begin, row_begin + m) and its results go to ids / d2 ([m][k]).
struct KnnReq {
    const float* queries;
    int* ids;
    float* d2;
    unsigned* err;   // the request's own error word (non-finite query)
    int k, row_begin;
};

// One query set against one tree (one set of a batched forest, or all the
// requests of a served batch on one tree).  Rows of `queries` are the set's
// queries; `perm` (may be null) lists them in traversal order as row_base +
// row; ids written are stored ids - id_base.  With `reqs` the set spans
// several requests: perm lists batch rows, and each lane finds its request
// (queries, k, outputs) by row.
struct KnnSet {
    const float4* nodes;
    const float4* pts;
    long long num_nodes, npts;
    const float* queries;
    const int* perm;
    int* ids;
    float* d2;
    long long m;
    int root, id_base, k, row_base;
    int solo;   // 1: each lane walks its own query (sparse query sets); 0: warp packets
    int nreq;   // entries of reqs (0: the set is one request, fields above)
    const KnnReq* reqs;
};
// A warp job: traversal positions [pos, pos + 32) of one set.
struct KnnJob {
    int set, pos;
};

struct KnnArgs {
    const KnnSet* sets;   // multi-set launch (with jobs); null for the single-tree fields below
    const KnnJob* jobs;
    int njobs;
    int* job_head;        // device work-queue head (persistent warps take jobs from it)
    const float4* nodes;
    const float4* pts;
    const float* queries;
    const int* perm;      // sorted position -> query row (nullptr: identity)
    int* ids;
    float* d2;
    unsigned* err;
    int* visits;          // optional [m][2]: nodes and points each query needed
    unsigned long long* stats;  // optional [8] event counters (diagnostics)
    long long m;
    long long num_nodes;
    long long npts;
    int d, k;
    int transpose_max;    // use the transposed scan when at most this many lanes need a bucket
    int solo;             // single tree: per-query traversal; many sets: some set has solo set
    int nreq;             // single tree serving several requests: entries of reqs
    const KnnReq* reqs;   // (queries / ids / d2 / k above unused; perm lists batch rows)
    int self_q;           // single tree: the queries are the tree's own points, taken in
                          // leaf order from the packed records (queries, perm unused)
    const int2* pos_jobs;    // warp w takes the positions [x, x + y) of job w (y <= 32):
    const int* pos_njobs;    // one leaf's queries, or a 32-query piece of them
    long long pos_jobs_cap;  // warps launched for the jobs (their number is at most this)
    unsigned long long rkey; // radius-bounded query (kKnnRadius): key (max_d2 bits, 0xffffffff),
                             // a point is a neighbour only if its key is below it; 0: unbounded
};

// Kernel modes: one tree and one query set; one tree and the queries of
// several requests (per-lane request lookup); many sets from a job queue (a
// set may span several requests); one tree and one query set with the work
// counters (visits, stats) compiled in; one tree and one query set with a
// search radius (Algorithm 1's r).
enum KnnMode { kKnnOneSet = 0, kKnnOneTreeReqs = 1, kKnnManySets = 2, kKnnStats = 3, kKnnRadius = 4 };

constexpr unsigned long long kKeyEmpty = (0x7f800000ull << 32) | 0xffffffffull;
constexpr int kKnnThreads = 128;

// Replace the root of the lane's max-heap h[0..k) (stride kKnnThreads) by c
// and sift it down.  Keys are unique, so c never equals a child.  h[k] must
// hold 0, which no child exceeds, so a missing right child needs no test.
__device__ __forceinline__ void heap_replace_root(unsigned long long* h, int k, unsigned long long c)
{
    int i = 0;
    for (;;) {
        const int l = 2 * i + 1;
        if (l >= k) break;
        const unsigned long long cl = h[l * kKnnThreads];
        const unsigned long long cr = h[(l + 1) * kKnnThreads];
        const bool right = cr > cl;
        const unsigned long long cm = right ? cr : cl;
        if (cm < c) break;
        h[i * kKnnThreads] = cm;
        i = right ? l + 1 : l;
    }
    h[i * kKnnThreads] = c;
}

// The packet traversal's DFS stack (Algorithm 1's S) is the same for every lane
// of the warp, so it is held once, spread over the warp's registers: entry j
// lives in lane (j mod 32)'s slot j / 32.  A push writes one lane's slot, a
// pop reads the top entry back with one shuffle; no local memory is involved.
// Algorithm 1 pushes the far child and then the near child and pops the near
// child at once; the traversal keeps the near child as its next node instead
// and pushes only the far one (the same visit order), so the stack holds at
// most one far sibling per level above the current node: 64 entries cover the
// deepest valid tree (an inner node lies above depth kMaxDepth).
struct WarpStack {
    int s0 = 0, s1 = 0;
    static constexpr int kCap = 64;
    __device__ __forceinline__ void push(int& sp, int v, int lane)
    {
        if (lane == (sp & 31)) {
            if (sp & 32) s1 = v;
            else s0 = v;
        }
        sp++;
    }
    __device__ __forceinline__ int pop(int& sp) const
    {
        sp--;
        return __shfl_sync(kFull, (sp & 32) ? s1 : s0, sp & 31);
    }
};
static_assert(WarpStack::kCap >= kMaxDepth, "warp stack too small for the deepest tree");

// Squared distance from q to the tight box of a node record (dims in order, unfused).
template <int DP>
__device__ __forceinline__ float record_box_d2(const float4* rec, const float (&q)[DP])
{
    constexpr int NS = (4 + 2 * DP + 3) / 4;
    float f[4 * NS];
#pragma unroll
    for (int r = 1; r < NS; r++) {
        const float4 v = __ldg(rec + r);
        f[4 * r] = v.x;
        f[4 * r + 1] = v.y;
        f[4 * r + 2] = v.z;
        f[4 * r + 3] = v.w;
    }
    float bnd = 0.0f;
#pragma unroll
    for (int k = 0; k < DP; k++) {
        const float g = fmaxf(fmaxf(__fsub_rn(f[4 + k], q[k]), __fsub_rn(q[k], f[4 + DP + k])), 0.0f);
        bnd = __fadd_rn(bnd, __fmul_rn(g, g));
    }
    return bnd;
}

// One lane walks its own query (Algorithm 1 as written, with the corrections):
// its own stack of (node, bound) where a child's bound is its box distance,
// computed at the parent; the far child is pushed only if its bound does not
// exceed r', the near child last; buckets are scanned point by point.
template <int DP, bool RAD>
__device__ __forceinline__ void knn_lane_solo(const KnnArgs& a, const KnnSet& S, const float (&q)[DP],
                                              unsigned long long* h, int K, unsigned long long& kth,
                                              int& vnodes, int& vpts)
{
    constexpr int NV = (DP + 1 + 3) / 4;
    constexpr int NS = (4 + 2 * DP + 3) / 4;
    // Far children wait on the lane's stack with their bounds; the near child
    // is the next node at once (Algorithm 1 pushes it last and pops it first),
    // so the stack holds at most one entry per level above the current node.
    int stn[kMaxDepth];
    float stb[kMaxDepth];
    int sp = 0;
    int node = S.root;
    float nb = 0.0f;   // bound of `node`
    long long budget = 2LL * S.num_nodes + 8;
    for (;;) {
        if (--budget < 0) {
            atomicOr(a.err, kErrInternal);
            break;
        }
        const float kd = __uint_as_float((unsigned)(kth >> 32));
        if (nb > kd) {              // pruned: the next waiting far child
            if (sp == 0) break;
            sp--;
            node = stn[sp];
            nb = stb[sp];
            continue;
        }
        if ((unsigned)node >= (unsigned)S.num_nodes) {
            atomicOr(a.err, kErrInternal);
            break;
        }
        const float4* rec = S.nodes + (long long)node * NS;
        const int4 hd = __ldg(reinterpret_cast<const int4*>(rec));
        vnodes++;
        if ((unsigned)hd.w & kMetaLeaf) {
            if (hd.x < 0 || hd.y < 0 || (long long)hd.x + hd.y > S.npts) {
                atomicOr(a.err, kErrInternal);
                break;
            }
            vpts += hd.y;
            for (int j = 0; j < hd.y; j++) {
                const float4* src = S.pts + (long long)(hd.x + j) * NV;
                float pv[4 * NV];
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    const float4 p = __ldg(src + v);
                    pv[4 * v] = p.x;
                    pv[4 * v + 1] = p.y;
                    pv[4 * v + 2] = p.z;
                    pv[4 * v + 3] = p.w;
                }
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < DP; k++) {
                    const float t = __fsub_rn(q[k], pv[k]);
                    acc = k == 0 ? __fmul_rn(t, t) : __fadd_rn(acc, __fmul_rn(t, t));
                }
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)__float_as_int(pv[DP]);
                if (key < kth) {
                    heap_replace_root(h, K, key);
                    kth = RAD ? min(h[0], a.rkey) : h[0];
                }
            }
            if (sp == 0) break;
            sp--;
            node = stn[sp];
            nb = stb[sp];
        } else {
            const int c0 = hd.x;
            if ((unsigned)(c0 + 1) >= (unsigned)S.num_nodes || sp >= kMaxDepth) {
                atomicOr(a.err, kErrInternal);
                break;
            }
            const float b0 = record_box_d2<DP>(S.nodes + (long long)c0 * NS, q);
            const float b1 = record_box_d2<DP>(S.nodes + (long long)(c0 + 1) * NS, q);
            const int dim = (int)((unsigned)hd.w & kMetaDimMask);
            float qd = 0.0f;
#pragma unroll
            for (int k = 0; k < DP; k++)
                if (k == dim) qd = q[k];
            const bool right_near = qd >= __int_as_float(hd.z);
            const float bn = right_near ? b1 : b0, bf = right_near ? b0 : b1;
            if (bf <= kd) {
                stn[sp] = right_near ? c0 : c0 + 1;   // far child waits
                stb[sp] = bf;
                sp++;
            }
            node = right_near ? c0 + 1 : c0;          // near child next
            nb = bn;
        }
    }
}

// Traversal of one warp job: positions [g0, g0 + 32) of set S.  SOLO_OK
// compiles the per-query traversal in (taken when S.solo is set); without it
// the kernel holds the packet traversal alone and keeps its registers.  REQS
// compiles in the per-lane request lookup of sets that span several requests.
template <int DP, bool SOLO_OK, bool REQS, bool STATS, bool RAD>
__device__ __forceinline__ void knn_warp_job(const KnnArgs& a, const KnnSet& S, long long g0, int cnt,
                                             float (*sx)[32], int* sid, unsigned long long* h)
{
    constexpr int NV = (DP + 1 + 3) / 4;
    constexpr int NS = (4 + 2 * DP + 3) / 4;
    const int lane = threadIdx.x & 31;
    const long long pos = g0 + lane;
    const bool valid = lane < cnt && pos < S.m;
    int qi = 0;
    if (valid) qi = S.perm ? S.perm[pos] - S.row_base : (int)pos;
    const float* qsrc = S.queries;
    int* out_ids = S.ids;
    float* out_d2 = S.d2;
    unsigned* qerr = a.err;
    int K = S.k;
    if (REQS && S.nreq > 0 && valid) {
        // the request holding batch row qi: the last one starting at or before it
        int lo = 0, hi = S.nreq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.reqs[mid].row_begin <= qi) lo = mid; else hi = mid - 1;
        }
        const KnnReq R = S.reqs[lo];
        qsrc = R.queries;
        out_ids = R.ids;
        out_d2 = R.d2;
        qerr = R.err;
        K = R.k;
        qi -= R.row_begin;
    }
    float q[DP];
    bool finite = true;
    if (!REQS && a.self_q) {
        // all-points query: position pos is the packed point pos (coordinates,
        // zero padding, then its id), already finite and in leaf order
        if (valid) {
            const float* pp = reinterpret_cast<const float*>(S.pts + pos * NV);
#pragma unroll
            for (int k = 0; k < DP; k++) q[k] = pp[k];
            qi = __float_as_int(pp[DP]) - S.id_base;
        } else {
#pragma unroll
            for (int k = 0; k < DP; k++) q[k] = 0.0f;
        }
    } else {
#pragma unroll
        for (int k = 0; k < DP; k++) {
            q[k] = (valid && k < a.d) ? qsrc[(long long)qi * a.d + k] : 0.0f;
            finite &= (__float_as_uint(q[k]) & 0x7f800000u) != 0x7f800000u;
        }
    }
    if (!finite) atomicOr(qerr, kErrNonfinite);
    for (int i = 0; i < K; i++) h[i * kKnnThreads] = kKeyEmpty;
    h[K * kKnnThreads] = 0ull;   // sentinel below the heap
    // k-th best key so far (the heap root); invalid lanes never accept anything
    unsigned long long kth = valid ? (RAD ? a.rkey : kKeyEmpty) : 0ull;

    int vnodes = 0, vpts = 0;
    // diagnostics: inner nodes, leaf chunks, lanes=queries chunks, transposed
    // broadcasts, insertion-loop rounds, candidates, insertions
    // 7: pops no lane needed, 8-10: rounds, candidates, insertions of the
    // lanes = points scans
    unsigned st[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const bool stats = STATS && a.stats != nullptr;
    if (SOLO_OK && S.solo) {
        if (valid) knn_lane_solo<DP, RAD>(a, S, q, h, K, kth, vnodes, vpts);
    } else {
    WarpStack stack;
    int sp = 0;
    int node = S.root;
    if (!REQS && a.self_q) {
        // All-points query: the warp's queries are points of the leaf holding
        // position g0.  With no k-th distance known yet every lane needs every
        // node above that leaf, so walk straight down to it (go right where g0
        // is at or past the right child's first position), push each far
        // child, and start the search there.  Any leaf would keep the result
        // exact: the far children and the path cover the whole tree.
        for (int lv = 0; lv <= kMaxDepth; lv++) {
            if ((unsigned)node >= (unsigned)S.num_nodes || sp >= WarpStack::kCap) break;  // flagged below
            const int4 hd = __ldg(reinterpret_cast<const int4*>(S.nodes + (long long)node * NS));
            if ((unsigned)hd.w & kMetaLeaf) break;
            const int right = g0 >= hd.y ? 1 : 0;
            stack.push(sp, hd.x + 1 - right, lane);
            node = hd.x + right;
            if (STATS) vnodes += valid;
            if (stats) st[0]++;
        }
    }
    // A valid tree is visited in at most 2 * num_nodes steps; the cap only
    // guarantees termination (with an error flag) should a node table be corrupt.
    unsigned budget = (unsigned)min(S.num_nodes + 8, 0xffffffffLL);
    for (;;) {
        if (budget-- == 0 || (unsigned)node >= (unsigned)S.num_nodes) {
            if (lane == 0) atomicOr(a.err, kErrInternal);
            break;
        }
        const float4* rec = S.nodes + (long long)node * NS;
        float f[4 * NS];
#pragma unroll
        for (int r = 0; r < NS; r++) {
            const float4 v = __ldg(rec + r);
            f[4 * r] = v.x;
            f[4 * r + 1] = v.y;
            f[4 * r + 2] = v.z;
            f[4 * r + 3] = v.w;
        }
        // bound: squared distance to the tight box, dims in order, unfused
        float bnd = 0.0f;
#pragma unroll
        for (int k = 0; k < DP; k++) {
            const float g = fmaxf(fmaxf(__fsub_rn(f[4 + k], q[k]), __fsub_rn(q[k], f[4 + DP + k])), 0.0f);
            bnd = __fadd_rn(bnd, __fmul_rn(g, g));
        }
        const float kd = __uint_as_float((unsigned)(kth >> 32));
        const bool need = valid && !(bnd > kd);
        const unsigned needm = __ballot_sync(kFull, need);
        if (!needm) {
            if (stats) st[7]++;
            if (sp == 0) break;       // nothing left on the stack: done
            node = stack.pop(sp);
            continue;
        }
        if (STATS) vnodes += need;
        const int h0 = __float_as_int(f[0]);
        const int h1 = __float_as_int(f[1]);
        const unsigned meta = __float_as_uint(f[3]);
        if (meta & kMetaLeaf) {
            if (h0 < 0 || h1 < 0 || (long long)h0 + h1 > S.npts) {
                if (lane == 0) atomicOr(a.err, kErrInternal);
                break;
            }
            for (int b0 = 0; b0 < h1; b0 += 32) {
                const int c = min(32, h1 - b0);
                __syncwarp();
                if (lane < c) {
                    const float4* src = S.pts + (long long)(h0 + b0 + lane) * NV;
#pragma unroll
                    for (int v = 0; v < NV; v++) {
                        const float4 p = __ldg(src + v);
                        const float pv[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const int k = 4 * v + e;
                            if (k < DP) sx[k][lane] = pv[e];
                            else if (k == DP) sid[lane] = __float_as_int(pv[e]);
                        }
                    }
                } else {
                    sx[0][lane] = INFINITY;   // sentinel: never within any radius
#pragma unroll
                    for (int k = 1; k < DP; k++) sx[k][lane] = 0.0f;
                    sid[lane] = -1;
                }
                __syncwarp();
                if (STATS && need) vpts += c;
                unsigned cand = 0;
                if (stats) st[1]++;
                const bool lanes_queries = __popc(needm) > a.transpose_max;
                if (lanes_queries) {
                    if (stats) st[2]++;
                    // every lane scans all 32 staged points (sentinels beyond c) and
                    // inserts each candidate at once, tightening its radius as it goes
                    float kdl = need ? kd : -1.0f;
#pragma unroll 1
                    for (int j = 0; j < 32; j += 4) {
                        float acc[4];
#pragma unroll
                        for (int k = 0; k < DP; k++) {
                            const float4 x4 = *reinterpret_cast<const float4*>(&sx[k][j]);
                            const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                            for (int e = 0; e < 4; e++) {
                                const float t = __fsub_rn(q[k], xv[e]);
                                acc[e] = k == 0 ? __fmul_rn(t, t) : __fadd_rn(acc[e], __fmul_rn(t, t));
                            }
                        }
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            if (acc[e] <= kdl) {
                                const unsigned long long key =
                                    ((unsigned long long)__float_as_uint(acc[e]) << 32) | (unsigned)sid[j + e];
                                if (stats) st[5]++;
                                if (key < kth) {
                                    heap_replace_root(h, K, key);
                                    kth = RAD ? min(h[0], a.rkey) : h[0];
                                    kdl = __uint_as_float((unsigned)(kth >> 32));
                                    if (stats) st[6]++;
                                }
                            }
                        }
                    }
                } else {
                    // lanes hold the points; needing queries are broadcast in turn
                    float px[DP];
#pragma unroll
                    for (int k = 0; k < DP; k++) px[k] = sx[k][lane];
                    unsigned rem = needm;
                    if (stats) st[3] += __popc(needm);
                    while (rem) {
                        const int L = __ffs(rem) - 1;
                        rem &= rem - 1;
                        const float kl = __shfl_sync(kFull, kd, L);
                        float acc = 0.0f;
#pragma unroll
                        for (int k = 0; k < DP; k++) {
                            const float t = __fsub_rn(__shfl_sync(kFull, q[k], L), px[k]);
                            acc = k == 0 ? __fmul_rn(t, t) : __fadd_rn(acc, __fmul_rn(t, t));
                        }
                        const unsigned bits = __ballot_sync(kFull, acc <= kl);
                        if (lane == L) cand = bits;
                    }
                }
                if (stats && !lanes_queries) {
                    const unsigned r = __reduce_max_sync(kFull, (unsigned)__popc(cand));
                    st[4] += r;
                    st[8] += r;
                    st[5] += __popc(cand);
                    st[9] += __popc(cand);
                }
                // exact insertion of this lane's candidates
                while (cand) {
                    const int j = __ffs(cand) - 1;
                    cand &= cand - 1;
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k < DP; k++) {
                        const float t = __fsub_rn(q[k], sx[k][j]);
                        acc = k == 0 ? __fmul_rn(t, t) : __fadd_rn(acc, __fmul_rn(t, t));
                    }
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)sid[j];
                    if (key < kth) {
                        heap_replace_root(h, K, key);
                        kth = RAD ? min(h[0], a.rkey) : h[0];
                        if (stats) {
                            st[6]++;
                            if (!lanes_queries) st[10]++;
                        }
                    }
                }
            }
        } else {
            if (stats) st[0]++;
            const int dim = (int)(meta & kMetaDimMask);
            const float sv = f[2];
            float qd = 0.0f;
#pragma unroll
            for (int k = 0; k < DP; k++)
                if (k == dim) qd = q[k];
            const bool right_side = qd >= sv;
            const unsigned br = __ballot_sync(kFull, need && right_side);
            const bool right_near = 2 * __popc(br) >= __popc(needm);
            if (sp >= WarpStack::kCap) {
                if (lane == 0) atomicOr(a.err, kErrInternal);
                break;
            }
            // a lane on the near side needs the far child only if the split
            // plane lies within its k-th distance (the far box lies beyond it;
            // not for index splits, nor where a refit moved points across it)
            const float pg = __fsub_rn(qd, sv);
            const bool far_need = need && ((meta & (kMetaIndex | kMetaCross)) || right_side != right_near ||
                                           !(__fmul_rn(pg, pg) > kd));
            if (__any_sync(kFull, far_need)) stack.push(sp, h0 + (right_near ? 0 : 1), lane);
            node = h0 + (right_near ? 1 : 0);                   // near child next
            continue;
        }
        if (sp == 0) break;   // a bucket was the last node: the traversal is complete
        node = stack.pop(sp);
    }
    }   // packet traversal
    __syncwarp();
    if (stats) {
        // st[0..4], 7, 8 are warp-uniform (counted once per warp); 5, 6, 9, 10 per lane
        st[5] = __reduce_add_sync(kFull, st[5]);
        st[6] = __reduce_add_sync(kFull, st[6]);
        st[9] = __reduce_add_sync(kFull, st[9]);
        st[10] = __reduce_add_sync(kFull, st[10]);
        if (lane == 0) {
            atomicAdd(&a.stats[0], 1ull);
            for (int i = 0; i < 11; i++) atomicAdd(&a.stats[1 + i], (unsigned long long)st[i]);
        }
    }
    if (STATS && a.visits && valid) {
        a.visits[2LL * qi] = vnodes;
        a.visits[2LL * qi + 1] = vpts;
    }
    if (valid) {
        // empty the heap in descending order into positions k-1 .. 0
        int* oi = out_ids + (long long)qi * K;
        float* od = out_d2 + (long long)qi * K;
        for (int sz = K; sz > 0; sz--) {
            const unsigned long long top = h[0];
            const int id = (int)(unsigned)(top & 0xffffffffull);
            oi[sz - 1] = id < 0 ? id : id - S.id_base;
            od[sz - 1] = __uint_as_float((unsigned)(top >> 32));
            if (sz > 1) {
                const unsigned long long last = h[(sz - 1) * kKnnThreads];
                h[(sz - 1) * kKnnThreads] = 0ull;   // sentinel of the shrunk heap
                heap_replace_root(h, sz - 1, last);
            }
        }
    }
}


// Resident blocks per SM the register allocation must allow.  The one-set
// packet traversal at low dimension runs at 12 blocks (40 registers, no
// spill; 2^24 3-D self-KNN 10.28 ms against 10.31 ms at 16 blocks and 32
// registers, which spill a few values); wider points keep about 48 registers.
// The request lookup and the job queue hold a few more values; kernels with
// the per-query traversal keep 64 registers (its per-lane stacks).
constexpr int knn_min_blocks(int dp, int mode, bool solo)
{
    return (solo || mode == kKnnManySets || mode == kKnnStats) ? 8
           : mode == kKnnOneTreeReqs                          ? (dp <= 4 ? 12 : 8)
                                                              : (dp <= 4 ? 12 : 10);
}

// MODE kKnnOneSet / kKnnOneTreeReqs: one tree, warp w takes positions
// [32 w, 32 w + 32).  MODE kKnnManySets: persistent warps take (set, 32
// positions) jobs from a device work queue.  SOLO = false: packet traversal
// only; SOLO = true: each set's shape is chosen by its solo flag.
template <int DP, int MODE, bool SOLO>
__global__ void __launch_bounds__(kKnnThreads, knn_min_blocks(DP, MODE, SOLO)) k_knn(KnnArgs a)
{
    griddep_enter();
    __shared__ __align__(16) float stage_x[kKnnThreads / 32][DP][32];
    __shared__ int stage_id[kKnnThreads / 32][32];
    extern __shared__ unsigned long long heap_mem[];   // [kmax + 1][kKnnThreads]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long* h = heap_mem + threadIdx.x;
    if (MODE != kKnnManySets) {
        // one tree: warp w takes positions [32 w, 32 w + 32)
        KnnSet S;
        S.nodes = a.nodes;
        S.pts = a.pts;
        S.num_nodes = a.num_nodes;
        S.npts = a.npts;
        S.queries = a.queries;
        S.perm = a.perm;
        S.ids = a.ids;
        S.d2 = a.d2;
        S.m = a.m;
        S.root = 0;
        S.id_base = 0;
        S.row_base = 0;
        S.solo = a.solo;
        S.nreq = MODE == kKnnOneTreeReqs ? a.nreq : 0;
        S.reqs = a.reqs;
        S.k = a.k;
        const long long gw = (long long)blockIdx.x * (kKnnThreads / 32) + warp;
        long long g0 = gw * 32;
        int cnt = 32;
        if (MODE != kKnnOneTreeReqs && a.pos_jobs) {
            // one leaf's queries (or a 32-query piece of them) per warp
            if (gw >= *a.pos_njobs) return;
            const int2 jb = a.pos_jobs[gw];
            g0 = jb.x;
            cnt = jb.y;
        }
        if (g0 >= a.m) return;
        knn_warp_job<DP, SOLO, MODE == kKnnOneTreeReqs, MODE == kKnnStats, MODE == kKnnRadius>(
            a, S, g0, cnt, stage_x[warp],
                                                                           stage_id[warp], h);
        return;
    }
    // many sets: persistent warps take jobs from the device work queue
    for (;;) {
        int j = 0;
        if (lane == 0) j = atomicAdd(a.job_head, 1);
        j = __shfl_sync(kFull, j, 0);
        if (j >= a.njobs) break;
        const KnnJob jb = a.jobs[j];
        const KnnSet S = a.sets[jb.set];
        knn_warp_job<DP, SOLO, true, false, false>(a, S, jb.pos, 32, stage_x[warp], stage_id[warp], h);
        __syncwarp();
    }
}

}  // namespace panda
