// build.cu -- kd-tree construction on GB300 (sm_103a).
//
// Method (arXiv 1607.08220): Sec. III-A steps ii-iv and Sec. III-A1.
//   * Data-parallel levels (step ii): every node with more than T points is
//     split by grid-wide passes, one level at a time: a 1024-point sample per
//     node gives the split dimension (maximum sample variance) and the sorted
//     "interval points"; a histogram of all node points over those interval
//     points gives the split value closest to 50% (Sec. III-A1); a stable
//     partition then scatters coordinates and ids to the other ping-pong
//     buffer.  Points move as coalesced structure-of-arrays columns.
//   * Subtree stage (step iii): every node of at most T points is finished by
//     one warp in shared memory, depth-first, with the same split rule
//     (with every point in the sample the rule is an exact selection).
//   * Packing (step iv): leaves of at most B points are written contiguously
//     as packed records (coordinates + id) in leaf order.
// Every node stores its tight bounding box (level-stage boxes are the union of
// their children's, computed bottom-up at the end).
//
// Split rule readings (identical in the CPU oracle, written independently):
//   sample positions floor(j*n/S'), S' = min(1024, n); FP32 variance summed
//   in 32 strided partials then a pairwise tree; argmax with ties to the lowest
//   dimension; c_j = #{x < v_j}; j* = argmin |2c_j - n| (ties to the smallest
//   j); left = x[dim] < s; duplicate fallback (next value above the node
//   minimum) and index split for constant nodes.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace panda {

struct BuildArgs {
    int n, d, dp, bucket, T, n_pad;
    const float* in;
    float* X[2];
    int* ID[2];
    Active* act[2];
    int act_cap;
    int* tile_base[2];
    Tile* tiles[2];
    int tile_cap;
    int* tleft;
    int* tleftoff;
    int* tbins;   // [tiles][1 + kWin]: a tile's count below the window, then its window bins
    float* vs;
    int* nhist;
    float* nvar;
    int* ndim;
    int* nmode;
    float* nsplit;
    int* nleft;
    int* nsel;
    Small* small;
    int small_cap;
    int* lvl_nodes;
    int* lvl_count;
    int* chunk_act;     // [chunks] children of level-list chunk c going to the next level
    int* chunk_small;   // [chunks] ... going to the subtree stage
    int* chunk_tiles;   // [chunks] tiles of next-level-list chunk c
    int chunk_cap;
    int lvl_stride;
    int* cnt;
    unsigned* err;
    const int* set_off;   // forest: [nsets + 1] point offsets of independent sets (null: one tree)
    int nsets;
    float4* nodes;
    long long node_cap;
    int ns;
    float4* pts;
    int nv;
};

__device__ __forceinline__ bool finite_bits(float v)
{
    return (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u;
}

// ------------------------------------------------------------------ A1

__global__ void k_transpose(BuildArgs a)
{
    griddep_enter();
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_pad; i += stride) {
        if (i < a.n) {
            for (int k = 0; k < a.d; k++) {
                float v = a.in[i * a.d + k];
                bad |= !finite_bits(v);
                a.X[0][(long long)k * a.n_pad + i] = v;
            }
            a.ID[0][i] = (int)i;
        } else {
            for (int k = 0; k < a.d; k++) a.X[0][(long long)k * a.n_pad + i] = 0.0f;
            a.ID[0][i] = -1;
        }
    }
    if (bad) atomicOr(a.err, kErrNonfinite);
}

// ------------------------------------------------------------------ block helpers

// Exclusive scan of one int per thread over the block (blockDim multiple of 32,
// <= 1024).  Returns the exclusive prefix; *total gets the block sum.
__device__ int block_excl_scan(int v, int* sh /*[33]*/, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = warp_incl_scan(v);
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? sh[lane] : 0;
        int wi = warp_incl_scan(w);
        if (lane < nw) sh[lane] = wi - w;
        if (lane == nw - 1) sh[32] = wi;
    }
    __syncthreads();
    int r = sh[warp] + incl - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// Tiles of the active list `x` (count A): node a covers [start, start+count),
// cut at absolute multiples of kTile so that interior tiles are aligned.
constexpr int kPlanPer = 1;   // consecutive active nodes per thread in one pass of the child plan
constexpr int kChildThreads = 256;
constexpr int kChildChunk = kChildThreads * kPlanPer;   // level-list nodes per child-plan block

// Tile records of level-list nodes [lo, hi) of list x, the first at tile
// offset `base0`; returns the offset after the last.  Per chunk of blockDim
// nodes one block scan gives every node's first tile, and the block's threads
// then take the chunk's tiles in turn, each finding its node by a binary
// search of those offsets, so a node cut into many tiles (the top levels) and
// many nodes of a few tiles each (the deep levels) keep every thread busy.
__device__ int block_plan_tiles_range(BuildArgs& a, int x, int lo, int hi, int base0)
{
    constexpr int kMaxThreads = 1024;
    __shared__ int sh[33];
    __shared__ int s_off[kMaxThreads], s_start[kMaxThreads], s_end[kMaxThreads];
    int base = base0;
    for (int c = lo; c < hi; c += blockDim.x) {
        const int ai = c + threadIdx.x;
        int nt = 0;
        if (ai < hi) {
            const Active nd = a.act[x][ai];
            nt = (nd.start + nd.count - 1) / kTile - nd.start / kTile + 1;
            s_start[threadIdx.x] = nd.start;
            s_end[threadIdx.x] = nd.start + nd.count;
        }
        int tot;
        const int excl = block_excl_scan(nt, sh, &tot);
        s_off[threadIdx.x] = excl;
        if (ai < hi) a.tile_base[x][ai] = base + excl;
        __syncthreads();
        const int nn = min((int)blockDim.x, hi - c);
        for (int q = threadIdx.x; q < tot; q += blockDim.x) {
            // the chunk's node holding tile q: the last r with s_off[r] <= q
            int r = 0;
#pragma unroll
            for (int step = kMaxThreads / 2; step >= 1; step >>= 1)
                if (r + step < nn && s_off[r + step] <= q) r += step;
            if (base + q >= a.tile_cap) {
                atomicOr(a.err, kErrTileOverflow);
                continue;
            }
            const int j = q - s_off[r];
            const int first = s_start[r] / kTile;
            Tile t;
            t.node = c + r;
            t.begin = max(s_start[r], (first + j) * kTile);
            t.end = min(s_end[r], (first + j + 1) * kTile);
            t.first = (j == 0);
            a.tiles[x][base + q] = t;
        }
        base += tot;
        __syncthreads();
    }
    return base;
}

// The whole tile plan of list x (one block): tile records, bases, counts.
__device__ void block_plan_tiles(BuildArgs& a, int x, int A)
{
    const int end = block_plan_tiles_range(a, x, 0, A, 0);
    if (threadIdx.x == 0) {
        a.tile_base[x][A] = end;
        a.cnt[kCntTiles0 + x] = min(end, a.tile_cap);
    }
}

// Roots: one tree (node 0) or, for a forest, node s for set s.  Roots with
// more than T points start the level stage; the others go straight to the
// subtree stage.
__global__ void k_init(BuildArgs a)
{
    griddep_enter();
    for (int c = threadIdx.x; c < a.chunk_cap; c += blockDim.x) {
        a.chunk_act[c] = 0;
        a.chunk_small[c] = 0;
    }
    __shared__ int sh[33];
    __shared__ int s_act, s_small;
    const int nsets = a.set_off ? a.nsets : 1;
    if (threadIdx.x == 0) {
        s_act = 0;
        s_small = 0;
    }
    __syncthreads();
    for (int c0 = 0; c0 < nsets; c0 += blockDim.x) {
        const int si = c0 + threadIdx.x;
        int start = 0, count = 0;
        if (si < nsets) {
            start = a.set_off ? a.set_off[si] : 0;
            count = a.set_off ? a.set_off[si + 1] - start : a.n;
        }
        const int act = (si < nsets && count > a.T) ? 1 : 0;
        const int sml = (si < nsets && !act) ? 1 : 0;
        int ta, ts;
        const int pa = block_excl_scan(act, sh, &ta) + s_act;
        const int ps = block_excl_scan(sml, sh, &ts) + s_small;
        if (act) {
            if (pa < a.act_cap) {
                Active r;
                r.start = start;
                r.count = count;
                r.node = si;
                r.depth = 0;
                a.act[0][pa] = r;
            } else {
                atomicOr(a.err, kErrActiveOverflow);
            }
        } else if (sml) {
            if (ps < a.small_cap) {
                Small sm;
                sm.start = start;
                sm.count = count;
                sm.node = si;
                sm.depth_parity = 0;
                a.small[ps] = sm;
            } else {
                atomicOr(a.err, kErrSmallOverflow);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_act += ta;
            s_small += ts;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.cnt[kCntActive0] = min(s_act, a.act_cap);
        a.cnt[kCntSmall] = s_small;
        a.cnt[kCntNodes] = nsets;
    }
    __syncthreads();
    block_plan_tiles(a, 0, min(s_act, a.act_cap));
}

// After a fixed number of level passes (graph-captured builds): nodes still
// active would have needed more passes; report it instead of building them.
__global__ void k_check_levels(BuildArgs a, int L)
{
    griddep_enter();
    if (threadIdx.x == 0 && a.cnt[kCntActive0 + (L & 1)] > 0) atomicOr(a.err, kErrLevels);
}

// ------------------------------------------------------------------ A2 + A3

// Histogram bin of x: #{v_j <= x} over the sorted interval points, found with
// a two-level search (every 32nd interval point first, then the 32 within).
__device__ __forceinline__ int hist_bin(const float* coarse, const float* fine, float x)
{
    int cb = count_le32(coarse, x);
    if (cb == 0) return 0;
    int blk = cb - 1;
    return blk * 32 + count_le32(fine + blk * 33, x);
}

// The first histogram pass of a node counts bins one by one only for the
// interval points of sample ranks kWinLo .. kWinHi, around the median rank
// 512 where c_j crosses n/2 (the sample's median rank of the node's median has
// a standard deviation of about 16; the window spans 8 of them each way), and
// only the count of points below v_kWinLo outside it.  For j in the window,
// c_j = #{x < v_kWinLo} + the window bins up to j, which is all the selection
// reads when 2 c_kWinLo <= n <= 2 c_kWinHi: every j below the window then has
// |2 c_j - n| >= |2 c_kWinLo - n| (equal only for v_j = v_kWinLo, so the
// same split value and count), and every j above it |2 c_j - n| >=
// |2 c_kWinHi - n|.  Otherwise the node takes the full histogram.
constexpr int kWinLo = 384, kWinHi = 640, kWin = kWinHi - kWinLo;
static_assert(kWin == 256 && kWinHi < kSamples, "count_le256 covers the window");

// #{a_i <= x} over 256 sorted values (binary search, branch-free).
__device__ __forceinline__ int count_le256(const float* a, float x)
{
    int c = 0;
#pragma unroll
    for (int s = 128; s >= 1; s >>= 1)
        if (a[c + s - 1] <= x) c += s;
    if (a[c] <= x) c++;
    return c;
}

constexpr int kSelectThreads = 256;   // selection blocks: 4 histogram bins per thread
static_assert(4 * kSelectThreads == kSamples, "the selection covers the sample bins with 4 per thread");
static_assert(kSamples == 1024, "sample positions use a shift by 10");

// Split selection from a node histogram (reading R3), by a block of
// kSelectThreads threads: thread t holds bins 4t .. 4t+3; c_j = #{x < v_j} is
// the inclusive prefix of the histogram up to bin j (one block scan of the
// thread sums) and j* = argmin |2 c_j - cnt| with ties to the smallest j (the
// minimum key |.| << 11 | j).  Every thread gets j* in *sel and c_{j*} in *left,
// and the prefixes c_kWinLo and c_kWinHi in *c_lo and *c_hi.
__device__ void block_select_split(const int* bins, int cnt, int sp, int* sel, int* left, int* c_lo, int* c_hi)
{
    __shared__ int shi[33];
    __shared__ unsigned long long s_key[kSelectThreads / 32];
    __shared__ int s_c[kSelectThreads / 32];
    __shared__ int s_sel, s_left, s_clo, s_chi;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int h[4], tot = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const int j = 4 * threadIdx.x + e;
        h[e] = j < sp ? bins[j] : 0;
        tot += h[e];
    }
    int total;
    int c = block_excl_scan(tot, shi, &total);
    unsigned long long best = ~0ull;
    int best_c = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const int j = 4 * threadIdx.x + e;
        c += h[e];
        if (j == kWinLo) s_clo = c;
        if (j == kWinHi) s_chi = c;
        long long err = 2LL * c - cnt;
        if (err < 0) err = -err;
        const unsigned long long key = ((unsigned long long)err << 11) | (unsigned)j;
        if (j < sp && key < best) {
            best = key;
            best_c = c;
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(kFull, best, o);
        const int oc = __shfl_xor_sync(kFull, best_c, o);
        if (ob < best) {
            best = ob;
            best_c = oc;
        }
    }
    if (lane == 0) {
        s_key[warp] = best;
        s_c[warp] = best_c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = s_key[0];
        int bc = s_c[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++)
            if (s_key[w] < b) {
                b = s_key[w];
                bc = s_c[w];
            }
        s_sel = (int)(b & 2047ull);
        s_left = bc;
    }
    __syncthreads();
    *sel = s_sel;
    *left = s_left;
    *c_lo = s_clo;
    *c_hi = s_chi;
    __syncthreads();
}

__device__ float block_reduce_min(float v, float* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_min(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float r = INFINITY;
    for (int w = 0; w < nw; w++) r = fminf(r, sh[w]);
    __syncthreads();
    return r;
}
__device__ float block_reduce_max(float v, float* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float r = -INFINITY;
    for (int w = 0; w < nw; w++) r = fmaxf(r, sh[w]);
    __syncthreads();
    return r;
}
__device__ int block_reduce_sum(int v, int* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int r = 0;
    for (int w = 0; w < nw; w++) r += sh[w];
    __syncthreads();
    return r;
}

constexpr int kSampleThreads = 256;   // k_sample's block (8 warps over 1024 samples)
constexpr int kSmallWarps = 8;        // k_sample_small: nodes per block, one per warp

// Split of a level-stage node whose points are all samples (n_node <= 1024,
// so S' = n_node), one warp per node.  R1's sample is then the node's own
// column runs, so R2's variances are taken over them in the order k_sample's
// samples would have (element j into partial j mod 32), and reading R3
// reduces to an exact selection: c(v) = #{x < v} grows with v, so the value
// minimising |2 c(v) - n| (ties to the smallest) is the value vp of rank
// floor(n/2) or the next larger value up -- no other value can do as well.  A
// radix selection over order-preserving keys (of x + 0: -0 and +0 are one
// value) finds vp, skipping the key bits every value shares; one pass counts
// na = #{x < vp}, nb = #{x <= vp} and finds up.  No sort, histogram pass or
// selection kernel runs for such a node (its mode becomes kModeSelected).
__global__ void __launch_bounds__(kSmallWarps * 32) k_sample_small(BuildArgs a, int L)
{
    griddep_enter();
    __shared__ float s_vals[kSmallWarps][kSamples];
    __shared__ int s_rh[kSmallWarps][256];
    __shared__ float s_var[kSmallWarps][kMaxDim];
    const int cur = L & 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ai = blockIdx.x * kSmallWarps + warp;
    if (ai >= a.cnt[kCntActive0 + cur]) return;
    const Active nd = a.act[cur][ai];
    const int cnt = nd.count;
    if (cnt > kSamples) return;   // a sampled node: k_sample
    const float* X = a.X[cur];
    float* var = s_var[warp];
    for (int k = 0; k < a.d; k++) {
        const float* col = X + (long long)k * a.n_pad + nd.start;
        float part = 0.0f;
        for (int j = lane; j < cnt; j += 32) part = __fadd_rn(part, col[j]);
        const float mean = __fdiv_rn(fixed_order_warp_total(part), (float)cnt);
        float p2 = 0.0f;
        for (int j = lane; j < cnt; j += 32) {
            const float c = __fsub_rn(col[j], mean);
            p2 = __fadd_rn(p2, __fmul_rn(c, c));
        }
        const float v = __fdiv_rn(fixed_order_warp_total(p2), (float)cnt);
        if (lane == 0) var[k] = v;
    }
    __syncwarp();
    const int dm = argmax_dims(var, a.d, 0u);
    if (lane == 0) {
        a.ndim[ai] = dm;
        for (int k = 0; k < a.d; k++) a.nvar[ai * kMaxDim + k] = var[k];
    }
    if (!(var[dm] > 0.0f)) {
        if (lane == 0) a.nmode[ai] = kModePending;   // constant along every dim: k_select's fallback
        return;
    }
    float* vals = s_vals[warp];
    int* rh = s_rh[warp];
    const float* col = X + (long long)dm * a.n_pad + nd.start;
    unsigned kmn = 0xffffffffu, kmx = 0u;
    for (int j = lane; j < cnt; j += 32) {
        const float x = col[j];
        vals[j] = x;
        const unsigned key = float_key(__fadd_rn(x, 0.0f));
        kmn = min(kmn, key);
        kmx = max(kmx, key);
    }
    kmn = __reduce_min_sync(kFull, kmn);
    kmx = __reduce_max_sync(kFull, kmx);
    __syncwarp();
    const int top = 32 - __clz(kmn ^ kmx);
    int rank = cnt >> 1;
    unsigned mask = (top >= 32) ? 0u : ~((1u << top) - 1u);
    unsigned prefix = kmn & mask;
    for (int hi = top; hi > 0; hi -= 8) {
        const int shift = hi >= 8 ? hi - 8 : 0;
        const int width = hi - shift;
        const unsigned dmask = (1u << width) - 1u;
        for (int b = lane; b < 256; b += 32) rh[b] = 0;
        __syncwarp();
#pragma unroll 4
        for (int j = lane; j < cnt; j += 32) {
            const unsigned key = float_key(__fadd_rn(vals[j], 0.0f));
            if ((key & mask) == prefix) atomicAdd(&rh[(key >> shift) & dmask], 1);
        }
        __syncwarp();
        // lane t holds digits 8t .. 8t+7; the digit holding `rank` and the count below it
        int loc = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) loc += rh[8 * lane + q];
        const int incl = warp_incl_scan(loc);
        const int excl = incl - loc;
        int found = -1, below = 0;
        if (rank >= excl && rank < incl) {
            int c = excl;
            for (int q = 0; q < 8; q++) {
                const int h = rh[8 * lane + q];
                if (rank < c + h) {
                    found = 8 * lane + q;
                    below = c;
                    break;
                }
                c += h;
            }
        }
        const int src = __ffs(__ballot_sync(kFull, found >= 0)) - 1;
        const int digit = __shfl_sync(kFull, found, src);
        below = __shfl_sync(kFull, below, src);
        prefix |= (unsigned)digit << shift;
        mask |= dmask << shift;
        rank -= below;
        __syncwarp();
    }
    const float vp = key_float(prefix);
    int na = 0, nb = 0;
    float up = INFINITY;
    for (int j = lane; j < cnt; j += 32) {
        const float x = vals[j];
        na += x < vp;
        nb += x <= vp;
        if (x > vp) up = fminf(up, x);
    }
    na = warp_sum(na);
    nb = warp_sum(nb);
    up = warp_min(up);
    long long e1 = 2LL * na - cnt;
    if (e1 < 0) e1 = -e1;
    float sv = vp;
    int cv = na;
    if (nb < cnt) {
        long long e2 = 2LL * nb - cnt;
        if (e2 < 0) e2 = -e2;
        if (e2 < e1) {
            sv = up;
            cv = nb;
        }
    }
    if (lane == 0) {
        if (cv > 0) {
            a.nsplit[ai] = sv;
            a.nleft[ai] = cv;
            a.nsel[ai] = -1;
            a.nmode[ai] = kModeSelected;
        } else {
            a.nmode[ai] = kModePending;   // heavy duplicates: k_select takes the fallback
        }
    }
}

// One block per active node of more than kSamples points: sample, per-dimension
// variance, split dimension, bitonic sort of the sample along it.

__global__ void __launch_bounds__(kSampleThreads) k_sample(BuildArgs a, int L)
{
    griddep_enter();
    extern __shared__ float S[];   // [d][kSamples]
    __shared__ float var[kMaxDim];
    __shared__ int sdim;
    const int cur = L & 1;
    const int ai = blockIdx.x;
    if (ai == 0 && threadIdx.x == 0) a.cnt[kCntRehist] = 0;   // the level's window misses
    if (ai >= a.cnt[kCntActive0 + cur]) return;
    const Active nd = a.act[cur][ai];
    const int cnt = nd.count;
    if (cnt <= kSamples) return;   // every point a sample: k_sample_small
    const int sp = kSamples;
    const float* X = a.X[cur];
    // sample j at floor(j * cnt / 1024); a thread's four samples of a dimension
    // are loaded before any is stored, so their (scattered) loads overlap
    static_assert(kSamples == 4 * kSampleThreads, "four samples per thread");
    long long pos[4];
#pragma unroll
    for (int r = 0; r < 4; r++) pos[r] = nd.start + (((long long)(threadIdx.x + r * kSampleThreads) * cnt) >> 10);
    for (int k = 0; k < a.d; k++) {
        const float* col = X + (long long)k * a.n_pad;
        float x[4];
#pragma unroll
        for (int r = 0; r < 4; r++) x[r] = col[pos[r]];
#pragma unroll
        for (int r = 0; r < 4; r++) S[k * kSamples + threadIdx.x + r * kSampleThreads] = x[r];
    }
    {
        int* nh = a.nhist + (long long)ai * (kSamples + 1);
        for (int b = threadIdx.x; b <= kSamples; b += blockDim.x) nh[b] = 0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < a.d; k += nw) {
        const float* col = S + k * kSamples;
        float part = 0.0f;
        for (int j = lane; j < sp; j += 32) part = __fadd_rn(part, col[j]);
        float mean = __fdiv_rn(fixed_order_warp_total(part), (float)sp);
        float p2 = 0.0f;
        for (int j = lane; j < sp; j += 32) {
            float c = __fsub_rn(col[j], mean);
            p2 = __fadd_rn(p2, __fmul_rn(c, c));
        }
        float v = __fdiv_rn(fixed_order_warp_total(p2), (float)sp);
        if (lane == 0) var[k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int dm = argmax_dims(var, a.d, 0u);
        sdim = dm;
        a.ndim[ai] = dm;
        a.nmode[ai] = (var[dm] > 0.0f) ? kModeValue : kModePending;
        for (int k = 0; k < a.d; k++) a.nvar[ai * kMaxDim + k] = var[k];
    }
    __syncthreads();
    const int dm = sdim;
    if (!(var[dm] > 0.0f)) return;
    // Sort of the 1024 samples along dm.  First each warp sorts its own 128
    // (bitonic network; warp w takes the compare-exchange pairs kPairsPerWarp * w
    // onwards, which touch only its 128 elements, so warp barriers suffice) and
    // leaves them ascending; then three rounds of merge-path merges (runs of
    // 128 -> 256 -> 512 -> 1024) between the sample row and a second row: each
    // thread finds where its 4 outputs start by a binary search of the
    // diagonal and merges them.
    constexpr int kPairsPerWarp = kSamples / 2 / (kSampleThreads / 32);
    constexpr int kRun = 2 * kPairsPerWarp;   // 128
    float* v = S + dm * kSamples;
    for (int size = 2; size <= kRun; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
            for (int r = 0; r < kPairsPerWarp / 32; r++) {
                const int t = warp * kPairsPerWarp + 32 * r + lane;
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = size == kRun || (i & size) == 0;
                const float x = v[i], y = v[j];
                if ((x > y) == up) {
                    v[i] = y;
                    v[j] = x;
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    float* src = v;
    float* dst = S + (a.d > 1 ? ((dm + 1) % a.d) : 1) * kSamples;   // a row no longer needed
    for (int len = kRun; len < kSamples; len <<= 1) {
        const int tpm = len / 2;                           // threads per merge: 4 outputs each
        const int mi = threadIdx.x / tpm;
        const int p = (threadIdx.x % tpm) * 4;
        const float* A = src + mi * 2 * len;
        const float* B = A + len;
        // the diagonal's split: i outputs from A, p - i from B (A first on ties)
        int lo = max(0, p - len), hi = min(p, len);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[p - mid - 1]) lo = mid + 1;
            else hi = mid;
        }
        int i = lo, j = p - lo;
        float* o = dst + mi * 2 * len + p;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const bool takeA = j >= len || (i < len && A[i] <= B[j]);
            o[e] = takeA ? A[i] : B[j];
            i += takeA;
            j += !takeA;
        }
        __syncthreads();
        float* tmp = src;
        src = dst;
        dst = tmp;
    }
    v = src;
    float* out = a.vs + (long long)ai * kSamples;
    for (int j = threadIdx.x; j < kSamples; j += blockDim.x) out[j] = v[j];
}

// ------------------------------------------------------------------ A4

// Window histogram of every tile of a value-split node (blocks stride over
// the tiles: levels whose nodes were selected exactly in k_sample have nothing
// to do here).  A point below v_kWinLo adds to bin kWinLo (c_kWinLo is then
// exact), one in [v_kWinLo, v_kWinHi) to its own bin #{v_j <= x} (a search of
// the 256 window points), and one at or above v_kWinHi to nothing.
__global__ void k_hist(BuildArgs a, int L)
{
    griddep_enter();
    __shared__ float win[kWin];
    __shared__ int hist[kWin];
    __shared__ int sh[33];
    __shared__ float queue[256 / 32][64];   // a warp's window values waiting for their search
    const int cur = L & 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* qw = queue[warp];
    const int ntiles = a.cnt[kCntTiles0 + cur];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = a.tiles[cur][t];
        const int ai = tl.node;
        if (a.nmode[ai] != kModeValue) continue;
        const int dm = a.ndim[ai];
        const float* vs = a.vs + (long long)ai * kSamples;
        for (int j = threadIdx.x; j < kWin; j += blockDim.x) {
            win[j] = vs[kWinLo + j];
            hist[j] = 0;
        }
        const float vlo = vs[kWinLo], vhi = vs[kWinHi];
        __syncthreads();
        const float* col = a.X[cur] + (long long)dm * a.n_pad;
        int below = 0;
        // Values in the window are queued per warp and searched 32 at a time,
        // so every lane of a search has a value (about a quarter of them fall
        // in the window).  The trip count is warp-uniform.
        int qn = 0;
        for (int w0 = (tl.begin & ~3) + 4 * (threadIdx.x & ~31); w0 < tl.end; w0 += 4 * blockDim.x) {
            const int i4 = w0 + 4 * lane;
            float4 x4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (i4 < tl.end) x4 = *reinterpret_cast<const float4*>(col + i4);
            const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int i = i4 + e;
                const bool in = i >= tl.begin && i < tl.end;
                const float x = xs[e];
                below += in && x < vlo;
                const bool w = in && x >= vlo && x < vhi;
                const unsigned m = __ballot_sync(kFull, w);
                if (w) qw[qn + __popc(m & lanemask_lt())] = x;
                qn += __popc(m);
                if (qn >= 32) {
                    __syncwarp();
                    const float y = qw[lane];
                    const float rest = lane + 32 < qn ? qw[lane + 32] : 0.0f;
                    __syncwarp();
                    if (lane + 32 < qn) qw[lane] = rest;
                    qn -= 32;
                    atomicAdd(&hist[count_le256(win, y) - 1], 1);
                }
            }
        }
        __syncwarp();
        if (lane < qn) atomicAdd(&hist[count_le256(win, qw[lane]) - 1], 1);
        below = block_reduce_sum(below, sh);
        int* nh = a.nhist + (long long)ai * (kSamples + 1);
        int* tb = a.tbins + (long long)t * (1 + kWin);   // this tile's own counts (k_tilecount)
        if (threadIdx.x == 0) {
            if (below) atomicAdd(&nh[kWinLo], below);
            tb[0] = below;
        }
        for (int b = threadIdx.x; b < kWin; b += blockDim.x) {
            const int h = hist[b];
            if (h) atomicAdd(&nh[kWinLo + 1 + b], h);
            tb[1 + b] = h;
        }
        __syncthreads();
    }
}

// Full histogram of every tile of a node the window missed, over all its
// interval points (a two-level search: every 32nd interval point, then the 32
// within); the launch returns at once when no node was missed.
__global__ void k_hist_full(BuildArgs a, int L)
{
    griddep_enter();
    if (a.cnt[kCntRehist] == 0) return;
    __shared__ float fine[32 * 33];
    __shared__ float coarse[32];
    __shared__ int hist[kSamples + 1];
    const int cur = L & 1;
    const int ntiles = a.cnt[kCntTiles0 + cur];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = a.tiles[cur][t];
        const int ai = tl.node;
        if (a.nmode[ai] != kModeRehist) continue;
        const int dm = a.ndim[ai];
        const float* vs = a.vs + (long long)ai * kSamples;
        for (int j = threadIdx.x; j < kSamples; j += blockDim.x) {
            float v = vs[j];
            fine[(j >> 5) * 33 + (j & 31)] = v;
            if ((j & 31) == 0) coarse[j >> 5] = v;
        }
        for (int b = threadIdx.x; b <= kSamples; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const float* col = a.X[cur] + (long long)dm * a.n_pad;
        for (int i4 = (tl.begin & ~3) + 4 * threadIdx.x; i4 < tl.end; i4 += 4 * blockDim.x) {
            float4 x4 = *reinterpret_cast<const float4*>(col + i4);
            float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                int i = i4 + e;
                if (i >= tl.begin && i < tl.end) atomicAdd(&hist[hist_bin(coarse, fine, xs[e])], 1);
            }
        }
        __syncthreads();
        int* nh = a.nhist + (long long)ai * (kSamples + 1);
        for (int b = threadIdx.x; b <= kSamples; b += blockDim.x) {
            int h = hist[b];
            if (h) atomicAdd(&nh[b], h);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ A5 (split select)


// FULL = false: the split from the window histogram (a node whose crossing
// lies outside the window is marked kModeRehist, its histogram cleared for the
// full pass).  FULL = true: the split of a kModeRehist node from the full one.
template <bool FULL>
__device__ void select_node(BuildArgs& a, int cur, int ai)
{
    __shared__ float shf[32];
    __shared__ int shi[33];
    const Active nd = a.act[cur][ai];
    const int cnt = nd.count;
    const int sp = cnt < kSamples ? cnt : kSamples;
    int mode = a.nmode[ai];
    // k_sample selected the split exactly.  The mode stays kModeSelected (the
    // later kernels tell only index splits apart): a write here would race with
    // the block's other warps still reading it.
    if (mode == kModeSelected) return;
    if (mode == (FULL ? kModeRehist : kModeValue)) {
        int sel, left, c_lo, c_hi;
        int* nh = a.nhist + (long long)ai * (kSamples + 1);
        block_select_split(nh, cnt, sp, &sel, &left, &c_lo, &c_hi);
        if (!FULL && (2LL * c_lo > cnt || 2LL * c_hi < cnt)) {
            for (int b = threadIdx.x; b <= kSamples; b += blockDim.x) nh[b] = 0;
            if (threadIdx.x == 0) {
                a.nmode[ai] = kModeRehist;
                atomicAdd(&a.cnt[kCntRehist], 1);
            }
            return;
        }
        if (left > 0) {
            if (threadIdx.x == 0) {
                a.nsplit[ai] = a.vs[(long long)ai * kSamples + sel];
                a.nleft[ai] = left;
                a.nsel[ai] = FULL ? -1 : sel;   // >= 0: decided from the window bins
                if (FULL) a.nmode[ai] = kModeValue;
            }
            return;
        }
        mode = kModePending;
    }
    // Duplicate fallback: first non-constant dim in descending-variance order,
    // split just above its minimum; index split if every dim is constant.
    const float* X = a.X[cur];
    const float* var = a.nvar + ai * kMaxDim;
    unsigned used = 0;
    int fdim = -1;
    float fsplit = 0.0f, min0 = 0.0f;
    for (int r = 0; r < a.d; r++) {
        int k = argmax_dims(var, a.d, used);
        used |= 1u << k;
        const float* col = X + (long long)k * a.n_pad + nd.start;
        float mn = INFINITY, mx = -INFINITY;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            float x = col[i];
            mn = fminf(mn, x);
            mx = fmaxf(mx, x);
        }
        mn = block_reduce_min(mn, shf);
        mx = block_reduce_max(mx, shf);
        if (k == 0) min0 = mn;
        if (mx > mn) {
            float nxt = INFINITY;
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                float x = col[i];
                if (x > mn) nxt = fminf(nxt, x);
            }
            fsplit = block_reduce_min(nxt, shf);
            fdim = k;
            break;
        }
    }
    int left;
    if (fdim >= 0) {
        const float* col = X + (long long)fdim * a.n_pad + nd.start;
        int c = 0;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) c += col[i] < fsplit;
        left = block_reduce_sum(c, shi);
        mode = kModeValue;
    } else {
        // every dim constant (all were visited): min0 is dim 0's value
        left = (cnt + 1) >> 1;
        mode = kModeIndex;
        fdim = 0;
        fsplit = min0;
    }
    if (threadIdx.x == 0) {
        a.nmode[ai] = mode;
        a.ndim[ai] = fdim;
        a.nsplit[ai] = fsplit;
        a.nleft[ai] = left;
        a.nsel[ai] = -1;
    }
}

// Split selection of every node of the level (blocks stride over the nodes).
__global__ void __launch_bounds__(kSelectThreads) k_select(BuildArgs a, int L)
{
    griddep_enter();
    const int cur = L & 1;
    const int A = a.cnt[kCntActive0 + cur];
    for (int ai = blockIdx.x; ai < A; ai += gridDim.x) {
        if (a.nmode[ai] == kModeSelected) continue;   // split in k_sample; no shared memory touched
        select_node<false>(a, cur, ai);
        __syncthreads();
    }
}

// Selection of the nodes the window missed, from their full histograms.
__global__ void __launch_bounds__(kSelectThreads) k_select_full(BuildArgs a, int L)
{
    griddep_enter();
    if (a.cnt[kCntRehist] == 0) return;
    const int cur = L & 1;
    const int A = a.cnt[kCntActive0 + cur];
    for (int ai = blockIdx.x; ai < A; ai += gridDim.x) {
        if (a.nmode[ai] != kModeRehist) continue;
        select_node<true>(a, cur, ai);
        __syncthreads();
    }
}

// Per-tile count of left points for nodes that span several tiles.
// Left count of every tile: one block per tile (grid-stride over the tiles),
// so a level of large nodes keeps many column loads in flight per SM.
__global__ void k_tilecount(BuildArgs a, int L)
{
    griddep_enter();
    __shared__ int sh[33];
    const int cur = L & 1;
    const int ntl = a.cnt[kCntTiles0 + cur];
    for (int t = blockIdx.x; t < ntl; t += gridDim.x) {
        const Tile tl = a.tiles[cur][t];
        const int ai = tl.node;
        const Active nd = a.act[cur][ai];
        const int ntiles = a.tile_base[cur][ai + 1] - a.tile_base[cur][ai];
        if (ntiles == 1) {
            if (threadIdx.x == 0) a.tleft[t] = a.nleft[ai];
            continue;
        }
        if (a.nmode[ai] == kModeIndex) {
            const int half = (nd.count + 1) >> 1;
            if (threadIdx.x == 0) a.tleft[t] = min(max(half - (tl.begin - nd.start), 0), tl.end - tl.begin);
            continue;
        }
        const int sel = a.nsel[ai];
        if (sel >= kWinLo && sel <= kWinHi) {
            // split v_sel from the window: the tile's x < v_sel are its points below
            // v_kWinLo plus those in window bins kWinLo + 1 .. sel
            const int* tb = a.tbins + (long long)t * (1 + kWin);
            int c = (threadIdx.x < sel - kWinLo) ? tb[1 + threadIdx.x] : 0;
            const int v = block_reduce_sum(c, sh);
            if (threadIdx.x == 0) a.tleft[t] = tb[0] + v;
            continue;
        }
        const float s = a.nsplit[ai];
        const float* col = a.X[cur] + (long long)a.ndim[ai] * a.n_pad;
        int c = 0;
        // four float4 loads in flight per thread before any is used
        const int step = 4 * blockDim.x;
        for (int i0 = (tl.begin & ~3) + 4 * threadIdx.x; i0 < tl.end; i0 += 4 * step) {
            float4 x4[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int p = i0 + u * step;
                x4[u] = p < tl.end ? *reinterpret_cast<const float4*>(col + p) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int p = i0 + u * step;
                c += (p >= tl.begin && p < tl.end && x4[u].x < s);
                c += (p + 1 >= tl.begin && p + 1 < tl.end && x4[u].y < s);
                c += (p + 2 >= tl.begin && p + 2 < tl.end && x4[u].z < s);
                c += (p + 3 >= tl.begin && p + 3 < tl.end && x4[u].w < s);
            }
        }
        const int v = block_reduce_sum(c, sh);
        if (threadIdx.x == 0) a.tleft[t] = v;
    }
}

// Left-count offsets of every node's tiles (exclusive scan of the per-tile
// left counts within the node), one warp per node over the whole grid.
__global__ void k_tileoff(BuildArgs a, int L)
{
    griddep_enter();
    __shared__ int s_act, s_small;
    const int cur = L & 1;
    const int A = a.cnt[kCntActive0 + cur];
    const int lane = threadIdx.x & 31;
    // the next level's tile sums (k_children adds, k_plan reads) start at zero
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < a.chunk_cap; c += blockDim.x) a.chunk_tiles[c] = 0;
    if (threadIdx.x == 0) {
        s_act = 0;
        s_small = 0;
    }
    __syncthreads();
    const int ai = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (ai < A) {
        if (lane == 0) {
            // children of node ai: to the next level (more than T points) or the subtree stage
            const int cl = a.nleft[ai], cr = a.act[cur][ai].count - cl;
            const int act = (cl > a.T) + (cr > a.T);
            atomicAdd(&s_act, act);
            atomicAdd(&s_small, 2 - act);
        }
        const int tb = min(a.tile_base[cur][ai], a.tile_cap);
        const int te = min(a.tile_base[cur][ai + 1], a.tile_cap);
        int running = 0;
        for (int j0 = tb; j0 < te; j0 += 32) {
            int j = j0 + lane;
            int v = j < te ? a.tleft[j] : 0;
            int incl = warp_incl_scan(v);
            if (j < te) a.tleftoff[j] = running + incl - v;
            running += __shfl_sync(kFull, incl, 31);
        }
        if (lane == 0 && running != a.nleft[ai]) atomicOr(a.err, kErrInternal);
    }
    __syncthreads();
    // this block's nodes lie in one chunk (blockDim / 32 divides kChildChunk)
    const int first = blockIdx.x * (blockDim.x >> 5);
    if (threadIdx.x == 0 && first < A) {
        const int c = first / kChildChunk;
        if (s_act) atomicAdd(&a.chunk_act[c], s_act);
        if (s_small) atomicAdd(&a.chunk_small[c], s_small);
    }
}

// Children of the level's nodes (next level or subtree stage), node headers of
// this level: one block per chunk of kChildChunk level-list nodes.  A block's
// first list positions are the sums of the chunks before it (from k_tileoff),
// so the lists come out in node order without any block waiting for another.
// Each block also adds the tile counts of the next-level nodes it creates to
// the chunk sums k_plan needs.  Counters are updated by k_plan.
__global__ void k_children(BuildArgs a, int L)
{
    griddep_enter();
    __shared__ int sh[33];
    __shared__ int s_tiles[3];
    const int cur = L & 1, nxt = cur ^ 1;
    const int A = a.cnt[kCntActive0 + cur];
    const int c = blockIdx.x;
    const int lo = c * kChildChunk;
    if (lo >= A) return;
    const int hi = min(A, lo + kChildChunk);
    const int base_id = a.cnt[kCntNodes];
    int act_base = 0, small_base = a.cnt[kCntSmall];
    for (int p = 0; p < c; p++) {
        act_base += a.chunk_act[p];
        small_base += a.chunk_small[p];
    }
    const int first_chunk = act_base / kChildChunk;
    if (threadIdx.x < 3) s_tiles[threadIdx.x] = 0;
    // thread t plans nodes a0 .. a0 + kPlanPer - 1 of the chunk: one block scan
    // of (children to the next level << 16 | children to the subtree stage)
    static_assert(2 * kChildChunk < (1 << 16), "packed child counts");
    const int a0 = lo + threadIdx.x * kPlanPer;
    int nxt_cnt = 0, sm_cnt = 0;
#pragma unroll
    for (int r = 0; r < kPlanPer; r++) {
        if (a0 + r < hi) {
            const int cl = a.nleft[a0 + r], cr = a.act[cur][a0 + r].count - cl;
            const int act = (cl > a.T) + (cr > a.T);
            nxt_cnt += act;
            sm_cnt += 2 - act;
        }
    }
    int tot;
    const int pk = block_excl_scan((nxt_cnt << 16) | sm_cnt, sh, &tot);
    int ia = act_base + (pk >> 16), is = small_base + (pk & 0xffff);
    for (int r = 0; r < kPlanPer; r++) {
        const int ai = a0 + r;
        if (ai >= hi) break;
        const Active nd = a.act[cur][ai];
        const int cl = a.nleft[ai], cr = nd.count - cl;
        const int child = base_id + 2 * ai;
        const int cdepth = nd.depth + 1;
        for (int side = 0; side < 2; side++) {
            const int cs = side ? nd.start + cl : nd.start;
            const int cc = side ? cr : cl;
            if (cc > a.T) {
                if (cdepth >= kMaxDepth) atomicOr(a.err, kErrDepth);
                if (ia < a.act_cap) {
                    Active ch;
                    ch.start = cs;
                    ch.count = cc;
                    ch.node = child + side;
                    ch.depth = cdepth;
                    a.act[nxt][ia] = ch;
                    const int nt = (cs + cc - 1) / kTile - cs / kTile + 1;
                    const int slot = ia / kChildChunk - first_chunk;   // 0..2: a block's children span <= 3 chunks
                    if (slot >= 0 && slot < 3) atomicAdd(&s_tiles[slot], nt);
                    else atomicOr(a.err, kErrInternal);
                } else {
                    atomicOr(a.err, kErrActiveOverflow);
                }
                ia++;
            } else {
                if (is < a.small_cap) {
                    Small sm;
                    sm.start = cs;
                    sm.count = cc;
                    sm.node = child + side;
                    sm.depth_parity = (cdepth << 1) | nxt;
                    a.small[is] = sm;
                } else {
                    atomicOr(a.err, kErrSmallOverflow);
                }
                is++;
            }
        }
        const int mode = a.nmode[ai];
        if (nd.node < a.node_cap) {
            unsigned meta = (unsigned)a.ndim[ai] | (mode == kModeIndex ? kMetaIndex : 0u);
            int4 h = make_int4(child, nd.start + cl, __float_as_int(a.nsplit[ai]), (int)meta);
            reinterpret_cast<int4*>(a.nodes)[(long long)nd.node * a.ns] = h;
        }
        a.lvl_nodes[L * a.lvl_stride + ai] = nd.node;
    }
    __syncthreads();
    if (threadIdx.x < 3 && s_tiles[threadIdx.x] > 0 && first_chunk + (int)threadIdx.x < a.chunk_cap)
        atomicAdd(&a.chunk_tiles[first_chunk + threadIdx.x], s_tiles[threadIdx.x]);
}

// Tile plan of the next level, one block per chunk of kChildChunk next-level
// nodes (tile offsets from the chunk sums of k_children); block 0 also updates
// the level counters and the last tile base.  (The child sums are read by
// every block here; k_partition clears them for the next level.)
__global__ void k_plan(BuildArgs a, int L)
{
    griddep_enter();
    const int cur = L & 1, nxt = cur ^ 1;
    const int A = a.cnt[kCntActive0 + cur];
    int an = 0, as = 0, at = 0;
    const int nchunks = min((A + kChildChunk - 1) / kChildChunk, a.chunk_cap);
    for (int p = 0; p < nchunks; p++) {
        an += a.chunk_act[p];
        as += a.chunk_small[p];
    }
    const int An = min(an, a.act_cap);
    const int c = blockIdx.x;
    const int lo = c * kChildChunk;
    int tile_base0 = 0;
    const int nxt_chunks = min((An + kChildChunk - 1) / kChildChunk, a.chunk_cap);
    for (int p = 0; p < c && p < nxt_chunks; p++) tile_base0 += a.chunk_tiles[p];
    for (int p = 0; p < nxt_chunks; p++) at += a.chunk_tiles[p];
    if (lo < An) block_plan_tiles_range(a, nxt, lo, min(An, lo + kChildChunk), tile_base0);
    if (c == 0) {
        if (threadIdx.x == 0) {
            a.tile_base[nxt][An] = at;
            a.cnt[kCntTiles0 + nxt] = min(at, a.tile_cap);
            const int base_id = a.cnt[kCntNodes];
            a.cnt[kCntNodes] = base_id + 2 * A;
            if (base_id + 2 * A > a.node_cap) atomicOr(a.err, kErrNodeOverflow);
            a.cnt[kCntActive0 + nxt] = An;
            if (an > a.act_cap) atomicOr(a.err, kErrActiveOverflow);
            a.cnt[kCntSmall] += as;
            a.lvl_count[L] = A;
            if (A > 0) a.cnt[kCntLevels] = L + 1;
        }
    }
}

// Stable partition of every tile: left (x[dim] < s, or the first half for an
// index split) then right, scattered into the other ping-pong buffer.  Offsets
// come from a warp-ballot / shuffle prefix scan within the block and from the
// per-tile left counts across blocks.
__global__ void k_partition(BuildArgs a, int L)
{
    griddep_enter();
    __shared__ int sh[33];
    const int cur = L & 1, nxt = cur ^ 1;
    const int t = blockIdx.x;
    if (t == 0)   // the next level's child sums (k_tileoff adds, k_children and k_plan read)
        for (int c = threadIdx.x; c < a.chunk_cap; c += blockDim.x) {
            a.chunk_act[c] = 0;
            a.chunk_small[c] = 0;
        }
    if (t >= a.cnt[kCntTiles0 + cur]) return;
    const Tile tl = a.tiles[cur][t];
    const int ai = tl.node;
    const Active nd = a.act[cur][ai];
    const int mode = a.nmode[ai];
    const int dim = a.ndim[ai];
    const float s = a.nsplit[ai];
    const int nleft = a.nleft[ai];
    const int loff = a.tleftoff[t];
    int lpos = nd.start + loff;
    int rpos = nd.start + nleft + (tl.begin - nd.start - loff);
    const int half = (nd.count + 1) >> 1;
    const float* Xs = a.X[cur];
    float* Xd = a.X[nxt];
    const int* Is = a.ID[cur];
    int* Id = a.ID[nxt];
    const long long np = a.n_pad;
    for (int c0 = tl.begin & ~3; c0 < tl.end; c0 += 4 * blockDim.x) {
        const int i4 = c0 + 4 * threadIdx.x;
        const bool in = i4 < tl.end;
        bool valid[4], left[4];
        float key[4] = {0.f, 0.f, 0.f, 0.f};
        float4 kx4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in) {
            kx4 = *reinterpret_cast<const float4*>(Xs + dim * np + i4);
            key[0] = kx4.x;
            key[1] = kx4.y;
            key[2] = kx4.z;
            key[3] = kx4.w;
        }
        int nl = 0, nv = 0;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            int i = i4 + e;
            valid[e] = in && i >= tl.begin && i < tl.end;
            left[e] = valid[e] && (mode == kModeIndex ? (i - nd.start < half) : (key[e] < s));
            nl += left[e];
            nv += valid[e];
        }
        int tot;
        int packed = block_excl_scan(nl | ((nv - nl) << 16), sh, &tot);
        int pl = lpos + (packed & 0xffff), pr = rpos + (packed >> 16);
        int dst[4];
        bool bad = false;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            dst[e] = left[e] ? pl : pr;
            pl += left[e];
            pr += valid[e] && !left[e];
            // a destination outside the node would mean inconsistent counts: never write it
            if (valid[e] && (dst[e] < nd.start || dst[e] >= nd.start + nd.count)) {
                valid[e] = false;
                bad = true;
            }
        }
        if (bad) atomicOr(a.err, kErrInternal);
        if (in) {
            for (int k = 0; k < a.d; k++) {
                const float4 v = k == dim ? kx4 : *reinterpret_cast<const float4*>(Xs + k * np + i4);
                float* o = Xd + k * np;
                if (valid[0]) o[dst[0]] = v.x;
                if (valid[1]) o[dst[1]] = v.y;
                if (valid[2]) o[dst[2]] = v.z;
                if (valid[3]) o[dst[3]] = v.w;
            }
            int4 id = *reinterpret_cast<const int4*>(Is + i4);
            if (valid[0]) Id[dst[0]] = id.x;
            if (valid[1]) Id[dst[1]] = id.y;
            if (valid[2]) Id[dst[2]] = id.z;
            if (valid[3]) Id[dst[3]] = id.w;
        }
        lpos += tot & 0xffff;
        rpos += tot >> 16;
    }
}

// ------------------------------------------------------------------ A6 + A7

struct WarpMem {
    float* sx;            // [d][TS] coordinates (TS = T + 4: room for the 16-byte alignment offset)
    unsigned short* ix[2];  // [T] local indices, ping-pong
    int* rh;              // [256] radix histogram
    float* box;           // [2][kMaxDim] lo, hi
    float* var;           // [kMaxDim]
    int4* stk;            // [kMaxDepth + 4]
};

__host__ __device__ __forceinline__ size_t warp_bytes(int d, int T)
{
    const size_t TS = (size_t)T + 4;
    size_t b = 4 * d * TS + 2 * 2 * (size_t)T + 256 * 4 + 3 * kMaxDim * 4;
    b = (b + 15) & ~(size_t)15;
    return b + (kMaxDepth + 4) * sizeof(int4);
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Write node `node`'s record: header + box (lo, hi over dp slots, zero padded).
__device__ void write_node(const BuildArgs& a, int node, int4 hdr, const float* box)
{
    const int lane = threadIdx.x & 31;
    if (node >= a.node_cap) return;
    float4* rec = a.nodes + (long long)node * a.ns;
    if (lane == 0) {
        reinterpret_cast<int4*>(rec)[0] = hdr;
    } else if (lane < a.ns) {
        float f[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int slot = 4 * lane + q - 4;   // 0..2dp-1 box slots
            float v = 0.0f;
            if (slot < a.dp) {
                if (slot < a.d) v = box[slot];
            } else if (slot < 2 * a.dp) {
                int k = slot - a.dp;
                if (k < a.d) v = box[kMaxDim + k];
            }
            f[q] = v;
        }
        rec[lane] = make_float4(f[0], f[1], f[2], f[3]);
    }
}

// Node ids come in pairs (children a, a+1) from a per-warp pool refilled from
// the global counter 64 ids at a time; ids left in a pool are holes in the
// node table that nothing references.
constexpr int kIdChunk = 64;
constexpr int kSubtreeMaxWarps = 32;   // warps of the one k_subtree block per SM

__global__ void k_subtree(BuildArgs a, int wbytes)
{
    griddep_enter();
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int T = a.T, d = a.d, TS = a.T + 4;
    unsigned char* base = smem + (size_t)warp * wbytes;
    WarpMem w;
    w.sx = reinterpret_cast<float*>(base);
    w.ix[0] = reinterpret_cast<unsigned short*>(w.sx + (size_t)d * TS);
    w.ix[1] = w.ix[0] + T;
    w.rh = reinterpret_cast<int*>(w.ix[1] + T);
    w.box = reinterpret_cast<float*>(w.rh + 256);
    w.var = w.box + 2 * kMaxDim;
    {
        size_t off = (size_t)((unsigned char*)(w.var + kMaxDim) - base);
        off = (off + 15) & ~(size_t)15;
        w.stk = reinterpret_cast<int4*>(base + off);
    }
    const int nsmall = min(a.cnt[kCntSmall], a.small_cap);
    int pool_next = 0, pool_end = 0;          // per-warp id pool (warp-uniform)
    int my_nodes = 0, my_leaves = 0, my_depth = 0;
    for (;;) {
        int si = 0;
        if (lane == 0) si = atomicAdd(&a.cnt[kCntSmallNext], 1);
        si = __shfl_sync(kFull, si, 0);
        if (si >= nsmall) break;
        const Small sn = a.small[si];
        const int start = sn.start, count = sn.count, par = sn.depth_parity & 1;
        if (count < 1 || count > T || start < 0 || start + count > a.n) {
            if (lane == 0) atomicOr(a.err, kErrInternal);
            continue;
        }
        // stage the node: 16-byte asynchronous copies of the aligned superset of
        // each column; element i of the node sits at offset off + i
        const int off = start & 3;
        const int g0 = start - off;
        const int nch = (off + count + 3) >> 2;
        {
            const float* Xs = a.X[par];
            for (int k = 0; k < d; k++) {
                const float* src = Xs + (long long)k * a.n_pad + g0;
                float* dst = w.sx + (size_t)k * TS;
                for (int c = lane; c < nch; c += 32) cp_async16(dst + 4 * c, src + 4 * c);
            }
            for (int i = lane; i < count; i += 32) w.ix[0][i] = (unsigned short)i;
            cp_async_wait_all();
        }
        const float* sxo = w.sx + off;
        // ids stay in global memory (read once, when a leaf is written): the
        // shared memory they would take is another warp's worth at d = 3
        const int* gid = a.ID[par] + start;
        int sp = 0;
        if (lane == 0) w.stk[0] = make_int4(0, count, sn.node, sn.depth_parity >> 1);
        sp = 1;
        __syncwarp();
        while (sp > 0) {
            const int4 e = w.stk[--sp];
            __syncwarp();
            const int ls = e.x, lc = e.y, node = e.z;
            const int depth = e.w & 0xffff, rel = e.w >> 16;
            const unsigned short* ixc = w.ix[rel & 1];
            unsigned short* ixn = w.ix[(rel + 1) & 1];
            const bool leaf = lc <= a.bucket || depth >= kMaxDepth;
            // box (and, for inner nodes, the sample variance: every point is a sample).
            // The point loops below are unrolled so that each lane has several
            // independent index and coordinate loads in flight (a lane's sums keep
            // their order): the stage is latency bound at 12 warps per SM.
            for (int k = 0; k < d; k++) {
                const float* col = sxo + (size_t)k * TS;
                float part = 0.0f, mn = INFINITY, mx = -INFINITY;
#pragma unroll 4
                for (int j = lane; j < lc; j += 32) {
                    float x = col[ixc[ls + j]];
                    part = __fadd_rn(part, x);
                    mn = fminf(mn, x);
                    mx = fmaxf(mx, x);
                }
                mn = warp_min(mn);
                mx = warp_max(mx);
                float vk = 0.0f;
                if (!leaf) {
                    float mean = __fdiv_rn(fixed_order_warp_total(part), (float)lc);
                    float p2 = 0.0f;
#pragma unroll 4
                    for (int j = lane; j < lc; j += 32) {
                        float c = __fsub_rn(col[ixc[ls + j]], mean);
                        p2 = __fadd_rn(p2, __fmul_rn(c, c));
                    }
                    vk = __fdiv_rn(fixed_order_warp_total(p2), (float)lc);
                }
                if (lane == 0) {
                    w.box[k] = mn;
                    w.box[kMaxDim + k] = mx;
                    w.var[k] = vk;
                }
            }
            __syncwarp();
            if (leaf) {
                if (lc > a.bucket && lane == 0) atomicOr(a.err, kErrDepth);
                const int pstart = start + ls;
                write_node(a, node, make_int4(pstart, lc, 0, (int)kMetaLeaf), w.box);
                for (int i = lane; i < lc; i += 32) {
                    const int p = ixc[ls + i];
                    float4* o = a.pts + (long long)(pstart + i) * a.nv;
                    for (int v4 = 0; v4 < a.nv; v4++) {
                        float f[4];
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            int slot = 4 * v4 + q;
                            float val = 0.0f;
                            if (slot < d) val = sxo[(size_t)slot * TS + p];
                            else if (slot == a.dp) val = __int_as_float(__ldg(gid + p));
                            f[q] = val;
                        }
                        o[v4] = make_float4(f[0], f[1], f[2], f[3]);
                    }
                }
                my_nodes++;
                my_leaves++;
                my_depth = max(my_depth, depth);
                __syncwarp();
                continue;
            }
            // ---- split rule (S' = lc: exact selection form of the sampled rule)
            int dim = argmax_dims(w.var, d, 0u);
            int mode = -1, cleft = 0;
            float s = 0.0f;
            if (w.var[dim] > 0.0f && w.box[kMaxDim + dim] > w.box[dim]) {
                const float* col = sxo + (size_t)dim * TS;
                // radix select of rank floor(lc/2) on order-preserving keys; the
                // bits above the highest bit where the node's min and max keys
                // differ are common to every key and are skipped
                // (keys of x + 0: -0 and +0 compare equal as floats and get one key)
                const uint32_t kmin = float_key(__fadd_rn(w.box[dim], 0.0f));
                const uint32_t kmax = float_key(__fadd_rn(w.box[kMaxDim + dim], 0.0f));
                const int top = 32 - __clz(kmin ^ kmax);
                int rank = lc >> 1;
                uint32_t mask = (top >= 32) ? 0u : ~((1u << top) - 1u);
                uint32_t prefix = kmin & mask;
                for (int hi = top; hi > 0; hi -= 8) {
                    const int shift = hi >= 8 ? hi - 8 : 0;
                    const int width = hi - shift;
                    const uint32_t dmask = (1u << width) - 1u;
                    for (int b = lane; b < 256; b += 32) w.rh[b] = 0;
                    __syncwarp();
#pragma unroll 4
                    for (int j = lane; j < lc; j += 32) {
                        uint32_t key = float_key(__fadd_rn(col[ixc[ls + j]], 0.0f));
                        if ((key & mask) == prefix) atomicAdd(&w.rh[(key >> shift) & dmask], 1);
                    }
                    __syncwarp();
                    int loc = 0;
#pragma unroll
                    for (int q = 0; q < 8; q++) loc += w.rh[8 * lane + q];
                    int incl = warp_incl_scan(loc);
                    int excl = incl - loc;
                    int found = -1, below = 0;
                    if (rank >= excl && rank < incl) {
                        int c = excl;
                        for (int q = 0; q < 8; q++) {
                            int h = w.rh[8 * lane + q];
                            if (rank < c + h) {
                                found = 8 * lane + q;
                                below = c;
                                break;
                            }
                            c += h;
                        }
                    }
                    unsigned bal = __ballot_sync(kFull, found >= 0);
                    int src = __ffs(bal) - 1;
                    int digit = __shfl_sync(kFull, found, src);
                    below = __shfl_sync(kFull, below, src);
                    prefix |= (uint32_t)digit << shift;
                    mask |= dmask << shift;
                    rank -= below;
                    __syncwarp();
                }
                const float vp = key_float(prefix);
                int na = 0, nb = 0;
                float up = INFINITY;
#pragma unroll 4
                for (int j = lane; j < lc; j += 32) {
                    float x = col[ixc[ls + j]];
                    na += x < vp;
                    nb += x <= vp;
                    if (x > vp) up = fminf(up, x);
                }
                na = warp_sum(na);
                nb = warp_sum(nb);
                up = warp_min(up);
                long long e1 = 2LL * na - lc;
                if (e1 < 0) e1 = -e1;
                float sv = vp;
                int cv = na;
                if (nb < lc) {
                    long long e2 = 2LL * nb - lc;
                    if (e2 < 0) e2 = -e2;
                    if (e2 < e1) {
                        sv = up;
                        cv = nb;
                    }
                }
                if (cv > 0) {
                    mode = kModeValue;
                    s = sv;
                    cleft = cv;
                }
            }
            if (mode < 0) {
                unsigned used = 0;
                for (int r = 0; r < d && mode < 0; r++) {
                    int k = argmax_dims(w.var, d, used);
                    used |= 1u << k;
                    const float mn = w.box[k], mx = w.box[kMaxDim + k];
                    if (mx > mn) {
                        const float* col = sxo + (size_t)k * TS;
                        float nxt = INFINITY;
                        for (int j = lane; j < lc; j += 32) {
                            float x = col[ixc[ls + j]];
                            if (x > mn) nxt = fminf(nxt, x);
                        }
                        nxt = warp_min(nxt);
                        int c = 0;
                        for (int j = lane; j < lc; j += 32) c += col[ixc[ls + j]] < nxt;
                        cleft = warp_sum(c);
                        s = nxt;
                        dim = k;
                        mode = kModeValue;
                    }
                }
                if (mode < 0) {
                    mode = kModeIndex;
                    dim = 0;
                    s = w.box[0];
                    cleft = (lc + 1) >> 1;
                }
            }
            // ---- stable partition by warp ballots
            {
                const float* col = sxo + (size_t)dim * TS;
                const int half = (lc + 1) >> 1;
                int lcnt = 0, rcnt = 0;
                for (int b0 = 0; b0 < lc; b0 += 32) {
                    const int j = b0 + lane;
                    const bool valid = j < lc;
                    const int p = valid ? ixc[ls + j] : 0;
                    const bool lft = valid && (mode == kModeIndex ? (j < half) : (col[p] < s));
                    const unsigned bl = __ballot_sync(kFull, lft);
                    const unsigned bv = __ballot_sync(kFull, valid);
                    const unsigned br = bv & ~bl;
                    if (lft) ixn[ls + lcnt + __popc(bl & lanemask_lt())] = (unsigned short)p;
                    else if (valid) ixn[ls + cleft + rcnt + __popc(br & lanemask_lt())] = (unsigned short)p;
                    lcnt += __popc(bl);
                    rcnt += __popc(br);
                }
                if (lane == 0 && lcnt != cleft) atomicOr(a.err, kErrInternal);
            }
            if (pool_next + 2 > pool_end) {
                int c0 = 0;
                if (lane == 0) c0 = atomicAdd(&a.cnt[kCntNodes], kIdChunk);
                pool_next = __shfl_sync(kFull, c0, 0);
                pool_end = pool_next + kIdChunk;
                if (pool_end > a.node_cap && lane == 0) atomicOr(a.err, kErrNodeOverflow);
            }
            const int c0 = pool_next;
            pool_next += 2;
            unsigned meta = (unsigned)dim | (mode == kModeIndex ? kMetaIndex : 0u);
            write_node(a, node, make_int4(c0, start + ls + cleft, __float_as_int(s), (int)meta), w.box);
            my_nodes++;
            __syncwarp();
            if (lane == 0) {
                const int ew = (depth + 1) | ((rel + 1) << 16);
                w.stk[sp] = make_int4(ls + cleft, lc - cleft, c0 + 1, ew);
                w.stk[sp + 1] = make_int4(ls, cleft, c0, ew);
            }
            sp += 2;
            __syncwarp();
        }
    }
    // the ids left in this warp's pool are holes nothing references: give them
    // an all-zero header (not a leaf) so a scan of the node table reads no garbage
    for (int id = pool_next + lane; id < pool_end; id += 32)
        if (id < a.node_cap) reinterpret_cast<int4*>(a.nodes)[(long long)id * a.ns] = make_int4(0, 0, 0, 0);
    if (lane == 0 && my_nodes) {
        atomicAdd(&a.cnt[kCntRealNodes], my_nodes);
        atomicAdd(&a.cnt[kCntLeaves], my_leaves);
        atomicMax(&a.cnt[kCntDepth], my_depth);
    }
}

// Bottom-up boxes of the level-stage nodes: union of the two children.
// Levels L_hi down to L_lo; a launch covers several levels only as one block
// (the block barrier orders them), a grid covers one level.
__global__ void k_boxes(BuildArgs a, int L_hi, int L_lo)
{
    griddep_enter();
    for (int L = L_hi; L >= L_lo; L--) {
        const int A = a.lvl_count[L];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A; i += gridDim.x * blockDim.x) {
            const int node = a.lvl_nodes[L * a.lvl_stride + i];
            if (node >= a.node_cap) continue;
            float* rec = reinterpret_cast<float*>(a.nodes + (long long)node * a.ns);
            const int c = reinterpret_cast<const int*>(rec)[0];
            if (c + 1 >= a.node_cap) continue;
            const float* r0 = reinterpret_cast<const float*>(a.nodes + (long long)c * a.ns);
            const float* r1 = reinterpret_cast<const float*>(a.nodes + (long long)(c + 1) * a.ns);
            for (int k = 0; k < a.d; k++) {
                rec[4 + k] = fminf(r0[4 + k], r1[4 + k]);
                rec[4 + a.dp + k] = fmaxf(r0[4 + a.dp + k], r1[4 + a.dp + k]);
            }
            for (int k = a.d; k < a.dp; k++) {
                rec[4 + k] = 0.0f;
                rec[4 + a.dp + k] = 0.0f;
            }
            for (int q = 4 + 2 * a.dp; q < 4 * a.ns; q++) rec[q] = 0.0f;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host

namespace {

struct Buffers {
    std::vector<void*> ptrs;
    cudaStream_t s;
    explicit Buffers(cudaStream_t st) : s(st) {}
    ~Buffers() { for (void* p : ptrs) ws_free(p, s); }
    template <typename T>
    panda_status get(T** out, size_t count, const char* what)
    {
        void* p = nullptr;
        panda_status st = ws_alloc(&p, std::max<size_t>(count, 1) * sizeof(T), s, what);
        if (st != PANDA_OK) return st;
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return PANDA_OK;
    }
};

// Nodes of at most T points go to the subtree stage (one warp each, in shared
// memory); above it the level passes split them.  512 rather than 1024: the
// subtree stage then runs about twice the warps per SM (2^24 cosmology build:
// subtree 2.61 -> 1.57 ms), and the extra level pass costs less than that,
// since nodes of at most 1024 points are split by exact selection in k_sample
// (all their points are samples) and the child plan is one block per chunk.
int subtree_threshold(int d, int bucket)
{
    (void)d;
    int T = 512;
    return std::max(T, bucket);
}

panda_status configure_kernels()
{
    static PerDeviceOnce once;
    return once_per_device(once, [] {
        PANDA_CUDA(cudaFuncSetAttribute(k_sample, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kMaxDim * kSamples * 4),
                   "configure k_sample");
        PANDA_CUDA(cudaFuncSetAttribute(k_subtree, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
                   "configure k_subtree");
        return PANDA_OK;
    });
}

struct Plan {
    int T, act_cap, tile_cap, small_cap, lvl_stride, max_levels;
    int sub_warps;   // warps of the k_subtree block (one block per SM)
    long long node_cap;
};

// Warps of the persistent k_subtree block: as many as the shared memory (one
// node of <= T points per warp) and the register file allow, checked with the
// occupancy calculator (register allocation rounds warps up).  Called before
// any enqueue, so a captured build needs no query.
panda_status subtree_warps(int d, int T, int* out)
{
    const int wb = (int)warp_bytes(d, T);
    int w = std::max(1, std::min(kSubtreeMaxWarps, (227 * 1024) / wb));
    for (; w > 1; w--) {
        int nb = 0;
        PANDA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_subtree, w * 32, (size_t)w * wb),
                   "k_subtree occupancy");
        if (nb >= 1) break;
    }
    *out = w;
    return PANDA_OK;
}

}  // namespace

// Build workspace: device buffers of one build (or of a reusable forest plan).
struct BuildState {
    BuildArgs a;
    Plan pl;
    std::vector<void*> bufs;
    int max_set = 0;   // largest tree (sets the number of level passes)
};

namespace {

panda_status build_alloc(BuildState& S, int n, int d, cudaStream_t stream)
{
    BuildArgs& a = S.a;
    const Plan& pl = S.pl;
    panda_status st;
    auto get = [&](auto** ptr, size_t count, const char* what) -> panda_status {
        void* p = nullptr;
        panda_status r = ws_alloc(&p, std::max<size_t>(count, 1) * sizeof(**ptr), stream, what);
        if (r != PANDA_OK) return r;
        S.bufs.push_back(p);
        *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(p);
        return PANDA_OK;
    };
#define GET(ptr, count, what) \
    if ((st = get(&(ptr), (count), what)) != PANDA_OK) return st
    const size_t np = (size_t)a.n_pad;
    for (int p = 0; p < 2; p++) {
        GET(a.X[p], np * d, "coordinate buffers");
        GET(a.ID[p], np, "id buffers");
        GET(a.act[p], (size_t)pl.act_cap, "level lists");
        GET(a.tile_base[p], (size_t)pl.act_cap + 1, "tile bases");
        GET(a.tiles[p], (size_t)pl.tile_cap, "tiles");
    }
    GET(a.tleft, (size_t)pl.tile_cap, "tile counts");
    GET(a.tleftoff, (size_t)pl.tile_cap, "tile offsets");
    GET(a.tbins, (size_t)pl.tile_cap * (1 + kWin), "tile window bins");
    GET(a.vs, (size_t)pl.act_cap * kSamples, "samples");
    GET(a.nhist, (size_t)pl.act_cap * (kSamples + 1), "histograms");
    GET(a.nvar, (size_t)pl.act_cap * kMaxDim, "variances");
    GET(a.ndim, (size_t)pl.act_cap, "split dims");
    GET(a.nmode, (size_t)pl.act_cap, "split modes");
    GET(a.nsplit, (size_t)pl.act_cap, "split values");
    GET(a.nleft, (size_t)pl.act_cap, "left counts");
    GET(a.nsel, (size_t)pl.act_cap, "split positions");
    GET(a.small, (size_t)pl.small_cap, "subtree list");
    GET(a.lvl_nodes, (size_t)pl.lvl_stride * pl.max_levels, "level nodes");
    GET(a.lvl_count, (size_t)pl.max_levels, "level counts");
    a.chunk_cap = pl.act_cap / kChildChunk + 2;
    GET(a.chunk_act, (size_t)a.chunk_cap, "child sums");
    GET(a.chunk_small, (size_t)a.chunk_cap, "child sums");
    GET(a.chunk_tiles, (size_t)a.chunk_cap, "tile sums");
    GET(a.cnt, (size_t)kCntSlots, "counters");
    GET(a.err, (size_t)1, "error word");
#undef GET
    return PANDA_OK;
}

void build_release(BuildState& S, cudaStream_t stream)
{
    for (void* p : S.bufs) ws_free(p, stream);
    S.bufs.clear();
}

void init_args(BuildState& S, const float* points, int n, int d, int bucket, const panda_tree* t)
{
    BuildArgs& a = S.a;
    const Plan& pl = S.pl;
    a.n = n;
    a.d = d;
    a.dp = t->dp;
    a.bucket = bucket;
    a.T = pl.T;
    a.n_pad = (n + 3) & ~3;
    a.in = points;
    a.act_cap = pl.act_cap;
    a.tile_cap = pl.tile_cap;
    a.small_cap = pl.small_cap;
    a.lvl_stride = pl.lvl_stride;
    a.node_cap = pl.node_cap;
    a.ns = t->ns;
    a.nv = t->nv;
    a.nodes = t->nodes;
    a.pts = t->points;
}

// Clear counters, transpose the points and seed the roots.
panda_status enqueue_start(BuildState& S, cudaStream_t stream, PhaseTimer& timer)
{
    BuildArgs& a = S.a;
    PANDA_CUDA(cudaMemsetAsync(a.cnt, 0, kCntSlots * sizeof(int), stream), "clear counters");
    PANDA_CUDA(cudaMemsetAsync(a.err, 0, sizeof(unsigned), stream), "clear error word");
    PANDA_CUDA(cudaMemsetAsync(a.lvl_count, 0, S.pl.max_levels * sizeof(int), stream), "clear levels");
    const int sms = num_sms();
    timer.begin("transpose");
    int blocks = (int)std::min<long long>((a.n_pad + 255) / 256, (long long)sms * 16);
    PANDA_LAUNCH(k_transpose, blocks, 256, 0, stream, a);
    PANDA_LAUNCH(k_init, 1, 1024, 0, stream, a);
    return PANDA_OK;
}

// The seven kernels of one data-parallel level pass.
panda_status enqueue_level(BuildState& S, int L, cudaStream_t stream, PhaseTimer& timer)
{
    BuildArgs& a = S.a;
    const Plan& pl = S.pl;
    const int d = a.d;
    const int acap = (int)std::min<long long>(L < 30 ? (1LL << L) * std::max(1, a.set_off ? a.nsets : 1)
                                                     : (1LL << 30), pl.act_cap);
    const int tcap = (int)std::min<long long>(pl.tile_cap, (long long)a.n / kTile + 2LL * acap + 2);
    timer.begin("level.sample");
    PANDA_LAUNCH(k_sample, acap, kSampleThreads, std::max(d, 2) * kSamples * 4, stream, a, L);
    PANDA_LAUNCH(k_sample_small, (acap + kSmallWarps - 1) / kSmallWarps, kSmallWarps * 32, 0, stream, a, L);
    timer.begin("level.hist");
    PANDA_LAUNCH(k_hist, std::min(tcap, 8 * num_sms()), 256, 0, stream, a, L);
    timer.begin("level.select");
    PANDA_LAUNCH(k_select, std::min(acap, 8 * num_sms()), kSelectThreads, 0, stream, a, L);
    PANDA_LAUNCH(k_hist_full, std::min(tcap, 8 * num_sms()), 256, 0, stream, a, L);
    PANDA_LAUNCH(k_select_full, std::min(acap, 8 * num_sms()), kSelectThreads, 0, stream, a, L);
    PANDA_LAUNCH(k_tilecount, std::min(tcap, 8 * num_sms()), 256, 0, stream, a, L);
    PANDA_LAUNCH(k_tileoff, (acap + 7) / 8, 256, 0, stream, a, L);
    const int nchunk = (acap + kChildChunk - 1) / kChildChunk;
    const int nxt_cap = (int)std::min<long long>(2LL * acap, pl.act_cap);
    PANDA_LAUNCH(k_children, nchunk, kChildThreads, 0, stream, a, L);
    PANDA_LAUNCH(k_plan, (nxt_cap + kChildChunk - 1) / kChildChunk, kChildThreads, 0, stream, a, L);
    timer.begin("level.partition");
    PANDA_LAUNCH(k_partition, tcap, 256, 0, stream, a, L);
    return PANDA_OK;
}

// Subtree stage and the level-stage boxes.
panda_status enqueue_finish(BuildState& S, int nlevels, cudaStream_t stream, PhaseTimer& timer)
{
    BuildArgs& a = S.a;
    const int sms = num_sms();
    timer.begin("subtree");
    const int wb = (int)warp_bytes(a.d, S.pl.T);
    const int wpb = S.pl.sub_warps;
    PANDA_LAUNCH(k_subtree, sms, wpb * 32, (size_t)wpb * wb, stream, a, wb);
    timer.begin("boxes");
    // bottom-up: a level with more nodes than one block covers at once gets a
    // grid of its own, the levels above it go together in one block
    int L = nlevels - 1;
    for (; L >= 0; L--) {
        const long long bound = std::min<long long>(
            L < 30 ? (1LL << L) * std::max(1, a.set_off ? a.nsets : 1) : (1LL << 30), S.pl.act_cap);
        if (bound <= 1024) break;
        PANDA_LAUNCH(k_boxes, (unsigned)((bound + 255) / 256), 256, 0, stream, a, L, L);
    }
    if (L >= 0) {
        PANDA_LAUNCH(k_boxes, 1, 1024, 0, stream, a, L, 0);
    }
    timer.end();
    return PANDA_OK;
}

int levels_for(int max_set, int T)
{
    if (max_set <= T) return 0;
    return (int)ceil(log2((double)max_set / T)) + 2;
}

void set_tree_counts(panda_tree* t, const int* hc, long long level_ids, long long n_small)
{
    // ids below level_ids belong to the level stage (subtree roots included,
    // which the subtree stage counts again); the rest of the table may hold holes
    t->node_slots = hc[kCntNodes];
    t->num_nodes = level_ids + hc[kCntRealNodes] - n_small;
    t->num_leaves = hc[kCntLeaves];
    t->depth = hc[kCntDepth];
}

panda_status build_once(const float* points, int n, int d, int bucket, cudaStream_t stream,
                        const Plan& pl, panda_tree* t, int* need_small, long long* need_nodes,
                        unsigned* err_out)
{
    PhaseTimer timer(stream);
    BuildState S;
    memset(&S.a, 0, sizeof(S.a));
    S.pl = pl;
    init_args(S, points, n, d, bucket, t);
    struct Release {
        BuildState& s;
        cudaStream_t st;
        ~Release() { build_release(s, st); }
    } release{S, stream};
    panda_status st = build_alloc(S, n, d, stream);
    if (st != PANDA_OK) return st;
    if ((st = enqueue_start(S, stream, timer)) != PANDA_OK) return st;
    int L = 0;
    const int levels_est = std::min(levels_for(n, pl.T), pl.max_levels);
    for (; L < levels_est; L++)
        if ((st = enqueue_level(S, L, stream, timer)) != PANDA_OK) return st;
    int hc[kCntSlots];
    unsigned herr = 0;
    for (;;) {
        PANDA_CUDA(cudaMemcpyAsync(hc, S.a.cnt, sizeof(hc), cudaMemcpyDeviceToHost, stream), "read counters");
        PANDA_CUDA(cudaMemcpyAsync(&herr, S.a.err, sizeof(herr), cudaMemcpyDeviceToHost, stream), "read error");
        PANDA_CUDA(cudaStreamSynchronize(stream), "level stage");
        if (herr) break;
        if (hc[kCntActive0 + (L & 1)] == 0) break;
        if (L >= pl.max_levels) {
            herr |= kErrDepth;
            break;
        }
        if ((st = enqueue_level(S, L, stream, timer)) != PANDA_OK) return st;
        L++;
    }
    *need_small = hc[kCntSmall];
    *err_out = herr;
    if (herr) return PANDA_OK;   // caller decides (retry or error)
    const int nlevels = hc[kCntLevels];
    const long long level_ids = hc[kCntNodes], n_small = hc[kCntSmall];
    if ((st = enqueue_finish(S, nlevels, stream, timer)) != PANDA_OK) return st;
    PANDA_CUDA(cudaMemcpyAsync(hc, S.a.cnt, sizeof(hc), cudaMemcpyDeviceToHost, stream), "read counters");
    PANDA_CUDA(cudaMemcpyAsync(&herr, S.a.err, sizeof(herr), cudaMemcpyDeviceToHost, stream), "read error");
    PANDA_CUDA(cudaStreamSynchronize(stream), "subtree stage");
    timer.finish();
    *need_nodes = hc[kCntNodes];
    *err_out = herr;
    set_tree_counts(t, hc, level_ids, n_small);
    return PANDA_OK;
}

}  // namespace

// ------------------------------------------------------------------ forests

// A forest of independent trees over the concatenated point sets (set s =
// rows [set_off[s], set_off[s+1])): root of set s is node s.  Its buffers are
// allocated once; forest_enqueue then launches a fixed number of level passes
// (enough for the largest set plus two) with no host synchronisation, so the
// whole build can be captured in a CUDA graph; running out of passes is
// reported through the error word (kErrLevels).
panda_status forest_create(const long long* set_sizes, int nsets, int d, int bucket, const float* points,
                           cudaStream_t stream, panda_tree* t, BuildState** out)
{
    *out = nullptr;
    if (nsets < 1 || d < 1 || d > kMaxDim || bucket < 1 || bucket > kMaxBucket) {
        set_error("forest: invalid sets, d or bucket");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    long long n = 0;
    int max_set = 0;
    std::vector<int> off(nsets + 1, 0);
    for (int s = 0; s < nsets; s++) {
        if (set_sizes[s] < 1) {
            set_error("forest: set %d is empty", s);
            return PANDA_ERR_INVALID_ARGUMENT;
        }
        off[s] = (int)n;
        n += set_sizes[s];
        max_set = std::max<long long>(max_set, set_sizes[s]);
        if (n >= (1LL << 31) - 4) {
            set_error("forest: more than 2^31 points in total");
            return PANDA_ERR_UNSUPPORTED;
        }
    }
    off[nsets] = (int)n;
    panda_status st = configure_kernels();
    if (st != PANDA_OK) return st;
    cudaGetDevice(&t->device);
    t->n = n;
    t->d = d;
    t->dp = padded_dim(d);
    t->bucket = bucket;
    t->nv = point_float4s(t->dp);
    t->ns = node_float4s(t->dp);
    BuildState* S = new BuildState();
    memset(&S->a, 0, sizeof(S->a));
    Plan& pl = S->pl;
    pl.T = subtree_threshold(d, bucket);
    t->threshold = pl.T;
    if ((st = subtree_warps(d, pl.T, &pl.sub_warps)) != PANDA_OK) {
        delete S;
        return st;
    }
    pl.act_cap = (int)(n / (pl.T + 1)) + 1;
    pl.tile_cap = (int)(n / kTile) + 2 * pl.act_cap + 4;
    pl.small_cap = nsets + 8 * pl.act_cap + 64;
    pl.lvl_stride = pl.act_cap;
    pl.max_levels = kMaxDepth + 1;
    pl.node_cap = 2LL * n + 8 + nsets + (long long)num_sms() * kSubtreeMaxWarps * kIdChunk;
    S->max_set = max_set;
    t->node_cap = pl.node_cap;
    void *pn = nullptr, *pp = nullptr, *po = nullptr;
    st = ws_alloc(&pn, (size_t)pl.node_cap * t->ns * sizeof(float4), stream, "forest nodes");
    if (st == PANDA_OK) st = ws_alloc(&pp, (size_t)n * t->nv * sizeof(float4), stream, "forest points");
    if (st == PANDA_OK) st = ws_alloc(&po, (size_t)(nsets + 1) * sizeof(int), stream, "forest set offsets");
    if (st != PANDA_OK) {
        ws_free(pn, stream);
        ws_free(pp, stream);
        ws_free(po, stream);
        delete S;
        return st;
    }
    t->nodes = static_cast<float4*>(pn);
    t->points = static_cast<float4*>(pp);
    S->bufs.push_back(po);
    init_args(*S, points, (int)n, d, bucket, t);
    S->a.set_off = static_cast<const int*>(po);
    S->a.nsets = nsets;
    cudaError_t e = cudaMemcpyAsync(po, off.data(), (nsets + 1) * sizeof(int), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) st = cuda_fail(e, "forest: set offsets");
    if (st == PANDA_OK) st = build_alloc(*S, (int)n, d, stream);
    if (st != PANDA_OK) {
        build_release(*S, stream);
        ws_free(pn, stream);
        ws_free(pp, stream);
        t->nodes = nullptr;
        t->points = nullptr;
        delete S;
        return st;
    }
    *out = S;
    return PANDA_OK;
}

int forest_levels(const BuildState* S) { return std::min(levels_for(S->max_set, S->pl.T) + 2, S->pl.max_levels); }

panda_status forest_enqueue(BuildState* S, cudaStream_t stream)
{
    PhaseTimer timer(stream);
    panda_status st = enqueue_start(*S, stream, timer);
    if (st != PANDA_OK) return st;
    const int L = forest_levels(S);
    for (int l = 0; l < L; l++)
        if ((st = enqueue_level(*S, l, stream, timer)) != PANDA_OK) return st;
    PANDA_LAUNCH(k_check_levels, 1, 32, 0, stream, S->a, L);
    return enqueue_finish(*S, L, stream, timer);
}

// After the stream has passed a forest build: its error word and node counts.
panda_status forest_collect(BuildState* S, panda_tree* t, unsigned* err, cudaStream_t stream)
{
    int hc[kCntSlots];
    PANDA_CUDA(cudaMemcpyAsync(hc, S->a.cnt, sizeof(hc), cudaMemcpyDeviceToHost, stream), "forest counters");
    PANDA_CUDA(cudaMemcpyAsync(err, S->a.err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream), "forest error");
    PANDA_CUDA(cudaStreamSynchronize(stream), "forest collect");
    // level-stage ids: roots plus two per split; subtree roots are counted twice
    long long level_ids = 0;
    int lc[kMaxDepth + 1];
    PANDA_CUDA(cudaMemcpy(lc, S->a.lvl_count, sizeof(int) * S->pl.max_levels, cudaMemcpyDeviceToHost),
               "forest level counts");
    level_ids = S->a.nsets;
    for (int l = 0; l < S->pl.max_levels; l++) level_ids += 2LL * lc[l];
    set_tree_counts(t, hc, level_ids, hc[kCntSmall]);
    return PANDA_OK;
}

void forest_destroy(BuildState* S, cudaStream_t stream)
{
    if (!S) return;
    build_release(*S, stream);
    delete S;
}

panda_status build_tree(const float* points, int64_t n64, int32_t d, int32_t bucket, cudaStream_t stream,
                        panda_tree** out)
{
    *out = nullptr;
    if (!points || n64 < 1 || n64 >= (1LL << 31) - 4 || d < 1 || bucket < 1) {
        set_error("panda_build: invalid argument (n=%lld d=%d bucket=%d)", (long long)n64, d, bucket);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (d > kMaxDim || bucket > kMaxBucket) {
        set_error("panda_build: unsupported d=%d or bucket=%d (max %d, %d)", d, bucket, kMaxDim, kMaxBucket);
        return PANDA_ERR_UNSUPPORTED;
    }
    if (!is_device_ptr(points)) {
        set_error("panda_build: points must be a device pointer");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    panda_status st = configure_kernels();
    if (st != PANDA_OK) return st;
    const int n = (int)n64;
    panda_tree* t = new panda_tree();
    cudaGetDevice(&t->device);
    t->n = n;
    t->d = d;
    t->dp = padded_dim(d);
    t->bucket = bucket;
    t->nv = point_float4s(t->dp);
    t->ns = node_float4s(t->dp);
    Plan pl;
    pl.T = subtree_threshold(d, bucket);
    t->threshold = pl.T;
    if ((st = subtree_warps(d, pl.T, &pl.sub_warps)) != PANDA_OK) return st;
    pl.act_cap = n / (pl.T + 1) + 1;
    pl.tile_cap = n / kTile + 2 * pl.act_cap + 4;
    pl.small_cap = 4 * pl.act_cap + 16;
    pl.lvl_stride = pl.act_cap;
    pl.max_levels = kMaxDepth + 1;
    // holes: each subtree warp may leave up to kIdChunk unused ids
    const long long hole_slack = (long long)num_sms() * kSubtreeMaxWarps * kIdChunk;
    const long long node_max = 2LL * n + 8 + hole_slack;
    pl.node_cap = 4LL * n / bucket + 8LL * pl.act_cap + 1024 + hole_slack;
    pl.node_cap = std::min<long long>(pl.node_cap, node_max);
    for (int attempt = 0; attempt < 3; attempt++) {
        t->node_cap = pl.node_cap;
        void* pn = nullptr;
        void* pp = nullptr;
        st = ws_alloc(&pn, (size_t)pl.node_cap * t->ns * sizeof(float4), stream, "tree nodes");
        if (st != PANDA_OK) break;
        st = ws_alloc(&pp, (size_t)n * t->nv * sizeof(float4), stream, "tree points");
        if (st != PANDA_OK) {
            ws_free(pn, stream);
            break;
        }
        t->nodes = static_cast<float4*>(pn);
        t->points = static_cast<float4*>(pp);
        int need_small = 0;
        long long need_nodes = 0;
        unsigned err = 0;
        st = build_once(points, n, d, bucket, stream, pl, t, &need_small, &need_nodes, &err);
        bool retry = false;
        if (st == PANDA_OK && err) {
            if (err & kErrNonfinite) {
                set_error("panda_build: non-finite coordinate in the input");
                st = PANDA_ERR_NONFINITE_INPUT;
            } else if (err & kErrDepth) {
                set_error("panda_build: a node below depth %d still holds more than %d points", kMaxDepth, bucket);
                st = PANDA_ERR_DEPTH;
            } else if (err & (kErrInternal | kErrTileOverflow | kErrActiveOverflow)) {
                set_error("panda_build: internal consistency check failed (0x%x)", err);
                st = PANDA_ERR_CUDA;
            } else {
                if (err & kErrSmallOverflow) pl.small_cap = std::max(pl.small_cap * 2, need_small + 16);
                if (err & kErrNodeOverflow) pl.node_cap = std::min<long long>(node_max, std::max(pl.node_cap * 2, need_nodes + 16));
                retry = true;
            }
        }
        if (st != PANDA_OK || retry) {
            cudaStreamSynchronize(stream);
            ws_free(t->nodes, stream);
            ws_free(t->points, stream);
            t->nodes = nullptr;
            t->points = nullptr;
            if (st != PANDA_OK) break;
            continue;
        }
        // root box for query ordering
        float rec[4 + 2 * kMaxDim + 4];
        cudaError_t e = cudaMemcpyAsync(rec, t->nodes, t->ns * sizeof(float4), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "read root");
            break;
        }
        for (int k = 0; k < d; k++) {
            t->root_lo[k] = rec[4 + k];
            t->root_hi[k] = rec[4 + t->dp + k];
        }
        *out = t;
        return PANDA_OK;
    }
    if (st == PANDA_OK) {
        set_error("panda_build: capacity retries exhausted");
        st = PANDA_ERR_OUT_OF_MEMORY;
    }
    delete t;
    return st;
}

}  // namespace panda
