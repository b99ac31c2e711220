// common.cuh -- shared definitions of the CUDA path (sm_103a).
//
// Method: PANDA's local kd-tree build and KNN query (arXiv 1607.08220,
// Sec. III-A, III-A1, Algorithm 1).  This header holds the constants, the
// device records and the small warp/block primitives the kernels share.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "panda.h"

namespace panda {

constexpr int kSamples = 1024;     // local-tree sample count (Sec. III-A1)
constexpr int kMaxDepth = 64;      // deepest level allowed below the root
constexpr int kMaxDim = 16;
constexpr int kMaxBucket = 256;
constexpr int kMaxK = 64;
// Default scan-shape switch of the packet traversal: a bucket needed by at most
// this many of a warp's lanes is scanned lanes = points (measured best between
// 12 and 24 on 3-D self-KNN and 10-D queries; 16 on both).
constexpr int kTransposeMaxDefault = 16;
constexpr int kTile = 16384;       // points per level-stage tile (multiple of 4)
constexpr unsigned kFull = 0xffffffffu;

// Device error word bits.
enum : unsigned {
    kErrNonfinite = 1u,
    kErrNodeOverflow = 2u,
    kErrSmallOverflow = 4u,
    kErrDepth = 8u,
    kErrActiveOverflow = 16u,
    kErrTileOverflow = 32u,
    kErrInternal = 64u,
    kErrLevels = 128u,   // a graph-captured build ran out of level passes
};

// Split modes of a node.
// kModeSelected: a value split whose split value and left count k_sample
// already found by exact selection (every point of the node is a sample);
// every kernel after the selection treats it as a value split.
// kModeRehist: a value split whose crossing of n/2 fell outside the window of
// interval points the first histogram counts one by one; a second pass
// histograms it over all interval points, and it is a value split after that.
enum : int { kModeValue = 0, kModeIndex = 1, kModePending = 2, kModeSelected = 3, kModeRehist = 4 };

// Node record: int32 a, int32 b, float split, uint32 meta, lo[DP], hi[DP], pad.
constexpr unsigned kMetaLeaf = 0x80000000u;
constexpr unsigned kMetaIndex = 0x40000000u;
// Set by a refit on an inner node whose children no longer lie on their sides of
// the split plane (a point crossed it): the plane is then no bound for pruning.
constexpr unsigned kMetaCross = 0x20000000u;
constexpr unsigned kMetaDimMask = 31u;

// Padded dimension class used by the packed layouts and the query kernels:
// padded coordinates are 0 in both points and queries, so they add +0 after
// the real dimensions and leave every distance bit-identical.
inline int padded_dim(int d)
{
    if (d <= 2) return 2;
    if (d <= 4) return d;
    if (d <= 8) return 8;
    if (d <= 10) return 10;
    return 16;
}
inline int node_float4s(int dp) { return (4 + 2 * dp + 3) / 4; }
inline int point_float4s(int dp) { return (dp + 1 + 3) / 4; }

struct Active {          // node processed by the data-parallel level stage
    int start, count, node, depth;
};
struct Small {           // node handed to the shared-memory subtree stage
    int start, count, node, depth_parity;  // depth << 1 | buffer parity
};
struct Tile {            // contiguous slice of one active node
    int node, begin, end, first;           // first = 1 for the node's first tile
};

// Counter slots in device memory.
enum : int {
    kCntActive0 = 0,   // active count at even levels
    kCntActive1 = 1,   // ... odd levels
    kCntTiles0 = 2,
    kCntTiles1 = 3,
    kCntSmall = 4,
    kCntNodes = 5,
    kCntSmallNext = 6,
    kCntLeaves = 7,
    kCntDepth = 8,
    kCntLevels = 9,    // number of level-stage levels that had active nodes
    kCntRealNodes = 10, // nodes written by the subtree stage (the rest of its id range are holes)
    kCntRehist = 11,   // nodes of the current level marked kModeRehist
    kCntSlots = 16,
};

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while its predecessor in the stream is finishing;
// griddep_wait() blocks until the predecessor grid has completed and its memory
// is visible (it returns at once for a kernel launched without the attribute),
// and griddep_launch_dependents() lets the next grid be scheduled once every
// block of this one is running.  Every kernel of the build and query calls both
// before it touches memory written by an earlier launch.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_enter()
{
    griddep_wait();
    griddep_launch_dependents();
}

__device__ __forceinline__ uint32_t float_key(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k)
{
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// FP32 sum of one value per lane in the fixed order of the split rule:
// lane p holds the sequential partial of elements j = p (mod 32); the
// partials are then added pairwise at offsets 16, 8, 4, 2, 1.  Lane 0's
// result is returned to every lane.
__device__ __forceinline__ float fixed_order_warp_total(float part)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) part = __fadd_rn(part, __shfl_down_sync(kFull, part, o));
    return __shfl_sync(kFull, part, 0);
}

// Index of the maximum by a sequential scan with strict '>' (ties keep the lowest
// dimension), skipping dims flagged in `used`.
__device__ __forceinline__ int argmax_dims(const float* var, int d, unsigned used)
{
    int best = -1;
    for (int k = 0; k < d; k++) {
        if (used & (1u << k)) continue;
        if (best < 0 || var[k] > var[best]) best = k;
    }
    return best;
}

// Number of sorted values a[0..32) that are <= x (a padded 32-entry row).
__device__ __forceinline__ int count_le32(const float* a, float x)
{
    int c = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1)
        if (a[c + s - 1] <= x) c += s;
    if (a[c] <= x) c++;
    return c;
}

}  // namespace panda
