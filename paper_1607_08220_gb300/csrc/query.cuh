// query.cuh -- exact KNN traversal kernel (Algorithm 1, corrected) for sm_103a.
//
// One warp serves 32 queries (one per lane) that were grouped by spatial key,
// so they traverse nearly the same nodes.  The warp walks one shared stack
// (Algorithm 1's S): at every popped node each lane computes its own bound,
// the squared distance from its query to the node's tight box, and the node
// is skipped only when every lane's bound is strictly greater than its current
// k-th distance (corrections C1, C3).  Inner nodes push the far child first
// and the near child last (Algorithm 1 lines 20-24); the near side is the one
// the majority of the lanes that need the node fall on.  A leaf bucket is
// staged once into shared memory and scanned by all lanes (Sec. III-C: the
// bucket scan is the SIMD-friendly part); each lane keeps its top-k list (the
// heap H) sorted in registers as 64-bit keys (d2 bits << 32 | id), so the
// radius r' is always the k-th key (correction C2).
#pragma once

#include "common.cuh"

namespace panda {

struct KnnArgs {
    const float4* nodes;
    const float4* pts;
    const float* queries;
    const int* perm;      // sorted position -> query row (nullptr: identity)
    int* ids;
    float* d2;
    unsigned* err;
    long long m;
    long long num_nodes;
    long long npts;
    int d, k;
};

constexpr unsigned long long kKeyEmpty = (0x7f800000ull << 32) | 0xffffffffull;

template <int KC>
__device__ __forceinline__ void topk_insert(unsigned long long (&s)[KC], unsigned long long c)
{
    bool lt[KC];
#pragma unroll
    for (int i = 0; i < KC; i++) lt[i] = c < s[i];
#pragma unroll
    for (int i = KC - 1; i >= 1; i--) s[i] = lt[i - 1] ? s[i - 1] : (lt[i] ? c : s[i]);
    s[0] = lt[0] ? c : s[0];
}

template <int DP>
__device__ __forceinline__ float point_d2(const float (&q)[DP], const float4* p)
{
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < DP; k++) {
        const float4 v = p[k >> 2];
        const float c = (k & 3) == 0 ? v.x : (k & 3) == 1 ? v.y : (k & 3) == 2 ? v.z : v.w;
        const float t = __fsub_rn(q[k], c);
        acc = __fadd_rn(acc, __fmul_rn(t, t));
    }
    return acc;
}

template <int DP>
__device__ __forceinline__ int point_id(const float4* p)
{
    const float4 v = p[DP >> 2];
    const float c = (DP & 3) == 0 ? v.x : (DP & 3) == 1 ? v.y : (DP & 3) == 2 ? v.z : v.w;
    return __float_as_int(c);
}

template <int DP, int KC>
__global__ void __launch_bounds__(128) k_knn(KnnArgs a)
{
    constexpr int NV = (DP + 1 + 3) / 4;
    constexpr int NS = (4 + 2 * DP + 3) / 4;
    __shared__ float4 stage[4][32 * NV];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long g0 = ((long long)blockIdx.x * 4 + warp) * 32;
    if (g0 >= a.m) return;
    const long long pos = g0 + lane;
    const bool valid = pos < a.m;
    int qi = 0;
    if (valid) qi = a.perm ? a.perm[pos] : (int)pos;
    float q[DP];
    bool finite = true;
#pragma unroll
    for (int k = 0; k < DP; k++) {
        q[k] = (valid && k < a.d) ? a.queries[(long long)qi * a.d + k] : 0.0f;
        finite &= (__float_as_uint(q[k]) & 0x7f800000u) != 0x7f800000u;
    }
    if (!finite) atomicOr(a.err, kErrNonfinite);
    unsigned long long s[KC];
#pragma unroll
    for (int i = 0; i < KC; i++) s[i] = (valid && i >= KC - a.k) ? kKeyEmpty : 0ull;

    int stack[kMaxDepth + 4];
    int sp = 0;
    stack[sp++] = 0;
    float4* st = stage[warp];
    // A valid tree is visited in at most 2 * num_nodes pops; the cap only
    // guarantees termination (with an error flag) should a node table be corrupt.
    long long budget = 2LL * a.num_nodes + 8;
    while (sp > 0) {
        if (--budget < 0 || (unsigned)stack[sp - 1] >= (unsigned)a.num_nodes) {
            if (lane == 0) atomicOr(a.err, kErrInternal);
            break;
        }
        const int node = stack[--sp];
        const float4* rec = a.nodes + (long long)node * NS;
        float f[4 * NS];
#pragma unroll
        for (int r = 0; r < NS; r++) {
            const float4 v = __ldg(rec + r);
            f[4 * r] = v.x;
            f[4 * r + 1] = v.y;
            f[4 * r + 2] = v.z;
            f[4 * r + 3] = v.w;
        }
        float bnd = 0.0f;
#pragma unroll
        for (int k = 0; k < DP; k++) {
            const float lo = f[4 + k], hi = f[4 + DP + k];
            const float g = q[k] < lo ? __fsub_rn(lo, q[k]) : (q[k] > hi ? __fsub_rn(q[k], hi) : 0.0f);
            bnd = __fadd_rn(bnd, __fmul_rn(g, g));
        }
        const float kd = __uint_as_float((unsigned)(s[KC - 1] >> 32));
        const bool need = valid && !(bnd > kd);
        if (!__any_sync(kFull, need)) continue;
        const int h0 = __float_as_int(f[0]);
        const int h1 = __float_as_int(f[1]);
        const unsigned meta = __float_as_uint(f[3]);
        if (meta & kMetaLeaf) {
            if (h0 < 0 || h1 < 0 || (long long)h0 + h1 > a.npts) {
                if (lane == 0) atomicOr(a.err, kErrInternal);
                break;
            }
            for (int b0 = 0; b0 < h1; b0 += 32) {
                const int c = min(32, h1 - b0);
                __syncwarp();
                if (lane < c) {
                    const float4* src = a.pts + (long long)(h0 + b0 + lane) * NV;
#pragma unroll
                    for (int v = 0; v < NV; v++) st[lane * NV + v] = __ldg(src + v);
                }
                __syncwarp();
                const unsigned long long kth = s[KC - 1];
                unsigned mask = 0;
                for (int j = 0; j < c; j++) {
                    const float4* p = st + j * NV;
                    const float dd = point_d2<DP>(q, p);
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(dd) << 32) | (unsigned)point_id<DP>(p);
                    if (key < kth) mask |= 1u << j;
                }
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const float4* p = st + j * NV;
                    const float dd = point_d2<DP>(q, p);
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(dd) << 32) | (unsigned)point_id<DP>(p);
                    if (key < s[KC - 1]) topk_insert<KC>(s, key);
                }
            }
        } else {
            const int dim = (int)(meta & kMetaDimMask);
            const float sv = f[2];
            float qd = 0.0f;
#pragma unroll
            for (int k = 0; k < DP; k++)
                if (k == dim) qd = q[k];
            const unsigned bn = __ballot_sync(kFull, need);
            const unsigned br = __ballot_sync(kFull, need && qd >= sv);
            const bool right_near = 2 * __popc(br) >= __popc(bn);
            if (sp + 2 > kMaxDepth + 4) {
                if (lane == 0) atomicOr(a.err, kErrInternal);
                break;
            }
            stack[sp++] = h0 + (right_near ? 0 : 1);   // far child first
            stack[sp++] = h0 + (right_near ? 1 : 0);   // near child last
        }
    }
    if (valid) {
        int* oi = a.ids + (long long)qi * a.k;
        float* od = a.d2 + (long long)qi * a.k;
#pragma unroll
        for (int i = 0; i < KC; i++) {
            const int j = i - (KC - a.k);
            if (j >= 0) {
                oi[j] = (int)(unsigned)(s[i] & 0xffffffffull);
                od[j] = __uint_as_float((unsigned)(s[i] >> 32));
            }
        }
    }
}

}  // namespace panda
