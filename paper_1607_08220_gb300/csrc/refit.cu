// refit.cu -- moves the points of a built tree to new positions and makes every
// node box tight again, keeping the tree's structure.
//
// Particles move after every simulation step; the paper rebuilds the tree
// every few steps and trades build time against tree quality (Sec. II).  A
// refit is the cheap step in between: every point keeps its leaf, every leaf
// gets the exact box of its points' new coordinates and every inner node the
// union of its children's boxes.  Queries stay exact -- pruning needs only
// that a box contains its points -- and slow down as the split planes drift
// away from the points.
//
// Boxes go up the tree without waiting: each leaf's warp climbs, and at each
// parent the first of the two children to arrive stops while the second
// (whose atomic add sees the first's arrival) writes the union and climbs on.
#include <string.h>

#include "common.cuh"
#include "runtime.h"

namespace panda {
namespace {

__global__ void k_refit_check(const float* pts, long long count, unsigned* err)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count && (__float_as_uint(pts[i]) & 0x7f800000u) == 0x7f800000u) atomicOr(err, kErrNonfinite);
}

// Packed slot i takes the new coordinates of the point it holds (its id).
__global__ void k_refit_points(float4* packed, long long n, int d, int dp, int nv, const float* pts,
                               unsigned* err)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float* rec = reinterpret_cast<float*>(packed + i * nv);
    const long long id = __float_as_int(rec[dp]);
    if (id < 0 || id >= n) {
        atomicOr(err, kErrInternal);
        return;
    }
    for (int k = 0; k < d; k++) rec[k] = pts[id * d + k];
}

// Parent of every child of an inner node (holes have an all-zero header; no
// real inner node has child 0).
__global__ void k_refit_parents(const float4* nodes, long long slots, int ns, int* parent)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slots) return;
    const int4 h = reinterpret_cast<const int4*>(nodes + i * ns)[0];
    if (((unsigned)h.w & kMetaLeaf) || h.x <= 0 || h.x + 1 >= slots) return;
    parent[h.x] = (int)i;
    parent[h.x + 1] = (int)i;
}

// One warp per node slot: leaves compute their box, then climb.
__global__ void k_refit_boxes(float4* nodes, long long slots, int ns, const float4* packed, long long n, int nv,
                              int d, int dp, const int* parent, int* arrive, unsigned* err)
{
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= slots) return;
    float* rec = reinterpret_cast<float*>(nodes + w * ns);
    const int4 h = reinterpret_cast<const int4*>(rec)[0];
    if (!((unsigned)h.w & kMetaLeaf)) return;
    if (h.x < 0 || h.y < 0 || (long long)h.x + h.y > n) {
        if (lane == 0) atomicOr(err, kErrInternal);
        return;
    }
    for (int k = 0; k < d; k++) {
        float mn = INFINITY, mx = -INFINITY;
        for (int j = lane; j < h.y; j += 32) {
            const float x = reinterpret_cast<const float*>(packed + (long long)(h.x + j) * nv)[k];
            mn = fminf(mn, x);
            mx = fmaxf(mx, x);
        }
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0) {
            rec[4 + k] = mn;
            rec[4 + dp + k] = mx;
        }
    }
    if (lane != 0) return;
    long long node = w;
    for (int step = 0; step <= kMaxDepth + 1; step++) {
        const int p = parent[node];
        if (p < 0) return;
        __threadfence();                          // this child's box before the arrival
        if (atomicAdd(&arrive[p], 1) == 0) return;  // the sibling finishes the parent
        __threadfence();                          // the sibling's box after its arrival
        float* pr = reinterpret_cast<float*>(nodes + (long long)p * ns);
        const int c = reinterpret_cast<const int*>(pr)[0];
        const float* r0 = reinterpret_cast<const float*>(nodes + (long long)c * ns);
        const float* r1 = reinterpret_cast<const float*>(nodes + (long long)(c + 1) * ns);
        for (int k = 0; k < d; k++) {
            pr[4 + k] = fminf(__ldcg(r0 + 4 + k), __ldcg(r1 + 4 + k));
            pr[4 + dp + k] = fmaxf(__ldcg(r0 + 4 + dp + k), __ldcg(r1 + 4 + dp + k));
        }
        // the split plane still separates the children (left box at or below
        // it, right box at or above it) or it no longer bounds the far child
        unsigned meta = reinterpret_cast<const unsigned*>(pr)[3];
        if (!(meta & kMetaIndex)) {
            const int dim = (int)(meta & kMetaDimMask);
            const float sv = pr[2];
            const bool sep = dim < d && __ldcg(r0 + 4 + dp + dim) <= sv && __ldcg(r1 + 4 + dim) >= sv;
            meta = sep ? (meta & ~kMetaCross) : (meta | kMetaCross);
            reinterpret_cast<unsigned*>(pr)[3] = meta;
        }
        node = p;
    }
    atomicOr(err, kErrInternal);   // deeper than any valid tree
}

}  // namespace
}  // namespace panda

using namespace panda;

extern "C" {

panda_status panda_refit(panda_tree* t, const float* points, void* stream)
{
    clear_error();
    if (!t || !points) {
        set_error("panda_refit: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (!is_device_ptr(points)) {
        set_error("panda_refit: points must be a device pointer");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // queries still in flight on other streams read the tree: refit starts after them
    wait_tree_uses(t, s);
    const long long slots = t->node_slots;
    void* scratch = nullptr;
    const size_t bytes = 16 + (size_t)slots * 2 * sizeof(int);
    panda_status st = ws_alloc(&scratch, bytes, s, "refit scratch");
    if (st != PANDA_OK) return st;
    unsigned* err = static_cast<unsigned*>(scratch);
    int* parent = reinterpret_cast<int*>(static_cast<char*>(scratch) + 16);
    int* arrive = parent + slots;
    unsigned herr = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, 16, s);
    // first make sure the new points are finite: nothing changes otherwise
    if (e == cudaSuccess) {
        const long long cnt = t->n * t->d;
        k_refit_check<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(points, cnt, err);
        st = note_launch("k_refit_check");
        if (st == PANDA_OK) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s);
        if (st == PANDA_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (st == PANDA_OK && e == cudaSuccess && herr) {
        ws_free(scratch, s);
        set_error("panda_refit: non-finite point coordinate");
        return PANDA_ERR_NONFINITE_INPUT;
    }
    if (st == PANDA_OK && e == cudaSuccess) e = cudaMemsetAsync(parent, 0xff, (size_t)slots * sizeof(int), s);
    if (st == PANDA_OK && e == cudaSuccess) e = cudaMemsetAsync(arrive, 0, (size_t)slots * sizeof(int), s);
    if (st == PANDA_OK && e == cudaSuccess) {
        k_refit_points<<<(unsigned)((t->n + 255) / 256), 256, 0, s>>>(t->points, t->n, t->d, t->dp, t->nv, points,
                                                                       err);
        st = note_launch("k_refit_points");
        if (st == PANDA_OK) {
            k_refit_parents<<<(unsigned)((slots + 255) / 256), 256, 0, s>>>(t->nodes, slots, t->ns, parent);
            st = note_launch("k_refit_parents");
        }
        if (st == PANDA_OK) {
            k_refit_boxes<<<(unsigned)((slots * 32 + 255) / 256), 256, 0, s>>>(t->nodes, slots, t->ns, t->points,
                                                                               t->n, t->nv, t->d, t->dp, parent,
                                                                               arrive, err);
            st = note_launch("k_refit_boxes");
        }
        // the root box (host copy: the Morton ordering's frame)
        float root[4 * 16];
        if (st == PANDA_OK)
            e = cudaMemcpyAsync(root, t->nodes, (size_t)t->ns * 16, cudaMemcpyDeviceToHost, s);
        if (st == PANDA_OK && e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s);
        if (st == PANDA_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (st == PANDA_OK && e == cudaSuccess) {
            for (int k = 0; k < t->d; k++) {
                t->root_lo[k] = root[4 + k];
                t->root_hi[k] = root[4 + t->dp + k];
            }
        }
    }
    ws_free(scratch, s);
    if (st != PANDA_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "panda_refit");
    if (herr) {
        set_error("panda_refit: internal consistency check failed (0x%x)", herr);
        return PANDA_ERR_CUDA;
    }
    return PANDA_OK;
}

}  // extern "C"
