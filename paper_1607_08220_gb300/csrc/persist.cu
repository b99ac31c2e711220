// persist.cu -- save a built tree to a file and load it back onto a device.
//
// The paper rebuilds trees every few steps and has no checkpoint; a saved tree
// lets a later run (or another process) query without rebuilding.  File
// layout, little-endian: an 8-byte magic, a header of int64 fields, the root
// box (2 x 16 floats), then the node table [node_slots][ns] float4 and the
// packed points [n][nv] float4 exactly as they sit in device memory.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace panda {
namespace {

constexpr char kMagic[8] = {'P', 'A', 'N', 'D', 'A', 'K', 'D', '1'};
constexpr int kFields = 12;   // n d dp bucket nv ns threshold node_slots num_nodes num_leaves depth node_cap

struct FileCloser {
    FILE* f;
    ~FileCloser()
    {
        if (f) fclose(f);
    }
};

}  // namespace
}  // namespace panda

using namespace panda;

extern "C" {

panda_status panda_tree_save(const panda_tree* t, const char* path)
{
    clear_error();
    if (!t || !path) {
        set_error("panda_tree_save: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    const size_t nb = (size_t)t->node_slots * t->ns * 16, pb = (size_t)t->n * t->nv * 16;
    std::vector<unsigned char> nodes(nb), pts(pb);
    PANDA_CUDA(cudaMemcpy(nodes.data(), t->nodes, nb, cudaMemcpyDeviceToHost), "panda_tree_save nodes");
    PANDA_CUDA(cudaMemcpy(pts.data(), t->points, pb, cudaMemcpyDeviceToHost), "panda_tree_save points");
    FileCloser fc{fopen(path, "wb")};
    if (!fc.f) {
        set_error("panda_tree_save: cannot open %s", path);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    const int64_t hdr[kFields] = {t->n, t->d, t->dp, t->bucket, t->nv, t->ns, t->threshold,
                                  t->node_slots, t->num_nodes, t->num_leaves, t->depth, t->node_slots};
    bool ok = fwrite(kMagic, 1, 8, fc.f) == 8 && fwrite(hdr, sizeof(int64_t), kFields, fc.f) == (size_t)kFields &&
              fwrite(t->root_lo, sizeof(float), 16, fc.f) == 16 && fwrite(t->root_hi, sizeof(float), 16, fc.f) == 16 &&
              fwrite(nodes.data(), 1, nb, fc.f) == nb && fwrite(pts.data(), 1, pb, fc.f) == pb;
    ok = (fclose(fc.f) == 0) && ok;
    fc.f = nullptr;
    if (!ok) {
        set_error("panda_tree_save: write to %s failed", path);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    return PANDA_OK;
}

panda_status panda_tree_load(const char* path, panda_tree** out)
{
    clear_error();
    if (!path || !out) {
        set_error("panda_tree_load: invalid argument");
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    *out = nullptr;
    FileCloser fc{fopen(path, "rb")};
    if (!fc.f) {
        set_error("panda_tree_load: cannot open %s", path);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    char magic[8];
    int64_t hdr[kFields];
    float lo[16], hi[16];
    if (fread(magic, 1, 8, fc.f) != 8 || memcmp(magic, kMagic, 8) != 0 ||
        fread(hdr, sizeof(int64_t), kFields, fc.f) != (size_t)kFields || fread(lo, sizeof(float), 16, fc.f) != 16 ||
        fread(hi, sizeof(float), 16, fc.f) != 16) {
        set_error("panda_tree_load: %s is not a saved tree", path);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    const int64_t n = hdr[0], d = hdr[1], dp = hdr[2], bucket = hdr[3], nv = hdr[4], ns = hdr[5];
    const int64_t slots = hdr[7];
    // the layout must be one this library writes
    if (n < 1 || n >= (1LL << 31) || d < 1 || d > kMaxDim || dp != padded_dim((int)d) || bucket < 1 ||
        nv != point_float4s((int)dp) || ns != node_float4s((int)dp) || slots < 1 || slots > 4 * n + (1LL << 24)) {
        set_error("panda_tree_load: %s has an unsupported header", path);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    const size_t nb = (size_t)slots * ns * 16, pb = (size_t)n * nv * 16;
    std::vector<unsigned char> nodes(nb), pts(pb);
    if (fread(nodes.data(), 1, nb, fc.f) != nb || fread(pts.data(), 1, pb, fc.f) != pb) {
        set_error("panda_tree_load: %s is truncated", path);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    // the kernels write output rows by stored id and follow child indices: a
    // file whose ids are not a permutation of 0..n-1 or whose node headers
    // point outside the tables is refused before anything reaches the device
    {
        std::vector<unsigned char> seen((size_t)n, 0);
        const float* pf = reinterpret_cast<const float*>(pts.data());
        for (int64_t i = 0; i < n; i++) {
            int32_t id;
            memcpy(&id, pf + i * nv * 4 + dp, 4);
            if (id < 0 || id >= n || seen[(size_t)id]) {
                set_error("panda_tree_load: %s holds an invalid point id", path);
                return PANDA_ERR_INVALID_ARGUMENT;
            }
            seen[(size_t)id] = 1;
        }
        const int32_t* nf = reinterpret_cast<const int32_t*>(nodes.data());
        for (int64_t i = 0; i < slots; i++) {
            const int32_t* h = nf + i * ns * 4;
            const bool leaf = ((uint32_t)h[3] & kMetaLeaf) != 0;
            const bool ok = leaf ? (h[0] >= 0 && h[1] >= 0 && (int64_t)h[0] + h[1] <= n)
                                 : (h[0] >= 0 && (int64_t)h[0] + 1 < slots);
            if (!ok) {
                set_error("panda_tree_load: %s holds an invalid node record", path);
                return PANDA_ERR_INVALID_ARGUMENT;
            }
        }
    }
    panda_tree* t = new panda_tree();
    cudaGetDevice(&t->device);
    t->pooled = false;
    t->n = n;
    t->d = (int32_t)d;
    t->dp = (int32_t)dp;
    t->bucket = (int32_t)bucket;
    t->nv = (int32_t)nv;
    t->ns = (int32_t)ns;
    t->threshold = (int32_t)hdr[6];
    t->node_slots = slots;
    t->node_cap = slots;
    t->num_nodes = hdr[8];
    t->num_leaves = hdr[9];
    t->depth = (int32_t)hdr[10];
    memcpy(t->root_lo, lo, sizeof(lo));
    memcpy(t->root_hi, hi, sizeof(hi));
    cudaError_t e = cudaMalloc(&t->nodes, nb);
    if (e == cudaSuccess) e = cudaMalloc(&t->points, pb);
    if (e == cudaSuccess) e = cudaMemcpy(t->nodes, nodes.data(), nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->points, pts.data(), pb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        panda_free(t);
        return cuda_fail(e, "panda_tree_load");
    }
    *out = t;
    return PANDA_OK;
}

}  // extern "C"
