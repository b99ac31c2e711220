// order.cuh -- query ordering by a spatial key (one counting sort): the
// arguments of the key kernel and the declarations of the ordering kernels
// defined in query.cu.
#pragma once

#include "common.cuh"

namespace panda {

struct OrderArgs {
    const float4* nodes;
    long long num_nodes;
    const float* queries;
    long long m;
    int d, ns, shift, mode;
    float lo[kMaxDim], inv[kMaxDim];
    int bits;
    unsigned* keys;
    int* hist;
    // several query sets, each against its own root of one forest (null: one tree):
    // query rows [qset_off[s], qset_off[s+1]) belong to set s, whose root is node s,
    // whose points start at set_poff[s] and whose bins start at set_bin[s]
    const int* qset_off;
    const int* set_poff;
    const int* set_bin;
    int nsets;
};

// key of every query (leaf bucket or Morton code >> shift) and its histogram
__global__ void k_order_keys(OrderArgs a);
// exclusive scan of hist[0..nb) in blocks of 4096 (block sums to bsum)
__global__ void k_scan_blocks(int* hist, int nb, int* bsum);
// exclusive scan of the block sums
__global__ void k_scan_sums(int* bsum, int nblocks);
// perm[position] = query row, grouped by key
__global__ void k_order_scatter(const unsigned* keys, long long m, int* cursor, const int* bsum, int* perm);

}  // namespace panda
