// predict.cu -- KNN prediction on top of a KNN result (Sec. I: the output for
// a query is a majority vote of its neighbours' labels for classification, or
// the average of their values for regression).
//
// One thread per query row.  Vote: the label with the largest count among the
// valid neighbours (0 <= id < n), the smallest label among equal counts, -1
// when there is none; counted by comparing every neighbour with every other
// (k <= 64).  Mean: FP32 running sum in rank order from +0, divided in FP32 by
// the number of valid neighbours; NaN when there is none.
#include <math.h>

#include "common.cuh"
#include "runtime.h"

namespace panda {
namespace {

__global__ void k_knn_vote(const int32_t* ids, long long m, int k, const int32_t* labels, long long n,
                           int32_t* out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const int32_t* row = ids + r * k;
    int best = -1, best_count = 0;
    for (int j = 0; j < k; j++) {
        const int id = row[j];
        if (id < 0 || id >= n) continue;
        const int lab = __ldg(labels + id);
        int c = 0;
        for (int i = 0; i < k; i++) {
            const int o = row[i];
            if (o >= 0 && o < n && __ldg(labels + o) == lab) c++;
        }
        if (c > best_count || (c == best_count && lab < best)) {
            best = lab;
            best_count = c;
        }
    }
    out[r] = best;
}

__global__ void k_knn_mean(const int32_t* ids, long long m, int k, const float* values, long long n, float* out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const int32_t* row = ids + r * k;
    float s = 0.0f;
    int c = 0;
    for (int j = 0; j < k; j++) {
        const int id = row[j];
        if (id < 0 || id >= n) continue;
        s = __fadd_rn(s, __ldg(values + id));
        c++;
    }
    out[r] = c ? __fdiv_rn(s, (float)c) : __int_as_float(0x7fc00000);
}

panda_status check_args(const void* ids, int64_t m, int32_t k, const void* table, int64_t n, const void* out,
                        const char* what)
{
    if (m < 0 || k < 1 || n < 0 || (m > 0 && (!ids || !table || !out))) {
        set_error("%s: invalid argument", what);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    if (k > kMaxK) {
        set_error("%s: k=%d above the maximum %d", what, k, kMaxK);
        return PANDA_ERR_UNSUPPORTED;
    }
    if (m > 0 && (!is_device_ptr(ids) || !is_device_ptr(table) || !is_device_ptr(out))) {
        set_error("%s: ids, table and output must be device pointers", what);
        return PANDA_ERR_INVALID_ARGUMENT;
    }
    return PANDA_OK;
}

}  // namespace
}  // namespace panda

using namespace panda;

extern "C" {

panda_status panda_knn_vote(const int32_t* ids, int64_t m, int32_t k, const int32_t* labels, int64_t n,
                            int32_t* out_labels, void* stream)
{
    clear_error();
    panda_status st = check_args(ids, m, k, labels, n, out_labels, "panda_knn_vote");
    if (st != PANDA_OK || m == 0) return st;
    k_knn_vote<<<(unsigned)((m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(ids, m, k, labels, n, out_labels);
    return note_launch("k_knn_vote");
}

panda_status panda_knn_mean(const int32_t* ids, int64_t m, int32_t k, const float* values, int64_t n,
                            float* out_values, void* stream)
{
    clear_error();
    panda_status st = check_args(ids, m, k, values, n, out_values, "panda_knn_mean");
    if (st != PANDA_OK || m == 0) return st;
    k_knn_mean<<<(unsigned)((m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(ids, m, k, values, n, out_values);
    return note_launch("k_knn_mean");
}

}  // extern "C"
