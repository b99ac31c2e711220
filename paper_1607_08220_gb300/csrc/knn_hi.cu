// knn_hi.cu -- traversal kernel instances for padded widths 8, 10 and 16.
#include "knn_launch.cuh"

namespace panda {
template panda_status launch_knn_dp<8>(const KnnArgs&, cudaStream_t);
template panda_status launch_knn_dp<10>(const KnnArgs&, cudaStream_t);
template panda_status launch_knn_dp<16>(const KnnArgs&, cudaStream_t);
panda_status configure_knn_hi()
{
    panda_status st;
    if ((st = configure_knn<8>()) != PANDA_OK) return st;
    if ((st = configure_knn<10>()) != PANDA_OK) return st;
    if ((st = configure_knn<16>()) != PANDA_OK) return st;
    return PANDA_OK;
}
}  // namespace panda
