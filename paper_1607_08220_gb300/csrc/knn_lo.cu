// knn_lo.cu -- traversal kernel instances for padded widths 2, 3 and 4.
#include "knn_launch.cuh"

namespace panda {
template panda_status launch_knn_dp<2>(const KnnArgs&, cudaStream_t);
template panda_status launch_knn_dp<3>(const KnnArgs&, cudaStream_t);
template panda_status launch_knn_dp<4>(const KnnArgs&, cudaStream_t);
panda_status configure_knn_lo()
{
    panda_status st;
    if ((st = configure_knn<2>()) != PANDA_OK) return st;
    if ((st = configure_knn<3>()) != PANDA_OK) return st;
    if ((st = configure_knn<4>()) != PANDA_OK) return st;
    return PANDA_OK;
}
}  // namespace panda
