// knn_lo.cu -- traversal kernel instances for padded widths 2, 3 and 4.
#include "knn_launch.cuh"

namespace panda {
template panda_status launch_knn_dp<2>(const KnnArgs&, cudaStream_t);
template panda_status launch_knn_dp<3>(const KnnArgs&, cudaStream_t);
template panda_status launch_knn_dp<4>(const KnnArgs&, cudaStream_t);
}  // namespace panda
