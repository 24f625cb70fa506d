// Instantiation of the row, split-path, apply and adjoint kernels for degree 3, arithmetic type float.
#include "launch.cuh"

namespace wq {
template cudaError_t launch_rows<3, float>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint<3, float>(int, int, const AdjArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint_u<3, float>(const AdjUArgs &, int, cudaStream_t);
template cudaError_t launch_u<3, float>(const UArgs &, int, cudaStream_t);
template cudaError_t launch_rows_ug<3, float>(bool, bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_ug<3, float>(bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_2d<3, float>(int, bool, const RowsArgs &, int, cudaStream_t);
}
