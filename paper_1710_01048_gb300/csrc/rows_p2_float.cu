// Instantiation of the row, split-path, apply and adjoint kernels for degree 2, arithmetic type float.
#include "launch.cuh"

namespace wq {
template cudaError_t launch_rows<2, float>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint<2, float>(int, int, const AdjArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint_u<2, float>(const AdjUArgs &, int, cudaStream_t);
template cudaError_t launch_u<2, float>(const UArgs &, int, cudaStream_t);
template cudaError_t launch_rows_ug<2, float>(bool, bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_ug<2, float>(bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_2d<2, float>(int, bool, const RowsArgs &, int, cudaStream_t);
}
