// Instantiation of the row, split-path, apply and adjoint kernels for degree 3, arithmetic type double.
#include "launch.cuh"

namespace wq {
template cudaError_t launch_rows<3, double>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint<3, double>(int, int, const AdjArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint_u<3, double>(const AdjUArgs &, int, cudaStream_t);
template cudaError_t launch_u<3, double>(const UArgs &, int, cudaStream_t);
template cudaError_t launch_rows_ug<3, double>(bool, bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_ug<3, double>(bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_2d<3, double>(int, bool, const RowsArgs &, int, cudaStream_t);
}
