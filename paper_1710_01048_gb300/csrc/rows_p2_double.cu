// Instantiation of the row, split-path, apply and adjoint kernels for degree 2, arithmetic type double.
#include "launch.cuh"

namespace wq {
template cudaError_t launch_rows<2, double>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint<2, double>(int, int, const AdjArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint_u<2, double>(const AdjUArgs &, int, cudaStream_t);
template cudaError_t launch_u<2, double>(const UArgs &, int, cudaStream_t);
template cudaError_t launch_rows_ug<2, double>(bool, bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_ug<2, double>(bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_2d<2, double>(int, bool, const RowsArgs &, int, cudaStream_t);
}
