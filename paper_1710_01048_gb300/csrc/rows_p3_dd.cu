// Instantiation of the row, split-path, apply and adjoint kernels for degree 3, double-float arithmetic.
#include "launch.cuh"

namespace wq {
template cudaError_t launch_rows<3, dd>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint<3, dd>(int, int, const AdjArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint_u<3, dd>(const AdjUArgs &, int, cudaStream_t);
template cudaError_t launch_u<3, dd>(const UArgs &, int, cudaStream_t);
template cudaError_t launch_rows_ug<3, dd>(bool, bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_ug<3, dd>(bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_2d<3, dd>(int, bool, const RowsArgs &, int, cudaStream_t);
}
