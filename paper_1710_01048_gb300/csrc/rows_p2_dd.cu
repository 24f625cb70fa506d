// Instantiation of the row, split-path, apply and adjoint kernels for degree 2, double-float arithmetic.
#include "launch.cuh"

namespace wq {
template cudaError_t launch_rows<2, dd>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint<2, dd>(int, int, const AdjArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint_u<2, dd>(const AdjUArgs &, int, cudaStream_t);
template cudaError_t launch_u<2, dd>(const UArgs &, int, cudaStream_t);
template cudaError_t launch_rows_ug<2, dd>(bool, bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_ug<2, dd>(bool, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_apply_2d<2, dd>(int, bool, const RowsArgs &, int, cudaStream_t);
}
