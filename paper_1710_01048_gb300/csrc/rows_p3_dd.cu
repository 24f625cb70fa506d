// Instantiation of the row and adjoint kernels for degree 3, double-float arithmetic.
#include "launch.cuh"

namespace wq {
template cudaError_t launch_rows<3, dd>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
template cudaError_t launch_adjoint<3, dd>(int, int, const AdjArgs &, int, cudaStream_t);
}
