// Instantiation of the row kernels for degree 2, double-float arithmetic.
#include "launch.cuh"

namespace wq {
template cudaError_t launch_rows<2, dd>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
}
