// Instantiation of the persistent batch kernels, double-float arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<dd>(int *, int *);
template cudaError_t launch_batch_share<dd>(int, const BatchShare &, cudaStream_t);
}
