// Instantiation of the persistent batch kernels, FP64 arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<double>(int *, int *);
template cudaError_t launch_batch_share<double>(int, const BatchShare &, cudaStream_t);
}
