// Instantiation of the persistent batch kernels, FP32 (mixed mode) arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<float>(int *, int *);
template cudaError_t launch_batch_share<float>(int, const BatchShare &, cudaStream_t);
}
