// Instantiation of the persistent batch kernel, FP32 (mixed mode) arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<float>(int *);
template cudaError_t launch_batch<float>(const BatchSeg *, int, int, unsigned *, int, cudaStream_t);
}
