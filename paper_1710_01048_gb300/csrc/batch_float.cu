// Instantiation of the persistent batch kernels, FP32 (mixed mode) arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<float>(int *, int *);
template cudaError_t launch_batch<float>(const BatchUSeg *, int, int, const BatchSeg *, int, int, unsigned *, int, int,
                                      cudaStream_t);
}
