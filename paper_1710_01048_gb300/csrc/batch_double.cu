// Instantiation of the persistent batch kernels, FP64 arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<double>(int *, int *);
template cudaError_t launch_batch<double>(const BatchUSeg *, int, int, const BatchSeg *, int, int, unsigned *, int, int,
                                      cudaStream_t);
}
