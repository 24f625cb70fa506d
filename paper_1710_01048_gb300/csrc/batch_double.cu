// Instantiation of the persistent batch kernel, FP64 arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<double>(int *);
template cudaError_t launch_batch<double>(const BatchSeg *, int, int, unsigned *, int, cudaStream_t);
}
