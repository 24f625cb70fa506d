// Instantiation of the persistent batch kernel, double-float arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<dd>(int *);
template cudaError_t launch_batch<dd>(const BatchSeg *, int, int, unsigned *, int, cudaStream_t);
}
