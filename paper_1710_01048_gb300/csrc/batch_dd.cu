// Instantiation of the persistent batch kernels, double-float arithmetic.
#include "batch.cuh"

namespace wq {
template cudaError_t batch_prepare<dd>(int *, int *);
template cudaError_t launch_batch<dd>(const BatchUSeg *, int, int, const BatchSeg *, int, int, unsigned *, int, int,
                                      cudaStream_t);
}
