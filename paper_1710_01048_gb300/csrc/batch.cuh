// Persistent kernels that assemble M and K of many independent 3D patches
// (uneven sizes, degree 2 or 3) with the split 3D path: batch_u_kernel runs
// the partial-contraction blocks of every patch, batch_rows_kernel the row
// chunks of every patch.  Each kernel's work is a list of segments, one per
// patch; segment s owns items [first_item, first_item + nitems), one item per
// block of the single-patch kernel.  Each resident CTA takes the next item
// from a global counter (dynamic scheduling: items differ in cost by degree
// and size), copies the segment's arguments into shared memory and runs the
// single-patch kernel's body for that degree.
#pragma once

#include "launch.cuh"

namespace wq {

struct BatchUSeg {
  UArgs a;  // the patch's tables, coefficients and U buffer
  int p;
  int first_item, nitems;
};

struct BatchSeg {
  RowsArgs a;  // the patch's tables, U buffer, outputs and chunking
  int p;
  int first_item, nitems;
};

template <typename R> constexpr size_t batch_u_smem_bytes() {
  constexpr size_t a = ULayout<2, R>::BYTES, b = ULayout<3, R>::BYTES;
  return a > b ? a : b;
}

template <typename R> constexpr size_t batch_rows_smem_bytes() {
  constexpr size_t a = RowsLayoutUG<2, kUGChunk, true, true, R>::BYTES;
  constexpr size_t b = RowsLayoutUG<3, kUGChunk, true, true, R>::BYTES;
  return a > b ? a : b;
}

// The last segment whose first item is <= item (nseg >= 1).
template <typename S> __device__ __forceinline__ int batch_segment(const S *segs, int nseg, int item) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].first_item <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename R>
__global__ void __launch_bounds__(256) batch_u_kernel(const BatchUSeg *__restrict__ segs, int nseg, int nitems,
                                                      unsigned *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ UArgs sA;
  __shared__ int sItem, sSeg;
  for (;;) {
    __syncthreads();  // the previous item is done with shared memory
    if (threadIdx.x == 0) {
      const int item = (int)atomicAdd(counter, 1u);
      sItem = item;
      sSeg = item < nitems ? batch_segment(segs, nseg, item) : 0;
    }
    __syncthreads();
    const int item = sItem;
    if (item >= nitems) return;
    const BatchUSeg &S = segs[sSeg];
    for (int i = threadIdx.x; i < (int)(sizeof(UArgs) / sizeof(int)); i += blockDim.x)
      reinterpret_cast<int *>(&sA)[i] = reinterpret_cast<const int *>(&S.a)[i];
    const int p = S.p, bid = item - S.first_item;
    __syncthreads();
    if (p == 2) u_block<2, R>(sA, bid, smem_raw);
    else u_block<3, R>(sA, bid, smem_raw);
  }
}

// The row kernel holds two bodies in one register allocation; in
// double-float it asks for one resident CTA per SM fewer than the
// single-patch kernel so that the union does not spill.
template <typename R> constexpr int batch_rows_min_blocks() {
  return std::is_same<R, dd>::value ? rows_min_blocks<R>() - 1 : rows_min_blocks<R>();
}

template <typename R>
__global__ void __launch_bounds__(32 * kRowsWarps, batch_rows_min_blocks<R>())
    batch_rows_kernel(const BatchSeg *__restrict__ segs, int nseg, int nitems, unsigned *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RowsArgs sA;
  __shared__ int sItem, sSeg;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int item = (int)atomicAdd(counter, 1u);
      sItem = item;
      sSeg = item < nitems ? batch_segment(segs, nseg, item) : 0;
    }
    __syncthreads();
    const int item = sItem;
    if (item >= nitems) return;
    const BatchSeg &S = segs[sSeg];
    for (int i = threadIdx.x; i < (int)(sizeof(RowsArgs) / sizeof(int)); i += blockDim.x)
      reinterpret_cast<int *>(&sA)[i] = reinterpret_cast<const int *>(&S.a)[i];
    const int p = S.p, bid = item - S.first_item;
    __syncthreads();
    if (p == 2) rows_ug_block<2, kUGChunk, true, true, R>(sA, bid, smem_raw);
    else rows_ug_block<3, kUGChunk, true, true, R>(sA, bid, smem_raw);
  }
}

// Sets the kernels' shared-memory limits (once per process and type) and
// returns their resident CTAs per SM.
template <typename R> cudaError_t batch_prepare(int *u_ctas_per_sm, int *rows_ctas_per_sm) {
  static bool configured = false;
  const int ub = (int)batch_u_smem_bytes<R>(), rb = (int)batch_rows_smem_bytes<R>();
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(batch_u_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, ub);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(batch_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, rb);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(u_ctas_per_sm, batch_u_kernel<R>, 256, ub);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(rows_ctas_per_sm, batch_rows_kernel<R>, 32 * kRowsWarps, rb);
}

// counters[0] feeds the partial-contraction kernel, counters[1] the row kernel.
template <typename R>
cudaError_t launch_batch(const BatchUSeg *usegs, int nuseg, int nuitems, const BatchSeg *segs, int nseg, int nitems,
                         unsigned *counters, int ugrid, int grid, cudaStream_t s) {
  if (nuitems > 0 && ugrid > 0)
    batch_u_kernel<R><<<ugrid, 256, batch_u_smem_bytes<R>(), s>>>(usegs, nuseg, nuitems, counters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (nitems > 0 && grid > 0)
    batch_rows_kernel<R><<<grid, 32 * kRowsWarps, batch_rows_smem_bytes<R>(), s>>>(segs, nseg, nitems, counters + 1);
  return cudaGetLastError();
}

extern template cudaError_t batch_prepare<double>(int *, int *);
extern template cudaError_t batch_prepare<float>(int *, int *);
extern template cudaError_t batch_prepare<dd>(int *, int *);
extern template cudaError_t launch_batch<double>(const BatchUSeg *, int, int, const BatchSeg *, int, int, unsigned *,
                                                 int, int, cudaStream_t);
extern template cudaError_t launch_batch<float>(const BatchUSeg *, int, int, const BatchSeg *, int, int, unsigned *,
                                                int, int, cudaStream_t);
extern template cudaError_t launch_batch<dd>(const BatchUSeg *, int, int, const BatchSeg *, int, int, unsigned *, int,
                                             int, cudaStream_t);

}  // namespace wq
