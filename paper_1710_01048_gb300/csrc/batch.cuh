// Persistent kernel that assembles M and K of many independent 3D patches
// (uneven sizes, degree 2 or 3) in one launch.  The work is a list of
// segments, one per (patch, line class) with lines; segment s owns work items
// [first_item, first_item + nitems), one item per chunk of a line of rows,
// exactly the CTA work of rows_kernel.  Each resident CTA takes the next item
// from a global counter (dynamic scheduling: items differ in cost by degree,
// line class and chunk length), copies the segment's arguments into shared
// memory and runs the row kernel's body for that degree and class.
#pragma once

#include "launch.cuh"

namespace wq {

struct BatchSeg {
  RowsArgs a;            // the patch's tables, outputs and chunking for this class
  int p, cls;            // degree, line class (0 interior, 1 boundary)
  int first_item, nitems;
};

// Dynamic shared memory the batch kernel needs: the largest of the four bodies.
template <typename R> constexpr size_t batch_smem_bytes() {
  constexpr size_t a = RowsLayout<2, 3, 3, interior_chunk(2, sizeof(R)), true, true, R>::BYTES;
  constexpr size_t b = RowsLayout<2, 3, 6, kBoundaryChunk, true, true, R>::BYTES;
  constexpr size_t c = RowsLayout<3, 3, 4, interior_chunk(3, sizeof(R)), true, true, R>::BYTES;
  constexpr size_t d = RowsLayout<3, 3, 12, kBoundaryChunk, true, true, R>::BYTES;
  constexpr size_t ab = a > b ? a : b, cd = c > d ? c : d;
  return ab > cd ? ab : cd;
}

// The batch kernel holds four bodies in one register allocation: it asks for
// one resident CTA per SM fewer than the single-class kernels so that the
// union does not spill.
template <typename R> constexpr int batch_min_blocks() { return sizeof(R) == 4 ? 3 : 2; }

template <typename R>
__global__ void __launch_bounds__(32 * kRowsWarps, batch_min_blocks<R>())
    batch_rows_kernel(const BatchSeg *__restrict__ segs, int nseg, int nitems, unsigned *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RowsArgs sA;
  __shared__ int sItem, sSeg;
  for (;;) {
    __syncthreads();  // the previous item is done with shared memory
    if (threadIdx.x == 0) {
      const int item = (int)atomicAdd(counter, 1u);
      int seg = 0;
      if (item < nitems) {
        int lo = 0, hi = nseg - 1;  // the last segment with first_item <= item
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (segs[mid].first_item <= item) lo = mid; else hi = mid - 1;
        }
        seg = lo;
      }
      sItem = item;
      sSeg = seg;
    }
    __syncthreads();
    const int item = sItem;
    if (item >= nitems) return;
    const BatchSeg &S = segs[sSeg];
    for (int i = threadIdx.x; i < (int)(sizeof(RowsArgs) / sizeof(int)); i += blockDim.x)
      reinterpret_cast<int *>(&sA)[i] = reinterpret_cast<const int *>(&S.a)[i];
    const int p = S.p, cls = S.cls, bid = item - S.first_item;
    __syncthreads();
    if (p == 2) {
      if (cls == 0) rows_block<2, 3, 3, interior_chunk(2, sizeof(R)), true, true, R>(sA, bid, smem_raw);
      else rows_block<2, 3, 6, kBoundaryChunk, true, true, R>(sA, bid, smem_raw);
    } else {
      if (cls == 0) rows_block<3, 3, 4, interior_chunk(3, sizeof(R)), true, true, R>(sA, bid, smem_raw);
      else rows_block<3, 3, 12, kBoundaryChunk, true, true, R>(sA, bid, smem_raw);
    }
  }
}

// Sets the kernel's shared-memory limit (once per process and type) and
// returns its resident CTAs per SM.
template <typename R> cudaError_t batch_prepare(int *ctas_per_sm) {
  static bool configured = false;
  const int bytes = (int)batch_smem_bytes<R>();
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(batch_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, batch_rows_kernel<R>, 32 * kRowsWarps, bytes);
}

template <typename R>
cudaError_t launch_batch(const BatchSeg *segs, int nseg, int nitems, unsigned *counter, int grid, cudaStream_t s) {
  if (nitems <= 0 || grid <= 0) return cudaSuccess;
  batch_rows_kernel<R><<<grid, 32 * kRowsWarps, batch_smem_bytes<R>(), s>>>(segs, nseg, nitems, counter);
  return cudaGetLastError();
}

extern template cudaError_t batch_prepare<double>(int *);
extern template cudaError_t batch_prepare<float>(int *);
extern template cudaError_t batch_prepare<dd>(int *);
extern template cudaError_t launch_batch<double>(const BatchSeg *, int, int, unsigned *, int, cudaStream_t);
extern template cudaError_t launch_batch<float>(const BatchSeg *, int, int, unsigned *, int, cudaStream_t);
extern template cudaError_t launch_batch<dd>(const BatchSeg *, int, int, unsigned *, int, cudaStream_t);

}  // namespace wq
