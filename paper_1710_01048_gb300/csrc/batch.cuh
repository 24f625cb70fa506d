// Persistent kernels that assemble M and K of many independent 3D patches
// (uneven sizes, degree 2 or 3) with the split 3D path: batch_u_kernel runs
// the partial-contraction blocks of every patch of one degree,
// batch_rows_kernel the row chunks of those patches.  Each kernel's work is a
// list of segments, one per patch; segment s owns items [first_item,
// first_item + nitems), one item per block of the single-patch kernel, and a
// table gives each item's segment.  Each resident CTA takes the next item
// from a global counter (dynamic scheduling: items differ in cost by size
// and by boundary share), copies the segment's arguments into shared memory
// and runs the single-patch kernel's body; the counter's answer for its
// following item is fetched while it works on the current one.
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

// One degree's kernels are instantiated apart (batch_u_kernel<P, R>,
// batch_rows_kernel<P, R>), so each gets the single-patch kernel's register
// allocation and resident CTAs per SM; a batch of both degrees runs the two
// pairs of launches, one after the other or side by side on two streams.
template <int P, typename R> constexpr size_t batch_u_smem_bytes() { return ULayout<P, R>::BYTES; }

template <int P, typename R> constexpr size_t batch_rows_smem_bytes() {
  return RowsLayoutUG<P, kUGChunk, true, true, R>::BYTES;
}

template <int P, typename R>
__global__ void __launch_bounds__(256, WQ_U_MIN_BLOCKS)
    batch_u_kernel(const BatchUSeg *__restrict__ segs, const int *__restrict__ seg_of, int nitems, unsigned *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ UArgs sA;
  __shared__ int sItem, sSeg;
  if (threadIdx.x == 0) {
    const int item = (int)atomicAdd(counter, 1u);
    sItem = item;
    sSeg = item < nitems ? seg_of[item] : 0;
  }
  for (;;) {
    __syncthreads();  // sItem, sSeg set; the previous item is done with shared memory
    const int item = sItem;
    if (item >= nitems) return;
    const BatchUSeg &S = segs[sSeg];
    for (int i = threadIdx.x; i < (int)(sizeof(UArgs) / sizeof(int)); i += blockDim.x)
      reinterpret_cast<int *>(&sA)[i] = reinterpret_cast<const int *>(&S.a)[i];
    const int bid = item - S.first_item;
    unsigned next = 0;
    if (threadIdx.x == 0) next = atomicAdd(counter, 1u);  // the next item's fetch overlaps this one
    __syncthreads();
    u_block<P, R>(sA, bid, smem_raw);
    if (threadIdx.x == 0) {
      sItem = (int)next;
      sSeg = (int)next < nitems ? seg_of[next] : 0;
    }
  }
}

template <int P, typename R>
__global__ void __launch_bounds__(32 * kRowsWarps, rows_min_blocks<R>())
    batch_rows_kernel(const BatchSeg *__restrict__ segs, const int *__restrict__ seg_of, int nitems, unsigned *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RowsArgs sA;
  __shared__ int sItem, sSeg;
  if (threadIdx.x == 0) {
    const int item = (int)atomicAdd(counter, 1u);
    sItem = item;
    sSeg = item < nitems ? seg_of[item] : 0;
  }
  for (;;) {
    __syncthreads();
    const int item = sItem;
    if (item >= nitems) return;
    const BatchSeg &S = segs[sSeg];
    for (int i = threadIdx.x; i < (int)(sizeof(RowsArgs) / sizeof(int)); i += blockDim.x)
      reinterpret_cast<int *>(&sA)[i] = reinterpret_cast<const int *>(&S.a)[i];
    const int bid = item - S.first_item;
    unsigned next = 0;
    if (threadIdx.x == 0) next = atomicAdd(counter, 1u);
    __syncthreads();
    rows_ug_block<P, kUGChunk, true, true, R>(sA, bid, smem_raw);
    if (threadIdx.x == 0) {
      sItem = (int)next;
      sSeg = (int)next < nitems ? seg_of[next] : 0;
    }
  }
}

// One degree's share of a batch: its segments (items numbered from 0 within
// the share), the segment of each item, its two counters ([0] partial
// contractions, [1] rows) and the persistent grids.
struct BatchShare {
  const BatchUSeg *usegs;
  const BatchSeg *segs;
  const int *useg_of, *seg_of;
  int nuseg, nuitems, nseg, nitems;
  unsigned *counters;
  int ugrid, grid;
};

// Sets the kernels' shared-memory limits (once per process and type) and
// returns their resident CTAs per SM, [0] for degree 2 and [1] for degree 3.
template <typename R> cudaError_t batch_prepare(int u_ctas_per_sm[2], int rows_ctas_per_sm[2]) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(batch_u_kernel<2, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batch_u_smem_bytes<2, R>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batch_u_kernel<3, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)batch_u_smem_bytes<3, R>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batch_rows_kernel<2, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)batch_rows_smem_bytes<2, R>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batch_rows_kernel<3, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)batch_rows_smem_bytes<3, R>());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&u_ctas_per_sm[0], batch_u_kernel<2, R>, 256,
                                                                batch_u_smem_bytes<2, R>());
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&u_ctas_per_sm[1], batch_u_kernel<3, R>, 256,
                                                      batch_u_smem_bytes<3, R>());
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rows_ctas_per_sm[0], batch_rows_kernel<2, R>,
                                                      32 * kRowsWarps, batch_rows_smem_bytes<2, R>());
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rows_ctas_per_sm[1], batch_rows_kernel<3, R>,
                                                      32 * kRowsWarps, batch_rows_smem_bytes<3, R>());
  return e;
}

// The partial-contraction launch, then the row launch, of degree p's share on s.
template <typename R> cudaError_t launch_batch_share(int p, const BatchShare &S, cudaStream_t s) {
  if (S.nuitems > 0 && S.ugrid > 0) {
    if (p == 2)
      batch_u_kernel<2, R><<<S.ugrid, 256, batch_u_smem_bytes<2, R>(), s>>>(S.usegs, S.useg_of, S.nuitems, S.counters);
    else
      batch_u_kernel<3, R><<<S.ugrid, 256, batch_u_smem_bytes<3, R>(), s>>>(S.usegs, S.useg_of, S.nuitems, S.counters);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (S.nitems > 0 && S.grid > 0) {
    if (p == 2)
      batch_rows_kernel<2, R><<<S.grid, 32 * kRowsWarps, batch_rows_smem_bytes<2, R>(), s>>>(S.segs, S.seg_of,
                                                                                            S.nitems, S.counters + 1);
    else
      batch_rows_kernel<3, R><<<S.grid, 32 * kRowsWarps, batch_rows_smem_bytes<3, R>(), s>>>(S.segs, S.seg_of,
                                                                                            S.nitems, S.counters + 1);
  }
  return cudaGetLastError();
}

extern template cudaError_t batch_prepare<double>(int *, int *);
extern template cudaError_t batch_prepare<float>(int *, int *);
extern template cudaError_t batch_prepare<dd>(int *, int *);
extern template cudaError_t launch_batch_share<double>(int, const BatchShare &, cudaStream_t);
extern template cudaError_t launch_batch_share<float>(int, const BatchShare &, cudaStream_t);
extern template cudaError_t launch_batch_share<dd>(int, const BatchShare &, cudaStream_t);

}  // namespace wq
