// Dispatch from runtime (dimension, terms, line class) to the row-kernel
// instantiations.  Interior lines (rows whose inner-direction rules have
// P+1 points) run 8 warps per CTA and chunks of up to 16 rows; boundary lines
// (up to P(P+1) points per inner direction) run 4 warps and chunks of 8.
#pragma once

#include "assemble.cuh"

namespace wq {

constexpr int kInteriorWarps = 8, kInteriorChunk = 16;
constexpr int kBoundaryWarps = 4, kBoundaryChunk = 8;

template <int P, int D, int LM, int NW, int TMAX, bool DO_M, bool DO_K, typename R>
cudaError_t launch_one(const RowsArgs &a, int nblocks, cudaStream_t s) {
  using L = RowsLayout<P, D, LM, NW, TMAX, DO_M, DO_K, R>;
  auto kern = rows_kernel<P, D, LM, NW, TMAX, DO_M, DO_K, R>;
  static bool configured = false;  // one attribute call per instantiation and process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  kern<<<nblocks, NW * 32, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int P, int D, bool DO_M, bool DO_K, typename R>
cudaError_t launch_class(int cls, const RowsArgs &a, int nblocks, cudaStream_t s) {
  if (cls == 0) return launch_one<P, D, P + 1, kInteriorWarps, kInteriorChunk, DO_M, DO_K, R>(a, nblocks, s);
  return launch_one<P, D, P *(P + 1), kBoundaryWarps, kBoundaryChunk, DO_M, DO_K, R>(a, nblocks, s);
}

template <int P, typename R>
cudaError_t launch_rows(int D, bool do_m, bool do_k, int cls, const RowsArgs &a, int nblocks, cudaStream_t s) {
  if (D == 2) {
    if (do_m && do_k) return launch_class<P, 2, true, true, R>(cls, a, nblocks, s);
    if (do_m) return launch_class<P, 2, true, false, R>(cls, a, nblocks, s);
    return launch_class<P, 2, false, true, R>(cls, a, nblocks, s);
  }
  if (do_m && do_k) return launch_class<P, 3, true, true, R>(cls, a, nblocks, s);
  if (do_m) return launch_class<P, 3, true, false, R>(cls, a, nblocks, s);
  return launch_class<P, 3, false, true, R>(cls, a, nblocks, s);
}

// Maximum dynamic shared memory any instantiation of this (P, R) needs.
template <int P, typename R>
constexpr size_t max_rows_smem() {
  size_t m = 0;
  size_t v[] = {
      RowsLayout<P, 3, P *(P + 1), kBoundaryWarps, kBoundaryChunk, true, true, R>::BYTES,
      RowsLayout<P, 3, P + 1, kInteriorWarps, kInteriorChunk, true, true, R>::BYTES,
      RowsLayout<P, 2, P *(P + 1), kBoundaryWarps, kBoundaryChunk, true, true, R>::BYTES,
      RowsLayout<P, 2, P + 1, kInteriorWarps, kInteriorChunk, true, true, R>::BYTES};
  for (size_t x : v) m = x > m ? x : m;
  return m;
}

extern template cudaError_t launch_rows<2, double>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<3, double>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<2, float>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<3, float>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);

}  // namespace wq
