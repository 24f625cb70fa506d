// Dispatch from runtime (dimension, terms, line class) to the row-kernel
// instantiations.  Interior lines (inner-direction rules with P+1 points)
// run chunks of up to interior_chunk(P, sizeof(R)) rows; boundary lines (up to P(P+1)
// points per inner direction) chunks of up to kBoundaryChunk rows.  Each CTA
// has (2P+1) threads per row of its chunk.
#pragma once

#include "adjoint.cuh"
#include "adjoint_u.cuh"
#include "assemble.cuh"
#include "ukernel.cuh"

namespace wq {

#ifndef WQ_INTERIOR_CHUNK
#define WQ_INTERIOR_CHUNK 24
#endif
#ifndef WQ_INTERIOR_CHUNK_P3_8B
#define WQ_INTERIOR_CHUNK_P3_8B 20
#endif
#ifndef WQ_BOUNDARY_CHUNK
#define WQ_BOUNDARY_CHUNK 16
#endif
// Interior-line chunk length by degree and arithmetic element size: degree 3
// in double or double-float keeps its shared memory small enough for three
// resident CTAs per SM.
constexpr int interior_chunk(int p, int elem_bytes) {
  return (p == 3 && elem_bytes == 8) ? WQ_INTERIOR_CHUNK_P3_8B : WQ_INTERIOR_CHUNK;
}
constexpr int kInteriorChunkMax =
    WQ_INTERIOR_CHUNK > WQ_INTERIOR_CHUNK_P3_8B ? WQ_INTERIOR_CHUNK : WQ_INTERIOR_CHUNK_P3_8B;
constexpr int kBoundaryChunk = WQ_BOUNDARY_CHUNK;
constexpr int kGeneralChunk = 8;  // the comparison rules (kernel class 2)

// Upper bound on the x1 points of one chunk's rows that the kernel's shared
// memory holds (checked by the host against the actual tables).
constexpr int chunk_points_bound(int p, int tmax) { return tmax * (p + 1) + p * (p + 1) * (p - 1); }
constexpr int chunk_points_bound_general(int p, int tmax) { return tmax * (p + 1) * (p + 1); }

template <int P, int D, int LM, int TMAX, bool DO_M, bool DO_K, typename R>
cudaError_t launch_one(const RowsArgs &a, int nblocks, cudaStream_t s) {
  using L = RowsLayout<P, D, LM, TMAX, DO_M, DO_K, R>;
  static_assert(L::MAXPTS1 == (L::GENERAL ? chunk_points_bound_general(P, TMAX) : chunk_points_bound(P, TMAX)),
                "chunk bound");
  auto kern = rows_kernel<P, D, LM, TMAX, DO_M, DO_K, R>;
  static bool configured = false;  // one attribute call per instantiation and process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  kern<<<nblocks, L::NT, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int P, int D, bool DO_M, bool DO_K, typename R>
cudaError_t launch_class(int cls, const RowsArgs &a, int nblocks, cudaStream_t s) {
  if (cls == 0) return launch_one<P, D, P + 1, interior_chunk(P, sizeof(R)), DO_M, DO_K, R>(a, nblocks, s);
  if (cls == 1) return launch_one<P, D, P *(P + 1), kBoundaryChunk, DO_M, DO_K, R>(a, nblocks, s);
  // class 2, the comparison rules: FP64 only
  if constexpr (std::is_same<R, double>::value)
    return launch_one<P, D, (P + 1) * (P + 1), kGeneralChunk, DO_M, DO_K, R>(a, nblocks, s);
  return cudaErrorNotSupported;
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

// Matrix-free apply on 2D meshes: the fused row kernel in APPLY mode (M and,
// if do_k, K), per line class.
template <int P, int LM, int TMAX, bool DO_K, typename R>
cudaError_t launch_apply_fused_one(const RowsArgs &a, int nblocks, cudaStream_t s) {
  using L = RowsLayout<P, 2, LM, TMAX, true, DO_K, R, true>;
  auto kern = rows_kernel<P, 2, LM, TMAX, true, DO_K, R, true>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  kern<<<nblocks, L::NT, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int P, typename R>
cudaError_t launch_apply_2d(int cls, bool do_k, const RowsArgs &a, int nblocks, cudaStream_t s) {
  constexpr int TI = interior_chunk(P, sizeof(R));
  if (cls == 0)
    return do_k ? launch_apply_fused_one<P, P + 1, TI, true, R>(a, nblocks, s)
                : launch_apply_fused_one<P, P + 1, TI, false, R>(a, nblocks, s);
  return do_k ? launch_apply_fused_one<P, P *(P + 1), kBoundaryChunk, true, R>(a, nblocks, s)
              : launch_apply_fused_one<P, P *(P + 1), kBoundaryChunk, false, R>(a, nblocks, s);
}

template <int P, typename R>
cudaError_t launch_adjoint(int D, int cls, const AdjArgs &a, int nblocks, cudaStream_t s) {
  if (D == 2) {
    if (cls == 0) return launch_adjoint_one<P, 2, P + 1, interior_chunk(P, sizeof(R)), R>(a, nblocks, s);
    return launch_adjoint_one<P, 2, P *(P + 1), kBoundaryChunk, R>(a, nblocks, s);
  }
  // 3D: the x1 stage per chunk into Ubar slots; launch_adjoint_u does the rest
  if (cls == 0) return launch_adjoint_x1_one<P, interior_chunk(P, sizeof(R)), R>(a, nblocks, s);
  return launch_adjoint_x1_one<P, kBoundaryChunk, R>(a, nblocks, s);
}

extern template cudaError_t launch_u<2, double>(const UArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows_ug<2, double>(bool, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_ug<2, double>(bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_2d<2, double>(int, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_u<2, float>(const UArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows_ug<2, float>(bool, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_ug<2, float>(bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_2d<2, float>(int, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_u<2, dd>(const UArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows_ug<2, dd>(bool, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_ug<2, dd>(bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_2d<2, dd>(int, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_u<3, double>(const UArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows_ug<3, double>(bool, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_ug<3, double>(bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_2d<3, double>(int, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_u<3, float>(const UArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows_ug<3, float>(bool, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_ug<3, float>(bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_2d<3, float>(int, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_u<3, dd>(const UArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows_ug<3, dd>(bool, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_ug<3, dd>(bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_apply_2d<3, dd>(int, bool, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<2, double>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<3, double>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<2, float>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<3, float>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<2, dd>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_rows<3, dd>(int, bool, bool, int, const RowsArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint<2, double>(int, int, const AdjArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint<3, double>(int, int, const AdjArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint<2, float>(int, int, const AdjArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint<3, float>(int, int, const AdjArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint<2, dd>(int, int, const AdjArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint<3, dd>(int, int, const AdjArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint_u<2, double>(const AdjUArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint_u<3, double>(const AdjUArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint_u<2, float>(const AdjUArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint_u<3, float>(const AdjUArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint_u<2, dd>(const AdjUArgs &, int, cudaStream_t);
extern template cudaError_t launch_adjoint_u<3, dd>(const AdjUArgs &, int, cudaStream_t);

}  // namespace wq
