// Geometry factor of a separable map folded into one point of the 1D tables
// (Eq. Mass, Eq. Stiffness with J diagonal):
//   mass kind:      V = W * |J_aa(x)| * B_{e+i}(x)
//   stiffness kind: V = W / |J_aa(x)| * B'_{e+i}(x)
// with J_aa(x) = sum_i g_{a,e+i} B'_{e+i}(x) (Eq. Gmap1).  Shared by the
// single-mesh and the batched fold kernels so that both give the same bits.
#pragma once

#include <cuda_runtime.h>

#include "wq_internal.h"

namespace wq {

// Writes point q's p+1 folded values in FP64, FP32 and (unless vdd is null)
// double-float form and returns the status bits it raises (geometry where
// J_aa <= 0, non-finite where J_aa is NaN or Inf).
__device__ __forceinline__ unsigned fold_point(int q, int np, int kind, const int *elem, const double *w,
                                               const double *t0, const double *t1, const double *g, double *v64,
                                               float *v32, float2 *vdd) {
  unsigned bits = 0;
  const int e = elem[q];
  double J = 0.0;
  for (int i = 0; i < np; i++) J = fma(g[e + i], t1[(size_t)q * np + i], J);
  if (!(J > 0.0)) bits |= isfinite(J) ? kBitGeometry : kBitNonFinite;
  const double aj = fabs(J);
  const double f = kind == WQ_KIND_MASS ? w[q] * aj : w[q] / aj;
  const double *T = kind == WQ_KIND_MASS ? t0 : t1;
  for (int i = 0; i < np; i++) {
    const double v = f * T[(size_t)q * np + i];
    const float vh = (float)v;
    v64[(size_t)q * np + i] = v;
    v32[(size_t)q * np + i] = vh;
    if (vdd) vdd[(size_t)q * np + i] = make_float2(vh, (float)(v - (double)vh));
  }
  return bits;
}

// Coefficient i of the cubic coefficient spline in the arithmetic type of
// the call (float for WQ_MIXED, a double-float pair for WQ_DF64; WQ_FP64
// reads the double array itself); returns the non-finite bit for NaN/Inf.
// Shared by the single-mesh and the batched preparation kernels.
__device__ __forceinline__ unsigned coef_point(const double *c, size_t i, int prec, float *c32, float2 *cdd) {
  const double v = c[i];
  if (prec == WQ_MIXED) {
    c32[i] = (float)v;
  } else if (prec == WQ_DF64) {
    const float h = (float)v;
    cdd[i] = make_float2(h, (float)(v - (double)h));
  }
  return isfinite(v) ? 0u : kBitNonFinite;
}

}  // namespace wq
