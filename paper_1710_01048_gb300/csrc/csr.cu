// Band -> CSR conversion.  In the band layout the valid entries of a row
// (columns inside the mesh) already appear in increasing column order, and a
// row's valid count factors over the directions,
//   cnt(r) = prod_a cnt_a(r_a),  cnt_a(r) = min(n_a-1, r+p) - max(0, r-p) + 1,
// so the row pointer has the closed form
//   ptr(r) = S3(r3) P2 P1 + cnt3(r3) S2(r2) P1 + cnt3(r3) cnt2(r2) S1(r1)
// with S_a(r) = sum_{r' < r} cnt_a(r') and P_a = S_a(n_a): no scan is needed,
// and one thread per band entry writes its value and column directly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "wq_internal.h"

namespace {

struct CsrDims {
  long long n[3];
  int p, dim, band, nb;
};

__host__ __device__ __forceinline__ long long cnt_dir(long long r, long long n, int p) {
  const long long hi = r + p < n - 1 ? r + p : n - 1;
  const long long lo = r - p > 0 ? r - p : 0;
  return hi - lo + 1;
}

// S(r) = sum_{r' < r} cnt(r'): every row contributes 2p+1 minus the columns
// cut off at either end (p - r' at the start for r' < p, and symmetrically
// at the end).
__host__ __device__ __forceinline__ long long prefix_dir(long long r, long long n, int p) {
  long long s = r * (2 * p + 1);
  const long long k0 = r < p ? r : p;  // rows r' < min(r, p) lose p - r' columns at the start
  s -= k0 * p - k0 * (k0 - 1) / 2;
  // rows r' in [max(n - p, 0), r) lose r' + p - (n - 1) columns at the end
  const long long e0 = n - p > 0 ? n - p : 0;
  if (r > e0) {
    const long long a = e0 + p - (n - 1), m = r - e0;  // losses a, a+1, ..., a+m-1
    s -= m * a + m * (m - 1) / 2;
  }
  return s;
}

__host__ __device__ __forceinline__ long long row_ptr(long long r, const CsrDims &D) {
  long long rr[3] = {0, 0, 0};
  long long t = r;
  for (int a = 0; a < D.dim; a++) {
    rr[a] = t % D.n[a];
    t /= D.n[a];
  }
  long long ptr = 0, inner = 1;
  // ptr = sum over a of (prod_{b > a} cnt_b(r_b)) * S_a(r_a) * prod_{b < a} P_b
  long long outer_cnt = 1;
  for (int a = D.dim - 1; a >= 0; a--) {
    inner = 1;
    for (int b = 0; b < a; b++) inner *= prefix_dir(D.n[b], D.n[b], D.p);
    ptr += outer_cnt * prefix_dir(rr[a], D.n[a], D.p) * inner;
    outer_cnt *= cnt_dir(rr[a], D.n[a], D.p);
  }
  return ptr;
}

__host__ __device__ __forceinline__ long long row_cnt(long long r, const CsrDims &D) {
  long long c = 1;
  for (int a = 0; a < D.dim; a++) {
    c *= cnt_dir(r % D.n[a], D.n[a], D.p);
    r /= D.n[a];
  }
  return c;
}

template <typename T>
__global__ void band_to_csr_kernel(const CsrDims D, const T *__restrict__ band, long long row_begin,
                                   long long row_end, long long base_ptr, int64_t *__restrict__ rowptr,
                                   int32_t *__restrict__ col, T *__restrict__ val) {
  const long long total = (row_end - row_begin) * (long long)D.band;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = row_begin + t / D.band;
    const int j = (int)(t % D.band);
    long long rr[3] = {0, 0, 0}, q = r;
    for (int a = 0; a < D.dim; a++) {
      rr[a] = q % D.n[a];
      q /= D.n[a];
    }
    // the entry's offsets d_a and its rank among the row's valid entries
    int jj = j;
    bool ok = true;
    long long rank = 0, stride = 1, colidx = 0, cstride = 1;
    for (int a = 0; a < D.dim; a++) {
      const int d = jj % D.nb - D.p;
      jj /= D.nb;
      const long long s = rr[a] + d;
      const long long dmin = rr[a] - D.p > 0 ? -(long long)D.p : -rr[a];
      ok = ok && s >= 0 && s < D.n[a];
      rank += (d - dmin) * stride;
      stride *= cnt_dir(rr[a], D.n[a], D.p);
      colidx += s * cstride;
      cstride *= D.n[a];
    }
    if (j == 0) {
      rowptr[r - row_begin] = row_ptr(r, D) - base_ptr;
      if (r == row_end - 1) rowptr[row_end - row_begin] = row_ptr(r, D) + stride - base_ptr;
    }
    if (ok) {
      const long long pos = row_ptr(r, D) - base_ptr + rank;
      col[pos] = (int)colidx;
      val[pos] = band[t];
    }
  }
}

CsrDims dims_of(const wq_rules *R) {
  CsrDims D;
  D.p = R->p;
  D.dim = R->dim;
  D.nb = 2 * R->p + 1;
  D.band = 1;
  for (int a = 0; a < 3; a++) D.n[a] = a < R->dim ? R->n[a] : 1;
  for (int a = 0; a < R->dim; a++) D.band *= D.nb;
  return D;
}

}  // namespace

extern "C" {

int64_t wq_band_nnz_rows(const wq_rules *R, int64_t row_begin, int64_t row_end) {
  if (!R) return -1;
  const int64_t rows = (int64_t)R->n[0] * R->n[1] * R->n[2];
  if (row_begin < 0 || row_end > rows || row_begin > row_end) return -1;
  if (row_begin == row_end) return 0;
  const CsrDims D = dims_of(R);
  return row_ptr(row_end - 1, D) + row_cnt(row_end - 1, D) - row_ptr(row_begin, D);
}

wq_status wq_band_to_csr(const wq_rules *R, wq_precision prec, const void *band, int64_t row_begin, int64_t row_end,
                         int64_t *rowptr, int32_t *col, void *val, void *stream) {
  wq::TraceRange trace("wq_band_to_csr");
  if (!R || !R->on_device) return WQ_ERR_ARG;
  if (prec != WQ_FP64 && prec != WQ_MIXED && prec != WQ_DF64) return WQ_ERR_ARG;
  const int64_t rows = (int64_t)R->n[0] * R->n[1] * R->n[2];
  if (row_begin < 0 || row_end > rows || row_begin > row_end) return WQ_ERR_ARG;
  if (rows > INT32_MAX) return WQ_ERR_UNSUPPORTED;
  if (!rowptr) return WQ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (row_begin == row_end) {
    return cudaMemsetAsync(rowptr, 0, sizeof(int64_t), s) == cudaSuccess ? WQ_OK : WQ_ERR_CUDA;
  }
  if (!band || !col || !val) return WQ_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != R->device) return WQ_ERR_ARG;
  const CsrDims D = dims_of(R);
  const long long base = row_ptr(row_begin, D);
  const long long total = (row_end - row_begin) * (long long)D.band;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (total + 255) / 256;
  const int blocks = (int)std::min<long long>(want, (long long)std::max(nsm, 1) * 16);
  if (prec == WQ_MIXED)
    band_to_csr_kernel<float><<<blocks, 256, 0, s>>>(D, static_cast<const float *>(band), row_begin, row_end, base,
                                                     rowptr, col, static_cast<float *>(val));
  else
    band_to_csr_kernel<double><<<blocks, 256, 0, s>>>(D, static_cast<const double *>(band), row_begin, row_end,
                                                      base, rowptr, col, static_cast<double *>(val));
  return cudaGetLastError() == cudaSuccess ? WQ_OK : WQ_ERR_CUDA;
}

}  // extern "C"
