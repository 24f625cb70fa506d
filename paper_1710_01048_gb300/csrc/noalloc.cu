// wq_assemble_noalloc: mass/stiffness assembly that allocates no device
// memory, for callers that cannot call cudaMalloc -- code running inside a
// host application whose device memory is owned by someone else's pool or
// arena, or where allocation is forbidden while the application runs.
//
// Everything the ordinary path keeps in a wq_rules object's device block (the
// 1D row tables, the folded geometry tables, the line lists, the status
// word) lives here in one file-scope __device__ array of fixed size.  Every
// GPU that loads the library holds that array until the process exits.  The
// host tables come from a wq_rules object, which may be host-only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "fold.cuh"
#include "launch.cuh"
#include "wq_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

// The shared scratch of every wq_assemble_noalloc call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mutex;
unsigned char *g_scratch[kMaxDevices] = {};

size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
wq_status scratch_address(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return WQ_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return WQ_ERR_CUDA;
    }
    g_scratch[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch[dev];
  return WQ_OK;
}

// Byte offsets of the arrays inside the scratch.
struct Layout {
  size_t off[3][2], elem[3][2], w[3][2], t0[3][2], t1[3][2], beta[3][2], v64[3][2], v32[3][2], beta32[3][2];
  size_t lines_in, lines_bd, status, total;
};

Layout layout_of(const wq_rules *R) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  size_t t = 0;
  const size_t np = (size_t)R->p + 1;
  auto take = [&](size_t bytes) {
    size_t o = t;
    t += up(bytes);
    return o;
  };
  for (int a = 0; a < R->dim; a++)
    for (int k = 0; k < 2; k++) {
      const wq::HostDirKind &H = R->host[a][k];
      const size_t n = H.elem.size();
      L.off[a][k] = take(H.off.size() * sizeof(int));
      L.elem[a][k] = take(n * sizeof(int));
      L.w[a][k] = take(n * sizeof(double));
      L.t0[a][k] = take(n * np * sizeof(double));
      L.t1[a][k] = take(n * np * sizeof(double));
      L.beta[a][k] = take(n * 4 * sizeof(double));
      L.v64[a][k] = take(n * np * sizeof(double));
      L.v32[a][k] = take(n * np * sizeof(float));
      L.beta32[a][k] = take(n * 4 * sizeof(float));
    }
  L.lines_in = take(R->lines.interior.size() * sizeof(int) + sizeof(int));
  L.lines_bd = take(R->lines.boundary.size() * sizeof(int) + sizeof(int));
  L.status = take(sizeof(unsigned));
  L.total = t;
  return L;
}

struct NaSeg {
  const int *elem;
  const double *w, *t0, *t1, *beta, *g;
  double *v64;
  float *v32, *beta32;
  int start, kind;
};
struct NaFoldArgs {
  NaSeg seg[6];
  int nseg, total, np;
  unsigned *status;
};

// The geometry-factor fold (mass kind: W |J_aa| B; stiffness kind:
// W / |J_aa| B') into the scratch through wq::fold_point (FP64 and float
// tables, the arithmetic of the ordinary fold), plus the float copy of the
// cubic B-spline values at the points (beta) that the mixed mode reads; the
// coefficients themselves are converted by the row kernel.
__global__ void fold_noalloc_kernel(const NaFoldArgs A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned bits = 0;
  if (t < A.total) {
    int s = 0;
    while (s + 1 < A.nseg && t >= A.seg[s + 1].start) s++;
    const NaSeg &S = A.seg[s];
    const int q = t - S.start;
    bits = wq::fold_point(q, A.np, S.kind, S.elem, S.w, S.t0, S.t1, S.g, S.v64, S.v32, nullptr);
    for (int i = 0; i < 4; i++) S.beta32[(size_t)q * 4 + i] = (float)S.beta[(size_t)q * 4 + i];
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(A.status, bits);
}

}  // namespace

extern "C" wq_status wq_assemble_noalloc(const wq_rules *R, const double *const *geom, const double *coef,
                                         wq_precision prec, void *M, void *K, int64_t row_begin, int64_t row_end,
                                         void *stream, int check_status) {
  if (!R || !geom) return WQ_ERR_ARG;
  if (prec != WQ_FP64 && prec != WQ_MIXED) return WQ_ERR_ARG;
  if (R->mode != wq::kModeWQ || R->bnd_weighted) return WQ_ERR_UNSUPPORTED;
  const int64_t rows = (int64_t)R->n[0] * R->n[1] * R->n[2];
  if (row_begin < 0 || row_end > rows || row_begin > row_end) return WQ_ERR_ARG;
  if (row_begin == row_end) return WQ_OK;
  if (!M && !K) return WQ_ERR_ARG;
  for (int a = 0; a < R->dim; a++)
    if (!geom[a]) return WQ_ERR_ARG;
  const Layout L = layout_of(R);
  if (L.total > kScratchBytes) return WQ_ERR_UNSUPPORTED;

  unsigned char *base = nullptr;
  wq_status st = scratch_address(&base);
  if (st != WQ_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t np = (size_t)R->p + 1;

  // The array keeps the previous call's contents: start the status at zero
  // and overwrite every table this call reads.
  bool ok = cudaMemsetAsync(base + L.status, 0, sizeof(unsigned), s) == cudaSuccess;
  auto put = [&](size_t off, const void *src, size_t bytes) {
    if (ok && bytes) ok = cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
  };
  for (int a = 0; a < R->dim; a++)
    for (int k = 0; k < 2; k++) {
      const wq::HostDirKind &H = R->host[a][k];
      const size_t n = H.elem.size();
      put(L.off[a][k], H.off.data(), H.off.size() * sizeof(int));
      put(L.elem[a][k], H.elem.data(), n * sizeof(int));
      put(L.w[a][k], H.w.data(), n * sizeof(double));
      put(L.t0[a][k], H.t0.data(), n * np * sizeof(double));
      put(L.t1[a][k], H.t1.data(), n * np * sizeof(double));
      put(L.beta[a][k], H.beta.data(), n * 4 * sizeof(double));
    }
  put(L.lines_in, R->lines.interior.data(), R->lines.interior.size() * sizeof(int));
  put(L.lines_bd, R->lines.boundary.data(), R->lines.boundary.size() * sizeof(int));
  if (!ok) {
    cudaGetLastError();
    return WQ_ERR_CUDA;
  }

  NaFoldArgs fa;
  std::memset(&fa, 0, sizeof(fa));
  int total = 0, ns = 0;
  for (int a = 0; a < R->dim; a++)
    for (int k = 0; k < 2; k++) {
      NaSeg &S = fa.seg[ns++];
      S.elem = reinterpret_cast<const int *>(base + L.elem[a][k]);
      S.w = reinterpret_cast<const double *>(base + L.w[a][k]);
      S.t0 = reinterpret_cast<const double *>(base + L.t0[a][k]);
      S.t1 = reinterpret_cast<const double *>(base + L.t1[a][k]);
      S.beta = reinterpret_cast<const double *>(base + L.beta[a][k]);
      S.g = geom[a];
      S.v64 = reinterpret_cast<double *>(base + L.v64[a][k]);
      S.v32 = reinterpret_cast<float *>(base + L.v32[a][k]);
      S.beta32 = reinterpret_cast<float *>(base + L.beta32[a][k]);
      S.start = total;
      S.kind = k;
      total += (int)R->host[a][k].elem.size();
    }
  fa.nseg = ns;
  fa.total = total;
  fa.np = R->p + 1;
  unsigned *status = reinterpret_cast<unsigned *>(base + L.status);
  fa.status = status;
  fold_noalloc_kernel<<<(total + 255) / 256, 256, 0, s>>>(fa);
  if (cudaGetLastError() != cudaSuccess) return WQ_ERR_CUDA;

  wq::RowsArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  for (int a = 0; a < 3; a++) {
    const int aa = a < R->dim ? a : 0;
    for (int k = 0; k < 2; k++) {
      ra.off[a][k] = reinterpret_cast<const int *>(base + L.off[aa][k]);
      ra.elem[a][k] = reinterpret_cast<const int *>(base + L.elem[aa][k]);
      ra.V[a][k] = prec == WQ_FP64 ? (const void *)(base + L.v64[aa][k]) : (const void *)(base + L.v32[aa][k]);
      ra.beta[a][k] = prec == WQ_FP64 ? (const void *)(base + L.beta[aa][k]) : (const void *)(base + L.beta32[aa][k]);
    }
    ra.n[a] = R->n[a];
    ra.N[a] = R->nel[a];
    ra.nc[a] = R->nc[a];
  }
  ra.coef = coef;
  ra.M = M;
  ra.K = K;
  ra.bnd_grouped = 1;  // Gauss-Legendre boundary rows
  ra.row_begin = row_begin;
  ra.row_end = row_end;
  ra.status = status;
  const int n1 = R->n[0];
  const int first_line = (int)(row_begin / n1), last_line = (int)((row_end - 1) / n1);
  for (int cls = 0; cls < 2; cls++) {
    const std::vector<int> &lines = cls == 0 ? R->lines.interior : R->lines.boundary;
    auto lo = std::lower_bound(lines.begin(), lines.end(), first_line);
    auto hi = std::upper_bound(lines.begin(), lines.end(), last_line);
    const int nl = (int)(hi - lo);
    if (nl <= 0) continue;
    const int tmax = cls == 0 ? wq::interior_chunk(R->p, prec == WQ_MIXED ? 4 : 8) : wq::kBoundaryChunk;
    const int T = wq::chunk_length(R, tmax);
    if (wq::max_chunk_points(R, T) > wq::chunk_points_bound(R->p, tmax)) return WQ_ERR_UNSUPPORTED;
    ra.T = T;
    ra.nch = (n1 + T - 1) / T;
    ra.lines = reinterpret_cast<const int *>(base + (cls == 0 ? L.lines_in : L.lines_bd)) + (lo - lines.begin());
    const bool dm = M != nullptr, dk = K != nullptr;
    cudaError_t e;
    if (R->p == 2)
      e = prec == WQ_FP64 ? wq::launch_rows<2, double>(R->dim, dm, dk, cls, ra, nl * ra.nch, s)
                          : wq::launch_rows<2, float>(R->dim, dm, dk, cls, ra, nl * ra.nch, s);
    else
      e = prec == WQ_FP64 ? wq::launch_rows<3, double>(R->dim, dm, dk, cls, ra, nl * ra.nch, s)
                          : wq::launch_rows<3, float>(R->dim, dm, dk, cls, ra, nl * ra.nch, s);
    if (e != cudaSuccess) return WQ_ERR_CUDA;
  }
  if (!check_status) return WQ_OK;
  if (cudaStreamSynchronize(s) != cudaSuccess) return WQ_ERR_CUDA;
  unsigned bits = 0;
  if (cudaMemcpy(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return WQ_ERR_CUDA;
  if (bits & wq::kBitChecked) return WQ_ERR_CHECK;
  if (bits & wq::kBitNonFinite) return WQ_ERR_NONFINITE;
  if (bits & wq::kBitGeometry) return WQ_ERR_GEOMETRY;
  return WQ_OK;
}
