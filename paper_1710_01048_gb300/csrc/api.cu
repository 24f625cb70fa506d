// C ABI of libwq: rule construction, device upload, the geometry-factor fold
// kernel and the assembly launches.  Every entry point returns a wq_status
// and never lets a C++ exception escape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fold.cuh"
#include "launch.cuh"
#include "wq_internal.h"

using wq::HostDirKind;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Folds the geometry factor into the 1D tables of every direction and kind
// (one thread per point, wq::fold_point).
struct FoldSeg {
  const int *elem;
  const double *w, *t0, *t1, *g;
  double *v64;
  float *v32;
  float2 *vdd;
  int start, kind;
};
struct FoldArgs {
  FoldSeg seg[6];
  int nseg, total, np;
  unsigned *status;
};

__global__ void fold_kernel(const FoldArgs A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned bits = 0;
  if (t < A.total) {
    int s = 0;
    while (s + 1 < A.nseg && t >= A.seg[s + 1].start) s++;
    const FoldSeg &S = A.seg[s];
    bits = wq::fold_point(t - S.start, A.np, S.kind, S.elem, S.w, S.t0, S.t1, S.g, S.v64, S.v32, S.vdd);
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(A.status, bits);
}

// Checks the coefficients for NaN/Inf and writes them in the arithmetic type
// of the call (float for the mixed mode, double-float pairs for df64; the
// FP64 mode reads the caller's array directly).
__global__ void coef_prepare_kernel(const double *__restrict__ c, size_t n, int prec, float *c32, float2 *cdd,
                                    unsigned *status) {
  unsigned bits = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bits |= wq::coef_point(c, i, prec, c32, cdd);
  bits = __reduce_or_sync(0xffffffffu, bits);
  if (bits && (threadIdx.x & 31) == 0) atomicOr(status, bits);
}

// dJ/dC of every coefficient: the sum, over the lines (x3 row ascending,
// then x2 row) and chunks (ascending) whose coefficient block contains it,
// of that block's entry.  One thread per coefficient.
__global__ void adjoint_gather_kernel(const wq::GatherArgs G) {
  const long long ncoef = (long long)G.nc[0] * G.nc[1] * G.nc[2];
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ncoef) return;
  const int P = G.p, NL = P + 4;
  const int c1 = (int)(g % G.nc[0]);
  const int c2 = (int)((g / G.nc[0]) % G.nc[1]);
  const int c3 = G.dim == 3 ? (int)(g / ((long long)G.nc[0] * G.nc[1])) : 0;
  const int n1 = G.n[0], N1 = G.N[0];
  double s = 0.0;
  const int r3lo = G.dim == 3 ? (c3 - 3 > 0 ? c3 - 3 : 0) : 0;
  const int r3hi = G.dim == 3 ? (c3 + P < G.n[2] - 1 ? c3 + P : G.n[2] - 1) : 0;
  for (int r3 = r3lo; r3 <= r3hi; r3++) {
    int e3lo = 0;
    bool in3 = true;
    if (G.dim == 3) {
      e3lo = r3 - P > 0 ? r3 - P : 0;
      const int e3hi = r3 < G.N[2] - 1 ? r3 : G.N[2] - 1;
      if (c3 < e3lo || c3 > e3hi + 3) continue;
      in3 = r3 >= P && r3 <= G.N[2] - 1;
    }
    const int r2lo = c2 - 3 > 0 ? c2 - 3 : 0, r2hi = c2 + P < G.n[1] - 1 ? c2 + P : G.n[1] - 1;
    for (int r2 = r2lo; r2 <= r2hi; r2++) {
      const int e2lo = r2 - P > 0 ? r2 - P : 0;
      const int e2hi = r2 < G.N[1] - 1 ? r2 : G.N[1] - 1;
      if (c2 < e2lo || c2 > e2hi + 3) continue;
      const bool in2 = r2 >= P && r2 <= G.N[1] - 1;
      const int T = (in2 && in3) ? G.T_int : G.T_bnd;
      const int nch = (n1 + T - 1) / T;
      const long long line = (long long)r2 + (long long)G.n[1] * r3;
      const long long base = line * n1;
      int chlo = (c1 - 2) / T - 1, chhi = (c1 + P) / T;
      if (chlo < 0) chlo = 0;
      if (chhi > nch - 1) chhi = nch - 1;
      for (int ch = chlo; ch <= chhi; ch++) {
        long long lo = (long long)ch * T, hi = lo + T;
        if (hi > n1) hi = n1;
        if (lo < G.row_begin - base) lo = G.row_begin - base;
        if (hi > G.row_end - base) hi = G.row_end - base;
        if (lo >= hi) continue;
        const int a = (int)lo, b = (int)hi;
        const int l1lo = a - P > 0 ? a - P : 0;
        const int e1hi = (b - 1) < N1 - 1 ? (b - 1) : N1 - 1;
        if (c1 < l1lo || c1 > e1hi + 3) continue;
        const long long slot = (line * G.nch_max + ch) * G.blk;
        const long long ent = G.dim == 3 ? ((long long)(c3 - e3lo) * NL + (c2 - e2lo)) * G.nl1max + (c1 - l1lo)
                                         : (long long)(c2 - e2lo) * G.nl1max + (c1 - l1lo);
        s += G.partial[slot + ent];
      }
    }
  }
  G.grad[g] = s;
}

// 3D: dJ/dC of every coefficient (c1, c2, c3): the sum, over the planes r3
// of the call whose x3 window holds c3 (ascending) and the line blocks of
// that plane whose x2 window holds c2 (ascending), of the block slot's
// entry [c1 - l1a][c2 - l2lo][c3 - l3lo] (adjoint_u_kernel; c1's column
// block is unique).  One thread per coefficient.
__global__ void adjoint_gather3_kernel(const wq::GatherArgs G) {
  const long long ncoef = (long long)G.nc[0] * G.nc[1] * G.nc[2];
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ncoef) return;
  const int P = G.p, NL = P + 4, NL2 = wq::kAULines + P + 3;
  const long long CBAR = (long long)wq::kAUCols * NL2 * NL;
  const int c1 = (int)(g % G.nc[0]);
  const int c2 = (int)((g / G.nc[0]) % G.nc[1]);
  const int c3 = (int)(g / ((long long)G.nc[0] * G.nc[1]));
  const int b1 = c1 / wq::kAUCols, l1 = c1 - b1 * wq::kAUCols;
  int r3lo = c3 - 3 > G.r3_lo ? c3 - 3 : G.r3_lo;
  int r3hi = c3 + P < G.r3_hi ? c3 + P : G.r3_hi;
  int b2lo = (c2 - wq::kAULines - 3) / wq::kAULines;
  if (b2lo < 0) b2lo = 0;
  int b2hi = (c2 + P) / wq::kAULines;
  if (b2hi > G.nblk2 - 1) b2hi = G.nblk2 - 1;
  double s = 0.0;
  for (int r3 = r3lo; r3 <= r3hi; r3++) {
    const int l3lo = r3 - P > 0 ? r3 - P : 0;
    const int l3hi = (r3 < G.N[2] - 1 ? r3 : G.N[2] - 1) + 3;
    if (c3 < l3lo || c3 > l3hi) continue;
    for (int b2 = b2lo; b2 <= b2hi; b2++) {
      const int r2a = b2 * wq::kAULines;
      const int r2e = (r2a + wq::kAULines - 1 < G.n[1] - 1 ? r2a + wq::kAULines - 1 : G.n[1] - 1);
      const int l2lo = r2a - P > 0 ? r2a - P : 0;
      const int l2hi = (r2e < G.N[1] - 1 ? r2e : G.N[1] - 1) + 3;
      if (c2 < l2lo || c2 > l2hi) continue;
      const long long blk = ((long long)(r3 - G.r3_lo) * G.nblk2 + b2) * G.nblk1 + b1;
      s += G.partial[blk * CBAR + ((long long)l1 * NL2 + (c2 - l2lo)) * NL + (c3 - l3lo)];
    }
  }
  G.grad[g] = s;
}

wq_status upload(wq_rules *R) {
  // fault injection for callers' error paths: the device allocation fails
  if (std::getenv("WQ_FAULT_DEVICE_ALLOC")) return WQ_ERR_OOM;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return WQ_ERR_CUDA;
  int np = R->p + 1;
  size_t total = 0;
  // sizes per (dir, kind): off, elem, w, t0, t1, beta, v64, v32, beta32, vdd, betadd, tl
  size_t off_sz[3][2][12];
  for (int a = 0; a < R->dim; a++)
    for (int k = 0; k < 2; k++) {
      const HostDirKind &H = R->host[a][k];
      size_t npts = H.elem.size();
      size_t s[12] = {H.off.size() * sizeof(int), npts * sizeof(int), npts * sizeof(double),
                      npts * np * sizeof(double), npts * np * sizeof(double), npts * 4 * sizeof(double),
                      npts * np * sizeof(double), npts * np * sizeof(float), npts * 4 * sizeof(float),
                      npts * np * sizeof(float2), npts * 4 * sizeof(float2), npts * (np - 1) * sizeof(double)};
      for (int i = 0; i < 12; i++) {
        off_sz[a][k][i] = total;
        total += align_up(s[i]);
      }
    }
  size_t lines_int = total;
  total += align_up(R->lines.interior.size() * sizeof(int) + sizeof(int));
  size_t lines_bnd = total;
  total += align_up(R->lines.boundary.size() * sizeof(int) + sizeof(int));
  size_t status_off = total;
  total += align_up(sizeof(unsigned));
  const size_t ncoef = (size_t)R->nc[0] * R->nc[1] * R->nc[2];
  size_t coef32_off = total;
  total += align_up(ncoef * sizeof(float));
  size_t coefdd_off = total;
  total += align_up(ncoef * sizeof(float2));

  void *block = nullptr;
  cudaError_t e = cudaMalloc(&block, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? WQ_ERR_OOM : WQ_ERR_CUDA;
  }
  char *base = static_cast<char *>(block);
  auto put = [&](size_t off, const void *src, size_t bytes) -> bool {
    return bytes == 0 || cudaMemcpy(base + off, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  bool ok = true;
  for (int a = 0; a < R->dim; a++)
    for (int k = 0; k < 2; k++) {
      const HostDirKind &H = R->host[a][k];
      size_t npts = H.elem.size();
      std::vector<float> b32(H.beta.begin(), H.beta.end());
      std::vector<float2> bdd(H.beta.size());
      for (size_t i = 0; i < H.beta.size(); i++) {
        float hi = (float)H.beta[i];
        bdd[i] = make_float2(hi, (float)(H.beta[i] - (double)hi));
      }
      ok = ok && put(off_sz[a][k][0], H.off.data(), H.off.size() * sizeof(int));
      ok = ok && put(off_sz[a][k][1], H.elem.data(), npts * sizeof(int));
      ok = ok && put(off_sz[a][k][2], H.w.data(), npts * sizeof(double));
      ok = ok && put(off_sz[a][k][3], H.t0.data(), npts * np * sizeof(double));
      ok = ok && put(off_sz[a][k][4], H.t1.data(), npts * np * sizeof(double));
      ok = ok && put(off_sz[a][k][5], H.beta.data(), npts * 4 * sizeof(double));
      ok = ok && put(off_sz[a][k][8], b32.data(), npts * 4 * sizeof(float));
      ok = ok && put(off_sz[a][k][10], bdd.data(), npts * 4 * sizeof(float2));
      ok = ok && put(off_sz[a][k][11], H.tl.data(), npts * (np - 1) * sizeof(double));
      wq::DevDirKind &Dk = R->dev[a][k];
      Dk.off = reinterpret_cast<const int *>(base + off_sz[a][k][0]);
      Dk.elem = reinterpret_cast<const int *>(base + off_sz[a][k][1]);
      Dk.w = reinterpret_cast<const double *>(base + off_sz[a][k][2]);
      Dk.t0 = reinterpret_cast<const double *>(base + off_sz[a][k][3]);
      Dk.t1 = reinterpret_cast<const double *>(base + off_sz[a][k][4]);
      Dk.beta = reinterpret_cast<const double *>(base + off_sz[a][k][5]);
      Dk.v64 = reinterpret_cast<double *>(base + off_sz[a][k][6]);
      Dk.v32 = reinterpret_cast<float *>(base + off_sz[a][k][7]);
      Dk.beta32 = reinterpret_cast<float *>(base + off_sz[a][k][8]);
      Dk.vdd = reinterpret_cast<float2 *>(base + off_sz[a][k][9]);
      Dk.betadd = reinterpret_cast<float2 *>(base + off_sz[a][k][10]);
      Dk.tl = reinterpret_cast<const double *>(base + off_sz[a][k][11]);
      Dk.npts = (int)npts;
    }
  ok = ok && put(lines_int, R->lines.interior.data(), R->lines.interior.size() * sizeof(int));
  ok = ok && put(lines_bnd, R->lines.boundary.data(), R->lines.boundary.size() * sizeof(int));
  ok = ok && cudaMemset(base + status_off, 0, sizeof(unsigned)) == cudaSuccess;
  if (!ok) {
    cudaFree(block);
    return WQ_ERR_CUDA;
  }
  R->dev_lines_interior = reinterpret_cast<const int *>(base + lines_int);
  R->dev_lines_boundary = reinterpret_cast<const int *>(base + lines_bnd);
  R->dev_status = reinterpret_cast<unsigned *>(base + status_off);
  R->dev_coef32 = reinterpret_cast<float *>(base + coef32_off);
  R->dev_coefdd = reinterpret_cast<float2 *>(base + coefdd_off);
  R->dev_block = block;
  R->dev_bytes = total;
  // the mixed-derivative kinds' tables (maps given by a full control net)
  if (!R->hostx[0].elem.empty()) {
    size_t xo[3][7], xt = 0;
    for (int a = 0; a < R->dim; a++) {
      const wq::HostCross &X = R->hostx[a];
      const size_t npts = X.elem.size();
      const size_t sz[7] = {npts * sizeof(int), npts * sizeof(double), npts * sizeof(double),
                            npts * np * sizeof(double), npts * np * sizeof(double), npts * 4 * sizeof(double),
                            npts * (np - 1) * sizeof(double)};
      for (int i = 0; i < 7; i++) {
        xo[a][i] = xt;
        xt += align_up(sz[i]);
      }
    }
    void *xb = nullptr;
    e = cudaMalloc(&xb, xt);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(block);
      R->dev_block = nullptr;
      return e == cudaErrorMemoryAllocation ? WQ_ERR_OOM : WQ_ERR_CUDA;
    }
    char *xbase = static_cast<char *>(xb);
    bool xok = true;
    for (int a = 0; a < R->dim; a++) {
      const wq::HostCross &X = R->hostx[a];
      const size_t npts = X.elem.size();
      const void *src[7] = {X.elem.data(), X.w2.data(), X.w3.data(), X.t0.data(), X.t1.data(), X.beta.data(),
                            X.tl.data()};
      const size_t sz[7] = {npts * sizeof(int), npts * sizeof(double), npts * sizeof(double),
                            npts * np * sizeof(double), npts * np * sizeof(double), npts * 4 * sizeof(double),
                            npts * (np - 1) * sizeof(double)};
      for (int i = 0; i < 7; i++)
        xok = xok && (sz[i] == 0 || cudaMemcpy(xbase + xo[a][i], src[i], sz[i], cudaMemcpyHostToDevice) == cudaSuccess);
      wq::DevCross &D = R->devx[a];
      D.elem = reinterpret_cast<const int *>(xbase + xo[a][0]);
      D.w2 = reinterpret_cast<const double *>(xbase + xo[a][1]);
      D.w3 = reinterpret_cast<const double *>(xbase + xo[a][2]);
      D.t0 = reinterpret_cast<const double *>(xbase + xo[a][3]);
      D.t1 = reinterpret_cast<const double *>(xbase + xo[a][4]);
      D.beta = reinterpret_cast<const double *>(xbase + xo[a][5]);
      D.tl = reinterpret_cast<const double *>(xbase + xo[a][6]);
      D.npts = (int)npts;
    }
    if (!xok) {
      cudaFree(xb);
      cudaFree(block);
      R->dev_block = nullptr;
      return WQ_ERR_CUDA;
    }
    R->dev_cross = xb;
    R->dev_bytes += xt;
    // derived tables of the non-separable path, staged on the host and copied at once
    std::vector<char> stage;
    auto push = [&stage](const void *src, size_t bytes) -> size_t {
      const size_t off = stage.size();
      stage.resize(align_up(off + bytes));
      if (bytes) std::memcpy(stage.data() + off, src, bytes);
      return off;
    };
    size_t go[3][3][3], gw64[3][4], gw32[3][4];
    for (int a = 0; a < R->dim; a++) {
      const wq::HostDirKind *Hk[2] = {&R->host[a][0], &R->host[a][1]};
      const wq::HostCross &X = R->hostx[a];
      const std::vector<double> *t0s[3] = {&Hk[0]->t0, &Hk[1]->t0, &X.t0};
      const std::vector<double> *tls[3] = {&Hk[0]->tl, &Hk[1]->tl, &X.tl};
      const std::vector<double> *bes[3] = {&Hk[0]->beta, &Hk[1]->beta, &X.beta};
      for (int k = 0; k < 3; k++) {
        const std::vector<double> *src[3] = {t0s[k], tls[k], bes[k]};
        for (int t = 0; t < 3; t++) {
          std::vector<float> f(src[t]->begin(), src[t]->end());
          go[a][k][t] = push(f.data(), f.size() * sizeof(float));
        }
      }
      const std::vector<double> *ws[4] = {&Hk[0]->w, &Hk[1]->w, &X.w2, &X.w3};
      const std::vector<double> *ts[4] = {&Hk[0]->t0, &Hk[1]->t1, &X.t0, &X.t1};
      for (int k = 0; k < 4; k++) {
        const size_t npts = ws[k]->size();
        std::vector<double> w64(npts * np);
        std::vector<float> w32(npts * np);
        for (size_t q = 0; q < npts; q++)
          for (int i = 0; i < np; i++) {
            w64[q * np + i] = (*ws[k])[q] * (*ts[k])[q * np + i];
            w32[q * np + i] = (float)w64[q * np + i];
          }
        gw64[a][k] = push(w64.data(), w64.size() * sizeof(double));
        gw32[a][k] = push(w32.data(), w32.size() * sizeof(float));
      }
    }
    void *gb = nullptr;
    e = cudaMalloc(&gb, stage.size());
    if (e != cudaSuccess || cudaMemcpy(gb, stage.data(), stage.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      if (gb) cudaFree(gb);
      cudaFree(xb);
      cudaFree(block);
      R->dev_block = nullptr;
      R->dev_cross = nullptr;
      return e == cudaErrorMemoryAllocation ? WQ_ERR_OOM : WQ_ERR_CUDA;
    }
    const char *gbase = static_cast<const char *>(gb);
    for (int a = 0; a < R->dim; a++) {
      wq::GmDevTab &G = R->gmt[a];
      for (int k = 0; k < 3; k++) {
        G.t0f[k] = reinterpret_cast<const float *>(gbase + go[a][k][0]);
        G.tlf[k] = reinterpret_cast<const float *>(gbase + go[a][k][1]);
        G.betaf[k] = reinterpret_cast<const float *>(gbase + go[a][k][2]);
      }
      for (int k = 0; k < 4; k++) {
        G.wt64[k] = reinterpret_cast<const double *>(gbase + gw64[a][k]);
        G.wt32[k] = reinterpret_cast<const float *>(gbase + gw32[a][k]);
      }
    }
    R->dev_gmtab = gb;
    R->dev_bytes += stage.size();
  }
  if (R->dim == 3 && R->mode == wq::kModeWQ) {
    const int nb = 2 * R->p + 1;
    const size_t ubytes = (size_t)R->n[1] * R->n[2] * 2 * R->nc[0] * nb * nb * sizeof(double);
    e = cudaMalloc(&R->dev_U, ubytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(block);
      if (R->dev_cross) cudaFree(R->dev_cross);
      if (R->dev_gmtab) cudaFree(R->dev_gmtab);
      R->dev_block = nullptr;
      R->dev_cross = nullptr;
      R->dev_gmtab = nullptr;
      R->dev_U = nullptr;
      return e == cudaErrorMemoryAllocation ? WQ_ERR_OOM : WQ_ERR_CUDA;
    }
    R->dev_bytes += ubytes;
  }
  R->device = dev;
  R->on_device = true;
  return WQ_OK;
}

wq_status check_launch(cudaError_t e) {
  if (e == cudaSuccess) return WQ_OK;
  return WQ_ERR_CUDA;
}

wq_status launch_fold(const wq_rules *R, const double *const *geom, cudaStream_t s) {
  FoldArgs fa;
  std::memset(&fa, 0, sizeof(fa));
  int total = 0, ns = 0;
  for (int a = 0; a < R->dim; a++)
    for (int k = 0; k < 2; k++) {
      const wq::DevDirKind &Dk = R->dev[a][k];
      FoldSeg &S = fa.seg[ns++];
      S.elem = Dk.elem;
      S.w = Dk.w;
      S.t0 = Dk.t0;
      S.t1 = Dk.t1;
      S.g = geom[a];
      S.v64 = Dk.v64;
      S.v32 = Dk.v32;
      S.vdd = Dk.vdd;
      S.start = total;
      S.kind = k;
      total += Dk.npts;
    }
  fa.nseg = ns;
  fa.total = total;
  fa.np = R->p + 1;
  fa.status = R->dev_status;
  fold_kernel<<<(total + 255) / 256, 256, 0, s>>>(fa);
  return check_launch(cudaGetLastError());
}

// Table pointers and sizes of a rules object for one arithmetic type.
void fill_tables(const wq_rules *R, wq_precision prec, wq::RowsArgs &ra) {
  std::memset(&ra, 0, sizeof(ra));
  for (int a = 0; a < 3; a++) {
    int aa = a < R->dim ? a : 0;
    for (int k = 0; k < 2; k++) {
      const wq::DevDirKind &Dk = R->dev[aa][k];
      ra.off[a][k] = Dk.off;
      ra.elem[a][k] = Dk.elem;
      ra.V[a][k] = prec == WQ_FP64 ? (const void *)Dk.v64
                   : prec == WQ_MIXED ? (const void *)Dk.v32 : (const void *)Dk.vdd;
      ra.beta[a][k] = prec == WQ_FP64 ? (const void *)Dk.beta
                      : prec == WQ_MIXED ? (const void *)Dk.beta32 : (const void *)Dk.betadd;
    }
    ra.n[a] = R->n[a];
    ra.N[a] = R->nel[a];
    ra.nc[a] = R->nc[a];
  }
  // boundary x1 rows: Gauss-Legendre, P+1 points per element in element
  // order, unless the boundary rows have their own weighted rules
  ra.bnd_grouped = (R->mode == wq::kModeWQ && !R->bnd_weighted) ? 1 : 0;
}

// Line range and chunking of one line class for rows [rb, re); returns the
// number of CTAs (0 if the class has no line in the range).
int chunk_class(const wq_rules *R, int cls, int elem_bytes, int64_t rb, int64_t re, wq::RowsArgs &ra,
                wq_status *st) {
  const int n1 = R->n[0];
  const int first_line = (int)(rb / n1), last_line = (int)((re - 1) / n1);
  const std::vector<int> &lines = cls == 0 ? R->lines.interior : R->lines.boundary;
  auto lo = std::lower_bound(lines.begin(), lines.end(), first_line);
  auto hi = std::upper_bound(lines.begin(), lines.end(), last_line);
  const int nl = (int)(hi - lo);
  if (nl <= 0) return 0;
  const int tmax = R->mode ? wq::kGeneralChunk : cls == 0 ? wq::interior_chunk(R->p, elem_bytes) : wq::kBoundaryChunk;
  const int bound = R->mode ? wq::chunk_points_bound_general(R->p, tmax) : wq::chunk_points_bound(R->p, tmax);
  const int T = wq::chunk_length(R, tmax);
  if (wq::max_chunk_points(R, T) > bound) {
    *st = WQ_ERR_UNSUPPORTED;
    return 0;
  }
  ra.T = T;
  ra.nch = (n1 + T - 1) / T;
  ra.lines = (cls == 0 ? R->dev_lines_interior : R->dev_lines_boundary) + (lo - lines.begin());
  return nl * ra.nch;
}

// The 3D split path: u_kernel for the lines of rows [row_begin, row_end)
// (their U into R->dev_U), then one launch of the row kernel over those
// lines (apply: of the apply kernel, y into ra.M / ra.K).
wq_status assemble_split(const wq_rules *R, wq_precision prec, wq::RowsArgs &ra, cudaStream_t s,
                         bool apply = false) {
  const int n1 = R->n[0], n2 = R->n[1];
  const int first_line = (int)(ra.row_begin / n1), last_line = (int)((ra.row_end - 1) / n1);
  wq::UArgs ua;
  std::memset(&ua, 0, sizeof(ua));
  std::memcpy(ua.off, ra.off, sizeof(ua.off));
  std::memcpy(ua.elem, ra.elem, sizeof(ua.elem));
  std::memcpy(ua.V, ra.V, sizeof(ua.V));
  std::memcpy(ua.beta, ra.beta, sizeof(ua.beta));
  for (int a = 0; a < 3; a++) {
    ua.n[a] = ra.n[a];
    ua.N[a] = ra.N[a];
    ua.nc[a] = ra.nc[a];
  }
  ua.coef = ra.coef;
  ua.coefR = ra.coefR;
  ua.U = R->dev_U;
  ua.line_lo = first_line;
  ua.line_hi = last_line;
  ua.r3_lo = first_line / n2;
  ua.nblk2 = (n2 + wq::kULines - 1) / wq::kULines;
  ua.nblk1 = (R->nc[0] + wq::kUCols - 1) / wq::kUCols;
  ua.status = R->dev_status;
  const int nplanes = last_line / n2 - ua.r3_lo + 1;
  const int ublocks = nplanes * ua.nblk2 * ua.nblk1;
  const int tmax = apply ? wq::kApplyChunk : wq::kUGChunk;
  const int T = wq::chunk_length(R, tmax);
  if (wq::max_chunk_points(R, T) > wq::chunk_points_bound(R->p, tmax)) return WQ_ERR_UNSUPPORTED;
  ra.lines = nullptr;
  ra.line0 = first_line;
  ra.T = T;
  ra.nch = (n1 + T - 1) / T;
  ra.Ug = R->dev_U;
  const int rblocks = (last_line - first_line + 1) * ra.nch;
  const bool dm = ra.M != nullptr, dk = ra.K != nullptr;
  cudaError_t e;
  if (R->p == 2) {
    e = prec == WQ_FP64   ? wq::launch_u<2, double>(ua, ublocks, s)
        : prec == WQ_MIXED ? wq::launch_u<2, float>(ua, ublocks, s)
                           : wq::launch_u<2, wq::dd>(ua, ublocks, s);
    if (e == cudaSuccess && apply)
      e = prec == WQ_FP64   ? wq::launch_apply_ug<2, double>(dk, ra, rblocks, s)
          : prec == WQ_MIXED ? wq::launch_apply_ug<2, float>(dk, ra, rblocks, s)
                             : wq::launch_apply_ug<2, wq::dd>(dk, ra, rblocks, s);
    else if (e == cudaSuccess)
      e = prec == WQ_FP64   ? wq::launch_rows_ug<2, double>(dm, dk, ra, rblocks, s)
          : prec == WQ_MIXED ? wq::launch_rows_ug<2, float>(dm, dk, ra, rblocks, s)
                             : wq::launch_rows_ug<2, wq::dd>(dm, dk, ra, rblocks, s);
  } else {
    e = prec == WQ_FP64   ? wq::launch_u<3, double>(ua, ublocks, s)
        : prec == WQ_MIXED ? wq::launch_u<3, float>(ua, ublocks, s)
                           : wq::launch_u<3, wq::dd>(ua, ublocks, s);
    if (e == cudaSuccess && apply)
      e = prec == WQ_FP64   ? wq::launch_apply_ug<3, double>(dk, ra, rblocks, s)
          : prec == WQ_MIXED ? wq::launch_apply_ug<3, float>(dk, ra, rblocks, s)
                             : wq::launch_apply_ug<3, wq::dd>(dk, ra, rblocks, s);
    else if (e == cudaSuccess)
      e = prec == WQ_FP64   ? wq::launch_rows_ug<3, double>(dm, dk, ra, rblocks, s)
          : prec == WQ_MIXED ? wq::launch_rows_ug<3, float>(dm, dk, ra, rblocks, s)
                             : wq::launch_rows_ug<3, wq::dd>(dm, dk, ra, rblocks, s);
  }
  return e == cudaSuccess ? WQ_OK : WQ_ERR_CUDA;
}

// Argument checks shared by assembly and apply (rows [rb, re) non-empty or
// empty; outputs checked by the caller).
wq_status check_call(const wq_rules *R, const double *const *geom, wq_precision prec, int64_t rb, int64_t re) {
  if (!R || !geom) return WQ_ERR_ARG;
  if (!R->on_device) return WQ_ERR_ARG;
  if (prec != WQ_FP64 && prec != WQ_MIXED && prec != WQ_DF64) return WQ_ERR_ARG;
  if (R->mode != wq::kModeWQ && prec != WQ_FP64) return WQ_ERR_UNSUPPORTED;
  int64_t rows = (int64_t)R->n[0] * R->n[1] * R->n[2];
  if (rb < 0 || re > rows || rb > re) return WQ_ERR_ARG;
  for (int a = 0; a < R->dim; a++)
    if (!geom[a]) return WQ_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != R->device) return WQ_ERR_ARG;
  return WQ_OK;
}

// Fold, coefficient preparation and the row-kernel arguments for rows [rb, re).
wq_status prepare_rows(const wq_rules *R, const double *const *geom, const double *coef, wq_precision prec,
                       int64_t rb, int64_t re, cudaStream_t s, wq::RowsArgs &ra) {
  wq_status st = launch_fold(R, geom, s);
  if (st != WQ_OK) return st;
  fill_tables(R, prec, ra);
  ra.coef = coef;
  if (coef) {
    const size_t ncoef = (size_t)R->nc[0] * R->nc[1] * R->nc[2];
    const int blocks = (int)std::min<size_t>((ncoef + 255) / 256, 152 * 8);
    coef_prepare_kernel<<<blocks, 256, 0, s>>>(coef, ncoef, prec, R->dev_coef32, R->dev_coefdd, R->dev_status);
    if (cudaGetLastError() != cudaSuccess) return WQ_ERR_CUDA;
    ra.coefR = prec == WQ_FP64 ? (const void *)coef
               : prec == WQ_MIXED ? (const void *)R->dev_coef32 : (const void *)R->dev_coefdd;
  }
  ra.row_begin = rb;
  ra.row_end = re;
  ra.status = R->dev_status;
  return WQ_OK;
}

wq_status assemble(const wq_rules *R, const double *const *geom, const double *coef, wq_precision prec, void *M,
                   void *K, int64_t rb, int64_t re, void *stream) {
  wq::TraceRange trace("wq_assemble");
  wq_status st = check_call(R, geom, prec, rb, re);
  if (st != WQ_OK) return st;
  if (rb != re && !M && !K) return WQ_ERR_ARG;
  if (rb == re) return WQ_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  wq::RowsArgs ra;
  st = prepare_rows(R, geom, coef, prec, rb, re, s, ra);
  if (st != WQ_OK) return st;
  ra.M = M;
  ra.K = K;
  if (R->dev_U) return assemble_split(R, prec, ra, s);
  for (int cls = 0; cls < 2; cls++) {
    wq_status cst = WQ_OK;
    const int nblocks = chunk_class(R, cls, prec == WQ_MIXED ? 4 : 8, rb, re, ra, &cst);
    if (cst != WQ_OK) return cst;
    if (nblocks == 0) continue;
    cudaError_t e;
    bool dm = M != nullptr, dk = K != nullptr;
    const int kcls = R->mode ? 2 : cls;
    if (R->p == 2)
      e = prec == WQ_FP64   ? wq::launch_rows<2, double>(R->dim, dm, dk, kcls, ra, nblocks, s)
          : prec == WQ_MIXED ? wq::launch_rows<2, float>(R->dim, dm, dk, kcls, ra, nblocks, s)
                             : wq::launch_rows<2, wq::dd>(R->dim, dm, dk, kcls, ra, nblocks, s);
    else
      e = prec == WQ_FP64   ? wq::launch_rows<3, double>(R->dim, dm, dk, kcls, ra, nblocks, s)
          : prec == WQ_MIXED ? wq::launch_rows<3, float>(R->dim, dm, dk, kcls, ra, nblocks, s)
                             : wq::launch_rows<3, wq::dd>(R->dim, dm, dk, kcls, ra, nblocks, s);
    if (e != cudaSuccess) return WQ_ERR_CUDA;
  }
  return WQ_OK;
}

// y_M = M x, y_K = K x (x NULL: x = 1) through the split path's apply kernels.
wq_status apply(const wq_rules *R, const double *const *geom, const double *coef, wq_precision prec,
                const void *x, void *yM, void *yK, int64_t rb, int64_t re, void *stream) {
  wq::TraceRange trace("wq_apply");
  wq_status st = check_call(R, geom, prec, rb, re);
  if (st != WQ_OK) return st;
  if (R->mode != wq::kModeWQ || R->bnd_weighted || (R->dim == 3 && !R->dev_U)) return WQ_ERR_UNSUPPORTED;
  if (rb != re && !yM && !yK) return WQ_ERR_ARG;
  if (rb == re) return WQ_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  wq::RowsArgs ra;
  st = prepare_rows(R, geom, coef, prec, rb, re, s, ra);
  if (st != WQ_OK) return st;
  ra.M = yM;
  ra.K = yK;
  ra.x = x;
  if (R->dim == 3) return assemble_split(R, prec, ra, s, true);
  // 2D: the fused row kernel in apply mode, per line class
  const bool dk = yK != nullptr;
  for (int cls = 0; cls < 2; cls++) {
    wq_status cst = WQ_OK;
    const int nblocks = chunk_class(R, cls, prec == WQ_MIXED ? 4 : 8, rb, re, ra, &cst);
    if (cst != WQ_OK) return cst;
    if (nblocks == 0) continue;
    cudaError_t e;
    if (R->p == 2)
      e = prec == WQ_FP64   ? wq::launch_apply_2d<2, double>(cls, dk, ra, nblocks, s)
          : prec == WQ_MIXED ? wq::launch_apply_2d<2, float>(cls, dk, ra, nblocks, s)
                             : wq::launch_apply_2d<2, wq::dd>(cls, dk, ra, nblocks, s);
    else
      e = prec == WQ_FP64   ? wq::launch_apply_2d<3, double>(cls, dk, ra, nblocks, s)
          : prec == WQ_MIXED ? wq::launch_apply_2d<3, float>(cls, dk, ra, nblocks, s)
                             : wq::launch_apply_2d<3, wq::dd>(cls, dk, ra, nblocks, s);
    if (e != cudaSuccess) return WQ_ERR_CUDA;
  }
  return WQ_OK;
}

}  // namespace

extern "C" {

const char *wq_status_string(wq_status s) {
  switch (s) {
    case WQ_OK: return "ok";
    case WQ_ERR_ARG: return "invalid argument";
    case WQ_ERR_UNSUPPORTED: return "unsupported degree, dimension or size";
    case WQ_ERR_NO_CONVERGENCE: return "quadrature rule did not converge or failed its exactness check";
    case WQ_ERR_GEOMETRY: return "Jacobian entry <= 0 at a quadrature point";
    case WQ_ERR_NONFINITE: return "non-finite geometry or coefficient";
    case WQ_ERR_CUDA: return "CUDA runtime error";
    case WQ_ERR_OOM: return "device allocation failed";
    case WQ_ERR_TIMEOUT: return "bounded device wait expired";
    case WQ_ERR_CHECK: return "a device-side range check failed (checked build)";
  }
  return "unknown status";
}

int wq_version(void) { return 100; }

wq_status wq_rule_1d(int degree, int kind, double *tau, double *omega) {
  if (!tau || !omega) return WQ_ERR_ARG;
  if (degree < 2 || degree > wq::kMaxP || (kind != WQ_KIND_MASS && kind != WQ_KIND_STIFFNESS))
    return WQ_ERR_UNSUPPORTED;
  return wq::default_rule(degree, kind, tau, omega);
}

wq_status wq_rule_1d_mixed(int degree, double *y, double *w, double *v) {
  if (!y || !w || !v) return WQ_ERR_ARG;
  if (degree < 2 || degree > wq::kMaxP) return WQ_ERR_UNSUPPORTED;
  return wq::mixed_rule(degree, y, w, v);
}

wq_status wq_rule_1d_from(int degree, int kind, const double *start, double *tau, double *omega) {
  if (!start || !tau || !omega) return WQ_ERR_ARG;
  return wq::solve_rule(degree, kind, start, tau, omega);
}

wq_status wq_rules_build(const wq_mesh *mesh, int flags, wq_rules **out) {
  wq::TraceRange trace("wq_rules_build");
  if (!mesh || !out) return WQ_ERR_ARG;
  *out = nullptr;
  if (mesh->dim < 2 || mesh->dim > 3 || mesh->degree < 2 || mesh->degree > wq::kMaxP) return WQ_ERR_UNSUPPORTED;
  const int rule_bits = flags & (WQ_RULES_GAUSS_LEGENDRE | WQ_RULES_NEWTON_COTES);
  if ((flags & ~(WQ_RULES_DEVICE | WQ_RULES_GAUSS_LEGENDRE | WQ_RULES_NEWTON_COTES | WQ_RULES_BOUNDARY_WEIGHTED)) != 0)
    return WQ_ERR_ARG;
  if (rule_bits == (WQ_RULES_GAUSS_LEGENDRE | WQ_RULES_NEWTON_COTES)) return WQ_ERR_ARG;
  if (rule_bits && (flags & WQ_RULES_BOUNDARY_WEIGHTED)) return WQ_ERR_ARG;
  for (int a = 0; a < mesh->dim; a++) {
    if (mesh->nel[a] < 1) return WQ_ERR_ARG;
    if (mesh->nel[a] > wq::kMaxNel) return WQ_ERR_UNSUPPORTED;
  }
  int64_t rows = 1;
  for (int a = 0; a < mesh->dim; a++) rows *= mesh->nel[a] + mesh->degree;
  if (rows > (int64_t)1 << 31) return WQ_ERR_UNSUPPORTED;
  wq_rules *R = nullptr;
  try {
    R = new wq_rules();
    R->mesh = *mesh;
    R->p = mesh->degree;
    R->dim = mesh->dim;
    R->mode = rule_bits == WQ_RULES_GAUSS_LEGENDRE ? wq::kModeGL
              : rule_bits == WQ_RULES_NEWTON_COTES   ? wq::kModeNC : wq::kModeWQ;
    R->bnd_weighted = (flags & WQ_RULES_BOUNDARY_WEIGHTED) != 0;
    for (int a = 0; a < 3; a++) {
      R->nel[a] = a < mesh->dim ? mesh->nel[a] : 1;
      R->n[a] = a < mesh->dim ? mesh->nel[a] + mesh->degree : 1;
      R->nc[a] = a < mesh->dim ? mesh->nel[a] + wq::kCoefDeg : 1;
    }
    wq_status st = wq::build_host_tables(R);
    if (st == WQ_OK && (flags & WQ_RULES_DEVICE)) st = upload(R);
    if (st != WQ_OK) {
      delete R;
      return st;
    }
  } catch (const std::bad_alloc &) {
    delete R;
    return WQ_ERR_OOM;
  } catch (...) {
    delete R;
    return WQ_ERR_ARG;
  }
  *out = R;
  return WQ_OK;
}

void wq_rules_free(wq_rules *rules) {
  if (!rules) return;
  if (rules->dev_block) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != rules->device) cudaSetDevice(rules->device);
    cudaFree(rules->dev_block);
    if (rules->dev_U) cudaFree(rules->dev_U);
    if (rules->dev_adj) cudaFree(rules->dev_adj);
    if (rules->dev_cross) cudaFree(rules->dev_cross);
    if (rules->dev_gmtab) cudaFree(rules->dev_gmtab);
    if (rules->dev_gm) cudaFree(rules->dev_gm);
    if (cur >= 0 && cur != rules->device) cudaSetDevice(cur);
  }
  delete rules;
}

wq_status wq_rules_row(const wq_rules *R, int dir, int kind, int row, int *npts, double *x, double *w, int *elem) {
  if (!R || dir < 0 || dir >= R->dim || kind < 0 || kind > 3 || row < 0 || row >= R->n[dir]) return WQ_ERR_ARG;
  if (kind >= 2) {
    const wq::HostCross &X = R->hostx[dir];
    if (X.elem.empty()) return WQ_ERR_UNSUPPORTED;
    int o0 = X.off[row], o1 = X.off[row + 1];
    if (npts) *npts = o1 - o0;
    for (int q = o0; q < o1; q++) {
      if (x) x[q - o0] = X.x[q];
      if (w) w[q - o0] = kind == 2 ? X.w2[q] : X.w3[q];
      if (elem) elem[q - o0] = X.elem[q];
    }
    return WQ_OK;
  }
  const HostDirKind &H = R->host[dir][kind];
  int o0 = H.off[row], o1 = H.off[row + 1];
  if (npts) *npts = o1 - o0;
  for (int q = o0; q < o1; q++) {
    if (x) x[q - o0] = H.x[q];
    if (w) w[q - o0] = H.w[q];
    if (elem) elem[q - o0] = H.elem[q];
  }
  return WQ_OK;
}

int64_t wq_rows(const wq_rules *R) { return R ? (int64_t)R->n[0] * R->n[1] * R->n[2] : 0; }

int64_t wq_band_width(const wq_rules *R) {
  if (!R) return 0;
  int64_t b = 1;
  for (int a = 0; a < R->dim; a++) b *= 2 * R->p + 1;
  return b;
}

int64_t wq_band_nnz(const wq_rules *R) {
  if (!R) return 0;
  int64_t z = 1;
  for (int a = 0; a < R->dim; a++) {
    int64_t n = R->n[a], p = R->p;
    int64_t per = 0;
    for (int64_t r = 0; r < n; r++) per += std::min(n - 1, r + p) - std::max<int64_t>(0, r - p) + 1;
    z *= per;
  }
  return z;
}

int64_t wq_coef_count(const wq_rules *R) { return R ? (int64_t)R->nc[0] * R->nc[1] * R->nc[2] : 0; }

double wq_flop_count(const wq_rules *R, int want_m, int want_k, int64_t row_begin, int64_t row_end,
                     double *coef_flops) {
  if (!R || row_begin < 0 || row_end > wq_rows(R) || row_begin > row_end) return -1.0;
  return wq::flop_count(R, want_m, want_k, row_begin, row_end, coef_flops);
}

wq_status wq_assemble_mass(const wq_rules *rules, const double *const *geom, const double *coef, wq_precision prec,
                           void *M, int64_t row_begin, int64_t row_end, void *stream) {
  if (row_begin != row_end && (!M)) return WQ_ERR_ARG;
  return assemble(rules, geom, coef, prec, M, nullptr, row_begin, row_end, stream);
}

wq_status wq_assemble_stiffness(const wq_rules *rules, const double *const *geom, const double *coef,
                                wq_precision prec, void *K, int64_t row_begin, int64_t row_end, void *stream) {
  if (row_begin != row_end && (!K)) return WQ_ERR_ARG;
  return assemble(rules, geom, coef, prec, nullptr, K, row_begin, row_end, stream);
}

wq_status wq_assemble_mass_stiffness(const wq_rules *rules, const double *const *geom, const double *coef,
                                     wq_precision prec, void *M, void *K, int64_t row_begin, int64_t row_end,
                                     void *stream) {
  if (row_begin != row_end && (!M || !K)) return WQ_ERR_ARG;
  return assemble(rules, geom, coef, prec, M, K, row_begin, row_end, stream);
}

wq_status wq_assemble_mass_stiffness_host(const wq_rules *R, const double *const *geom_host,
                                          const double *coef_host, wq_precision prec, void *M_host, void *K_host,
                                          double *const *geom_dev, double *coef_dev, void *M_dev, void *K_dev,
                                          int64_t row_begin, int64_t row_end, int nchunks, void *stream,
                                          void *copy_stream) {
  wq::TraceRange trace("wq_assemble_mass_stiffness_host");
  if (!R || !geom_host || !geom_dev) return WQ_ERR_ARG;
  if (nchunks < 1 || nchunks > 1024) return WQ_ERR_ARG;
  if (stream == copy_stream) return WQ_ERR_ARG;
  if (coef_host && !coef_dev) return WQ_ERR_ARG;
  for (int a = 0; a < R->dim; a++)
    if (!geom_host[a] || !geom_dev[a]) return WQ_ERR_ARG;
  wq_status st = check_call(R, geom_dev, prec, row_begin, row_end);
  if (st != WQ_OK) return st;
  if (row_begin == row_end) return WQ_OK;
  if (!M_host || !K_host || !M_dev || !K_dev) return WQ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream), cs = static_cast<cudaStream_t>(copy_stream);
  // inputs: host -> device on the compute stream
  for (int a = 0; a < R->dim; a++)
    if (cudaMemcpyAsync(geom_dev[a], geom_host[a], (size_t)R->n[a] * sizeof(double), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return WQ_ERR_CUDA;
  const size_t ncoef = (size_t)R->nc[0] * R->nc[1] * R->nc[2];
  if (coef_host &&
      cudaMemcpyAsync(coef_dev, coef_host, ncoef * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return WQ_ERR_CUDA;
  const double *coef = coef_host ? coef_dev : nullptr;
  // one event marks each range's assembly (re-recorded per range: a wait
  // binds to the record made before it), one the end of the copies
  cudaEvent_t ready = nullptr, done = nullptr;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return WQ_ERR_CUDA;
  if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
    cudaEventDestroy(ready);
    return WQ_ERR_CUDA;
  }
  const int64_t band = wq_band_width(R), rows = row_end - row_begin;
  const size_t esz = prec == WQ_MIXED ? sizeof(float) : sizeof(double);
  for (int k = 0; k < nchunks && st == WQ_OK; k++) {
    const int64_t rb = row_begin + rows * k / nchunks, re = row_begin + rows * (k + 1) / nchunks;
    if (rb == re) continue;
    const size_t off = (size_t)(rb - row_begin) * band * esz, bytes = (size_t)(re - rb) * band * esz;
    char *md = static_cast<char *>(M_dev) + off, *kd = static_cast<char *>(K_dev) + off;
    st = assemble(R, geom_dev, coef, prec, md, kd, rb, re, stream);
    if (st != WQ_OK) break;
    if (cudaEventRecord(ready, s) != cudaSuccess || cudaStreamWaitEvent(cs, ready, 0) != cudaSuccess ||
        cudaMemcpyAsync(static_cast<char *>(M_host) + off, md, bytes, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaMemcpyAsync(static_cast<char *>(K_host) + off, kd, bytes, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
      st = WQ_ERR_CUDA;
  }
  if (st == WQ_OK &&
      (cudaEventRecord(done, cs) != cudaSuccess || cudaStreamWaitEvent(s, done, 0) != cudaSuccess))
    st = WQ_ERR_CUDA;
  // destruction is deferred by the runtime until the recorded work completes
  cudaEventDestroy(ready);
  cudaEventDestroy(done);
  return st;
}

wq_status wq_apply_mass_stiffness(const wq_rules *rules, const double *const *geom, const double *coef,
                                  wq_precision prec, const void *x, void *yM, void *yK, int64_t row_begin,
                                  int64_t row_end, void *stream) {
  if (row_begin != row_end && !x) return WQ_ERR_ARG;
  return apply(rules, geom, coef, prec, x, yM, yK, row_begin, row_end, stream);
}

wq_status wq_assemble_load(const wq_rules *rules, const double *const *geom, const double *f, wq_precision prec,
                           void *b, int64_t row_begin, int64_t row_end, void *stream) {
  if (row_begin != row_end && !b) return WQ_ERR_ARG;
  return apply(rules, geom, f, prec, nullptr, b, nullptr, row_begin, row_end, stream);
}

wq_status wq_assemble_adjoint(const wq_rules *R, const double *const *geom, wq_precision prec, const void *G,
                              const void *H, double *grad, int64_t row_begin, int64_t row_end, void *stream) {
  wq::TraceRange trace("wq_assemble_adjoint");
  if (!R || !geom || !grad) return WQ_ERR_ARG;
  if (!R->on_device) return WQ_ERR_ARG;
  if (R->mode != wq::kModeWQ || R->bnd_weighted) return WQ_ERR_UNSUPPORTED;
  if (prec != WQ_FP64 && prec != WQ_MIXED && prec != WQ_DF64) return WQ_ERR_ARG;
  const int64_t rows = (int64_t)R->n[0] * R->n[1] * R->n[2];
  if (row_begin < 0 || row_end > rows || row_begin > row_end) return WQ_ERR_ARG;
  for (int a = 0; a < R->dim; a++)
    if (!geom[a]) return WQ_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != R->device) return WQ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ncoef = (size_t)R->nc[0] * R->nc[1] * R->nc[2];
  if (row_begin == row_end || (!G && !H))
    return cudaMemsetAsync(grad, 0, ncoef * sizeof(double), s) == cudaSuccess ? WQ_OK : WQ_ERR_CUDA;
  // the chunking of both line classes, and the block scratch it needs
  const int eb = prec == WQ_MIXED ? 4 : 8, n1 = R->n[0], p = R->p;
  const int T_int = wq::chunk_length(R, wq::interior_chunk(p, eb));
  const int T_bnd = wq::chunk_length(R, wq::kBoundaryChunk);
  const int nch_max = std::max((n1 + T_int - 1) / T_int, (n1 + T_bnd - 1) / T_bnd);
  const int nl1max = std::max(T_int, T_bnd) + p + 3, NL = p + 4;
  const long long blk = (long long)NL * nl1max;  // 2D chunk blocks
  const size_t nlines = (size_t)R->n[1] * R->n[2];
  // 3D: Ubar chunk slots (arithmetic type), then the line-block slots (double)
  const int NB = 2 * p + 1, NPAIR = NB * NB;
  const long long ubar_slot = 2LL * nl1max * NPAIR;
  const size_t rbytes = prec == WQ_MIXED ? 4 : 8;
  const size_t ubar_bytes = (nlines * nch_max * (size_t)ubar_slot * rbytes + 255) / 256 * 256;
  const int nblk2 = (R->n[1] + wq::kAULines - 1) / wq::kAULines;
  const int nblk1 = (R->nc[0] + wq::kAUCols - 1) / wq::kAUCols;
  const size_t cbar_vals = (size_t)wq::kAUCols * (wq::kAULines + p + 3) * NL;
  const size_t need = R->dim == 3 ? ubar_bytes + (size_t)R->n[2] * nblk2 * nblk1 * cbar_vals * sizeof(double)
                                  : nlines * nch_max * (size_t)blk * sizeof(double);
  if (need > R->dev_adj_bytes) {
    // grown, never shrunk; the previous contents are not needed
    if (R->dev_adj && cudaStreamSynchronize(s) != cudaSuccess) return WQ_ERR_CUDA;
    if (R->dev_adj) cudaFree(R->dev_adj);
    R->dev_adj = nullptr;
    R->dev_adj_bytes = 0;
    void *p_adj = nullptr;
    const cudaError_t e = cudaMalloc(&p_adj, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? WQ_ERR_OOM : WQ_ERR_CUDA;
    }
    R->dev_adj = static_cast<double *>(p_adj);
    R->dev_adj_bytes = need;
  }
  wq_status st = launch_fold(R, geom, s);
  if (st != WQ_OK) return st;
  wq::AdjArgs aa;
  std::memset(&aa, 0, sizeof(aa));
  fill_tables(R, prec, aa.rows);
  aa.rows.row_begin = row_begin;
  aa.rows.row_end = row_end;
  aa.rows.status = R->dev_status;
  aa.G = G;
  aa.H = H;
  aa.partial = R->dev_adj;
  aa.nch_max = nch_max;
  aa.nl1max = nl1max;
  aa.blk = blk;
  double *cbar = reinterpret_cast<double *>(reinterpret_cast<char *>(R->dev_adj) + ubar_bytes);
  if (R->dim == 3) {
    aa.ubar = R->dev_adj;
    aa.ubar_slot = ubar_slot;
  }
  for (int cls = 0; cls < 2; cls++) {
    wq_status cst = WQ_OK;
    const int nblocks = chunk_class(R, cls, eb, row_begin, row_end, aa.rows, &cst);
    if (cst != WQ_OK) return cst;
    if (nblocks == 0) continue;
    cudaError_t e;
    if (R->p == 2)
      e = prec == WQ_FP64   ? wq::launch_adjoint<2, double>(R->dim, cls, aa, nblocks, s)
          : prec == WQ_MIXED ? wq::launch_adjoint<2, float>(R->dim, cls, aa, nblocks, s)
                             : wq::launch_adjoint<2, wq::dd>(R->dim, cls, aa, nblocks, s);
    else
      e = prec == WQ_FP64   ? wq::launch_adjoint<3, double>(R->dim, cls, aa, nblocks, s)
          : prec == WQ_MIXED ? wq::launch_adjoint<3, float>(R->dim, cls, aa, nblocks, s)
                             : wq::launch_adjoint<3, wq::dd>(R->dim, cls, aa, nblocks, s);
    if (e != cudaSuccess) return WQ_ERR_CUDA;
  }
  const int n2 = R->n[1];
  const int first_line = (int)(row_begin / n1), last_line = (int)((row_end - 1) / n1);
  const int r3_lo = first_line / n2, r3_hi = last_line / n2;
  if (R->dim == 3) {
    wq::AdjUArgs ua;
    std::memset(&ua, 0, sizeof(ua));
    std::memcpy(ua.off, aa.rows.off, sizeof(ua.off));
    std::memcpy(ua.elem, aa.rows.elem, sizeof(ua.elem));
    std::memcpy(ua.V, aa.rows.V, sizeof(ua.V));
    std::memcpy(ua.beta, aa.rows.beta, sizeof(ua.beta));
    for (int a = 0; a < 3; a++) {
      ua.n[a] = R->n[a];
      ua.N[a] = R->nel[a];
      ua.nc[a] = R->nc[a];
    }
    ua.ubar = R->dev_adj;
    ua.ubar_slot = ubar_slot;
    ua.nch_max = nch_max;
    ua.nl1max = nl1max;
    ua.T_int = T_int;
    ua.T_bnd = T_bnd;
    ua.row_begin = row_begin;
    ua.row_end = row_end;
    ua.line_lo = first_line;
    ua.line_hi = last_line;
    ua.r3_lo = r3_lo;
    ua.nblk2 = nblk2;
    ua.nblk1 = nblk1;
    ua.cbar = cbar;
    ua.status = R->dev_status;
    const int nblocks = (r3_hi - r3_lo + 1) * nblk2 * nblk1;
    cudaError_t e;
    if (R->p == 2)
      e = prec == WQ_FP64   ? wq::launch_adjoint_u<2, double>(ua, nblocks, s)
          : prec == WQ_MIXED ? wq::launch_adjoint_u<2, float>(ua, nblocks, s)
                             : wq::launch_adjoint_u<2, wq::dd>(ua, nblocks, s);
    else
      e = prec == WQ_FP64   ? wq::launch_adjoint_u<3, double>(ua, nblocks, s)
          : prec == WQ_MIXED ? wq::launch_adjoint_u<3, float>(ua, nblocks, s)
                             : wq::launch_adjoint_u<3, wq::dd>(ua, nblocks, s);
    if (e != cudaSuccess) return WQ_ERR_CUDA;
  }
  wq::GatherArgs ga;
  std::memset(&ga, 0, sizeof(ga));
  ga.partial = R->dev_adj;
  ga.grad = grad;
  ga.dim = R->dim;
  ga.p = p;
  for (int a = 0; a < 3; a++) {
    ga.n[a] = R->n[a];
    ga.N[a] = R->nel[a];
    ga.nc[a] = R->nc[a];
  }
  ga.row_begin = row_begin;
  ga.row_end = row_end;
  ga.T_int = T_int;
  ga.T_bnd = T_bnd;
  ga.nch_max = nch_max;
  ga.nl1max = nl1max;
  ga.blk = blk;
  if (R->dim == 3) {
    ga.partial = cbar;
    ga.r3_lo = r3_lo;
    ga.r3_hi = r3_hi;
    ga.nblk2 = nblk2;
    ga.nblk1 = nblk1;
    adjoint_gather3_kernel<<<(unsigned)((ncoef + 255) / 256), 256, 0, s>>>(ga);
  } else {
    adjoint_gather_kernel<<<(unsigned)((ncoef + 255) / 256), 256, 0, s>>>(ga);
  }
  return check_launch(cudaGetLastError());
}

wq_status wq_status_check(const wq_rules *R, void *stream) {
  if (!R || !R->on_device) return WQ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return WQ_ERR_CUDA;
  unsigned bits = 0;
  if (cudaMemcpy(&bits, R->dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return WQ_ERR_CUDA;
  if (cudaMemset(R->dev_status, 0, sizeof(unsigned)) != cudaSuccess) return WQ_ERR_CUDA;
  if (bits & wq::kBitInternal) return WQ_ERR_UNSUPPORTED;
  if (bits & wq::kBitChecked) return WQ_ERR_CHECK;
  if (bits & wq::kBitNonFinite) return WQ_ERR_NONFINITE;
  if (bits & wq::kBitGeometry) return WQ_ERR_GEOMETRY;
  return WQ_OK;
}

}  // extern "C"
