// Batched assembly of many independent 3D patches: the plan object
// (wq_batch), its batched geometry fold, the two persistent launches of the
// split 3D path captured in a CUDA graph, and the autotuner of their tile
// parameters.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "batch.cuh"
#include "fold.cuh"
#include "wq_internal.h"

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// One (patch, direction, kind) table of the batched fold.
struct BFold {
  const int *elem;
  const double *w, *t0, *t1, *g;
  double *v64;
  float *v32;
  float2 *vdd;
  int start, np, kind;
};

__global__ void batch_fold_kernel(const BFold *__restrict__ segs, int nseg, int total, unsigned *status) {
  unsigned bits = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].start <= t) lo = mid; else hi = mid - 1;
    }
    const BFold &S = segs[lo];
    bits |= wq::fold_point(t - S.start, S.np, S.kind, S.elem, S.w, S.t0, S.t1, S.g, S.v64, S.v32, S.vdd);
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(status, bits);
}


// One patch's coefficients for the batched preparation: checked, and
// converted to the arithmetic type (FP64 reads the caller's array).
struct BCoef {
  const double *c;
  float *c32;
  float2 *cdd;
  long long start, n;
};

__global__ void batch_coef_kernel(const BCoef *__restrict__ segs, int nseg, long long total, int prec,
                                  unsigned *status) {
  unsigned bits = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].start <= t) lo = mid; else hi = mid - 1;
    }
    const BCoef &S = segs[lo];
    bits |= wq::coef_point(S.c, (size_t)(t - S.start), prec, S.c32, S.cdd);
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(status, bits);
}

}  // namespace

struct wq_batch {
  int npatch = 0;
  wq_precision prec = WQ_FP64;
  int device = -1, nsm = 0, max_ctas = 1, max_uctas = 1;
  int deg_uctas[2] = {1, 1}, deg_ctas[2] = {1, 1};  // per degree (index p - 2): resident CTAs per SM
  std::vector<wq_patch> patches;
  // device block: fold segments, batch segments, per-patch folded tables and
  // U buffers, counters, status
  void *dev_block = nullptr;
  BFold *dev_fold = nullptr;
  int nfold = 0, fold_total = 0;
  BCoef *dev_coef = nullptr;  // the patches' coefficient preparation
  int ncoefseg = 0;
  long long coef_total = 0;
  // segments, degree 3 first; share[d] (d = p - 2) describes degree p's part
  wq::BatchUSeg *dev_usegs = nullptr;
  wq::BatchSeg *dev_segs = nullptr;
  struct Share {
    int useg0, nuseg, nuitems, seg0, nseg, nitems;
    size_t umap0, map0;  // offsets of the item -> segment tables in dev_map
  } share[2] = {};
  int *dev_map = nullptr;  // item -> segment (within the share), both kernels, both degrees
  size_t dev_map_cap = 0;
  unsigned *dev_counter = nullptr, *dev_status = nullptr;  // counters [2 per degree], status
  std::vector<wq::RowsArgs> base_args;  // per patch, without chunking
  std::vector<wq::UArgs> base_uargs;    // per patch
  // chunk length, CTAs per SM of the partial-contraction and of the row
  // kernels, schedule of the two degrees (0: side by side, 1: degree 3 first)
  int config[4] = {wq::kUGChunk, 1, 1, 1};
  cudaStream_t cap_stream = nullptr, aux_stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

wq_status prepare(wq_batch *B) {
  int uctas[2] = {0, 0}, ctas[2] = {0, 0};
  cudaError_t e = B->prec == WQ_FP64   ? wq::batch_prepare<double>(uctas, ctas)
                  : B->prec == WQ_MIXED ? wq::batch_prepare<float>(uctas, ctas)
                                        : wq::batch_prepare<wq::dd>(uctas, ctas);
  if (e != cudaSuccess) return WQ_ERR_CUDA;
  for (int d = 0; d < 2; d++) {
    if (ctas[d] < 1 || uctas[d] < 1) return WQ_ERR_CUDA;
    B->deg_uctas[d] = uctas[d];
    B->deg_ctas[d] = ctas[d];
  }
  B->max_uctas = std::max(uctas[0], uctas[1]);
  B->max_ctas = std::max(ctas[0], ctas[1]);
  return WQ_OK;
}

// Builds the two segment lists for the current configuration and uploads them.
wq_status build_segments(wq_batch *B) {
  const int tchunk = B->config[0];
  if (tchunk < 1 || tchunk > wq::kUGChunk) return WQ_ERR_ARG;
  std::vector<wq::BatchUSeg> usegs(B->npatch);
  std::vector<wq::BatchSeg> segs(B->npatch);
  for (int i = 0; i < B->npatch; i++) {
    const wq_rules *R = B->patches[i].rules;
    wq::BatchUSeg &U = usegs[i];
    std::memset(&U, 0, sizeof(U));
    U.a = B->base_uargs[i];
    U.p = R->p;
    U.nitems = R->n[2] * U.a.nblk2 * U.a.nblk1;
    const int T = wq::chunk_length(R, tchunk);
    if (wq::max_chunk_points(R, T) > wq::chunk_points_bound(R->p, wq::kUGChunk)) return WQ_ERR_UNSUPPORTED;
    wq::BatchSeg &S = segs[i];
    std::memset(&S, 0, sizeof(S));
    S.a = B->base_args[i];
    S.a.T = T;
    S.a.nch = (R->n[0] + T - 1) / T;
    S.p = R->p;
    S.nitems = R->n[1] * R->n[2] * S.a.nch;
  }
  // degree 3 first, patch order within a degree; items numbered per degree
  std::stable_sort(usegs.begin(), usegs.end(), [](const wq::BatchUSeg &x, const wq::BatchUSeg &y) { return x.p > y.p; });
  std::stable_sort(segs.begin(), segs.end(), [](const wq::BatchSeg &x, const wq::BatchSeg &y) { return x.p > y.p; });
  wq_batch::Share sh[2] = {};
  for (int d = 0; d < 2; d++) {
    const int p = d + 2;
    long long utotal = 0, total = 0;
    sh[d].useg0 = sh[d].seg0 = -1;
    for (int i = 0; i < B->npatch; i++) {
      if (usegs[i].p == p) {
        if (sh[d].useg0 < 0) sh[d].useg0 = i;
        sh[d].nuseg++;
        usegs[i].first_item = (int)utotal;
        utotal += usegs[i].nitems;
      }
      if (segs[i].p == p) {
        if (sh[d].seg0 < 0) sh[d].seg0 = i;
        sh[d].nseg++;
        segs[i].first_item = (int)total;
        total += segs[i].nitems;
      }
    }
    if (total > 0x7fffffffLL || utotal > 0x7fffffffLL) return WQ_ERR_UNSUPPORTED;
    if (sh[d].useg0 < 0) sh[d].useg0 = 0;
    if (sh[d].seg0 < 0) sh[d].seg0 = 0;
    sh[d].nuitems = (int)utotal;
    sh[d].nitems = (int)total;
  }
  // the item -> segment tables: per degree, its u items, then its rows items
  std::vector<int> map;
  for (int d = 0; d < 2; d++) {
    sh[d].umap0 = map.size();
    for (int k = 0; k < sh[d].nuseg; k++) map.insert(map.end(), usegs[sh[d].useg0 + k].nitems, k);
    sh[d].map0 = map.size();
    for (int k = 0; k < sh[d].nseg; k++) map.insert(map.end(), segs[sh[d].seg0 + k].nitems, k);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return WQ_ERR_CUDA;  // no launch still reads the old lists
  if (map.size() > B->dev_map_cap) {
    if (B->dev_map) cudaFree(B->dev_map);
    B->dev_map = nullptr;
    B->dev_map_cap = 0;
    if (cudaMalloc(&B->dev_map, map.size() * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return WQ_ERR_OOM;
    }
    B->dev_map_cap = map.size();
  }
  if (cudaMemcpy(B->dev_usegs, usegs.data(), usegs.size() * sizeof(wq::BatchUSeg), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(B->dev_segs, segs.data(), segs.size() * sizeof(wq::BatchSeg), cudaMemcpyHostToDevice) != cudaSuccess ||
      (!map.empty() &&
       cudaMemcpy(B->dev_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
    return WQ_ERR_CUDA;
  B->share[0] = sh[0];
  B->share[1] = sh[1];
  return WQ_OK;
}

// Degree p's share with the current configuration's grids.
wq::BatchShare share_of(const wq_batch *B, int p) {
  const int d = p - 2;
  const wq_batch::Share &h = B->share[d];
  wq::BatchShare S;
  S.usegs = B->dev_usegs + h.useg0;
  S.segs = B->dev_segs + h.seg0;
  S.useg_of = B->dev_map + h.umap0;
  S.seg_of = B->dev_map + h.map0;
  S.nuseg = h.nuseg;
  S.nuitems = h.nuitems;
  S.nseg = h.nseg;
  S.nitems = h.nitems;
  S.counters = B->dev_counter + 2 * d;
  S.ugrid = B->nsm * std::min(B->config[1], B->deg_uctas[d]);
  S.grid = B->nsm * std::min(B->config[2], B->deg_ctas[d]);
  return S;
}

cudaError_t launch_share(const wq_batch *B, int p, cudaStream_t s) {
  const wq::BatchShare S = share_of(B, p);
  if (S.nuitems == 0 && S.nitems == 0) return cudaSuccess;
  return B->prec == WQ_FP64    ? wq::launch_batch_share<double>(p, S, s)
         : B->prec == WQ_MIXED ? wq::launch_batch_share<float>(p, S, s)
                               : wq::launch_batch_share<wq::dd>(p, S, s);
}

wq_status enqueue(const wq_batch *B, cudaStream_t s) {
  if (B->fold_total > 0) {
    const int blocks = std::min((B->fold_total + 255) / 256, B->nsm * 8);
    batch_fold_kernel<<<blocks, 256, 0, s>>>(B->dev_fold, B->nfold, B->fold_total, B->dev_status);
    if (cudaGetLastError() != cudaSuccess) return WQ_ERR_CUDA;
  }
  if (B->coef_total > 0) {
    const int blocks = (int)std::min<long long>((B->coef_total + 255) / 256, (long long)B->nsm * 8);
    batch_coef_kernel<<<blocks, 256, 0, s>>>(B->dev_coef, B->ncoefseg, B->coef_total, (int)B->prec, B->dev_status);
    if (cudaGetLastError() != cudaSuccess) return WQ_ERR_CUDA;
  }
  if (cudaMemsetAsync(B->dev_counter, 0, 4 * sizeof(unsigned), s) != cudaSuccess) return WQ_ERR_CUDA;
  const bool both = B->share[0].nseg > 0 && B->share[1].nseg > 0;
  cudaError_t e = cudaSuccess;
  if (B->config[3] == 1 || !both) {
    e = launch_share(B, 3, s);
    if (e == cudaSuccess) e = launch_share(B, 2, s);
  } else {
    // degree 2 on the second stream, forked from and joined back into s
    e = cudaEventRecord(B->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->aux_stream, B->fork, 0);
    if (e == cudaSuccess) e = launch_share(B, 3, s);
    if (e == cudaSuccess) e = launch_share(B, 2, B->aux_stream);
    if (e == cudaSuccess) e = cudaEventRecord(B->join, B->aux_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, B->join, 0);
  }
  return e == cudaSuccess ? WQ_OK : WQ_ERR_CUDA;
}

void drop_graph(wq_batch *B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
}

// Captures fold + counter reset + the two persistent launches into a CUDA graph.
wq_status capture(wq_batch *B) {
  drop_graph(B);
  if (cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return WQ_ERR_CUDA;
  wq_status st = enqueue(B, B->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(B->cap_stream, &g);
  if (st != WQ_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return WQ_ERR_CUDA;
  }
  B->graph = g;
  if (cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) {
    drop_graph(B);
    return WQ_ERR_CUDA;
  }
  return WQ_OK;
}

wq_status apply_config(wq_batch *B, const int *cfg) {
  int old[4];
  std::memcpy(old, B->config, sizeof(old));
  std::memcpy(B->config, cfg, sizeof(old));
  if (B->config[1] < 1 || B->config[1] > B->max_uctas || B->config[2] < 1 || B->config[2] > B->max_ctas ||
      (B->config[3] != 0 && B->config[3] != 1)) {
    std::memcpy(B->config, old, sizeof(old));
    return WQ_ERR_ARG;
  }
  wq_status st = build_segments(B);
  if (st != WQ_OK) {
    std::memcpy(B->config, old, sizeof(old));
    build_segments(B);
    return st;
  }
  return capture(B);
}

// The autotuner cache's key: the GPU (name, compute capability, SMs), the
// precision, the occupancy limits of the compiled library's four kernels,
// the degree mix and a hash (64-bit FNV-1a) of the patches' shapes in plan
// order; empty on a CUDA error.
std::string cache_key(const wq_batch *B) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, B->device) != cudaSuccess) return std::string();
  int np2 = 0, np3 = 0;
  long long rows = 0;
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](long long v) {
    for (int i = 0; i < 8; i++) {
      h ^= (uint64_t)((v >> (8 * i)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  for (const wq_patch &P : B->patches) {
    const wq_rules *R = P.rules;
    (R->p == 2 ? np2 : np3)++;
    rows += (long long)R->n[0] * R->n[1] * R->n[2];
    mix(R->p);
    for (int a = 0; a < 3; a++) mix(R->nel[a]);
    mix(P.coef != nullptr);
  }
  char buf[384];
  std::snprintf(buf, sizeof(buf), "v2|%s|cc%d.%d|sm%d|%s|occ%d,%d,%d,%d|p2x%d,p3x%d|rows%lld|shape%016llx",
                prop.name, prop.major, prop.minor, prop.multiProcessorCount,
                B->prec == WQ_FP64 ? "fp64" : B->prec == WQ_MIXED ? "mixed" : "df64", B->deg_uctas[0],
                B->deg_uctas[1], B->deg_ctas[0], B->deg_ctas[1], np2, np3, rows, (unsigned long long)h);
  return wq::tune_cache_clean_key(buf);
}

void destroy(wq_batch *B) {
  if (!B) return;
  drop_graph(B);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  if (B->aux_stream) cudaStreamDestroy(B->aux_stream);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->join) cudaEventDestroy(B->join);
  if (B->dev_block) cudaFree(B->dev_block);
  if (B->dev_map) cudaFree(B->dev_map);
  delete B;
}

}  // namespace

extern "C" {

wq_status wq_batch_create(const wq_patch *patches, int npatch, wq_precision prec, wq_batch **out) {
  if (!out) return WQ_ERR_ARG;
  *out = nullptr;
  if (!patches || npatch < 1) return WQ_ERR_ARG;
  if (prec != WQ_FP64 && prec != WQ_MIXED && prec != WQ_DF64) return WQ_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return WQ_ERR_CUDA;
  for (int i = 0; i < npatch; i++) {
    const wq_patch &P = patches[i];
    const wq_rules *R = P.rules;
    if (!R || !R->on_device || R->device != dev || R->dim != 3 || R->mode != wq::kModeWQ) return WQ_ERR_ARG;
    if (R->bnd_weighted) return WQ_ERR_UNSUPPORTED;
    if (!P.M || !P.K || !P.geom[0] || !P.geom[1] || !P.geom[2]) return WQ_ERR_ARG;
  }
  wq_batch *B = new (std::nothrow) wq_batch();
  if (!B) return WQ_ERR_OOM;
  B->npatch = npatch;
  B->prec = prec;
  B->device = dev;
  B->patches.assign(patches, patches + npatch);
  if (cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    destroy(B);
    return WQ_ERR_CUDA;
  }
  wq_status st = prepare(B);
  if (st != WQ_OK) {
    destroy(B);
    return st;
  }
  // device block layout
  size_t total = 0;
  const size_t fold_off = total;
  total += align_up(sizeof(BFold) * 6 * (size_t)npatch);
  const size_t coefseg_off = total;
  total += align_up(sizeof(BCoef) * (size_t)npatch);
  const size_t useg_off = total;
  total += align_up(sizeof(wq::BatchUSeg) * (size_t)npatch);
  const size_t seg_off = total;
  total += align_up(sizeof(wq::BatchSeg) * (size_t)npatch);
  const size_t cnt_off = total;
  total += align_up(5 * sizeof(unsigned));
  const size_t elem_bytes = prec == WQ_MIXED ? sizeof(float) : sizeof(double);
  std::vector<size_t> tab_off(6 * (size_t)npatch), u_off(npatch), c_off(npatch, 0);
  for (int i = 0; i < npatch; i++) {
    const wq_rules *R = patches[i].rules;
    const size_t np = (size_t)R->p + 1;
    for (int a = 0; a < 3; a++)
      for (int k = 0; k < 2; k++) {
        tab_off[(size_t)i * 6 + a * 2 + k] = total;
        const size_t m = (size_t)R->dev[a][k].npts * np;
        total += align_up(m * sizeof(double)) + align_up(m * sizeof(float)) + align_up(m * sizeof(float2));
      }
    // the patch's own U buffer (patches may share a rules object)
    const size_t nb = 2 * (size_t)R->p + 1;
    u_off[i] = total;
    total += align_up((size_t)R->n[1] * R->n[2] * 2 * R->nc[0] * nb * nb * elem_bytes);
    // the patch's coefficients in the arithmetic type (FP64 reads the caller's)
    if (patches[i].coef && prec != WQ_FP64) {
      c_off[i] = total;
      total += align_up((size_t)R->nc[0] * R->nc[1] * R->nc[2] * (prec == WQ_MIXED ? sizeof(float) : sizeof(float2)));
    }
  }
  if (cudaMalloc(&B->dev_block, total) != cudaSuccess) {
    cudaGetLastError();
    destroy(B);
    return WQ_ERR_OOM;
  }
  char *base = static_cast<char *>(B->dev_block);
  B->dev_fold = reinterpret_cast<BFold *>(base + fold_off);
  B->dev_coef = reinterpret_cast<BCoef *>(base + coefseg_off);
  std::vector<BCoef> coefs;
  B->dev_usegs = reinterpret_cast<wq::BatchUSeg *>(base + useg_off);
  B->dev_segs = reinterpret_cast<wq::BatchSeg *>(base + seg_off);
  B->dev_counter = reinterpret_cast<unsigned *>(base + cnt_off);
  B->dev_status = B->dev_counter + 4;
  std::vector<BFold> folds;
  int start = 0;
  B->base_args.resize(npatch);
  B->base_uargs.resize(npatch);
  for (int i = 0; i < npatch; i++) {
    const wq_patch &P = patches[i];
    const wq_rules *R = P.rules;
    const size_t np = (size_t)R->p + 1;
    wq::RowsArgs &ra = B->base_args[i];
    std::memset(&ra, 0, sizeof(ra));
    ra.bnd_grouped = 1;  // Gauss-Legendre boundary rows
    for (int a = 0; a < 3; a++) {
      for (int k = 0; k < 2; k++) {
        const wq::DevDirKind &Dk = R->dev[a][k];
        const size_t m = (size_t)Dk.npts * np;
        char *t = base + tab_off[(size_t)i * 6 + a * 2 + k];
        double *v64 = reinterpret_cast<double *>(t);
        float *v32 = reinterpret_cast<float *>(t + align_up(m * sizeof(double)));
        float2 *vdd = reinterpret_cast<float2 *>(t + align_up(m * sizeof(double)) + align_up(m * sizeof(float)));
        BFold F;
        F.elem = Dk.elem;
        F.w = Dk.w;
        F.t0 = Dk.t0;
        F.t1 = Dk.t1;
        F.g = P.geom[a];
        F.v64 = v64;
        F.v32 = v32;
        F.vdd = vdd;
        F.start = start;
        F.np = (int)np;
        F.kind = k;
        start += Dk.npts;
        folds.push_back(F);
        ra.off[a][k] = Dk.off;
        ra.elem[a][k] = Dk.elem;
        ra.V[a][k] = prec == WQ_FP64 ? (const void *)v64 : prec == WQ_MIXED ? (const void *)v32 : (const void *)vdd;
        ra.beta[a][k] = prec == WQ_FP64   ? (const void *)Dk.beta
                        : prec == WQ_MIXED ? (const void *)Dk.beta32 : (const void *)Dk.betadd;
      }
      ra.n[a] = R->n[a];
      ra.N[a] = R->nel[a];
      ra.nc[a] = R->nc[a];
    }
    ra.coef = P.coef;
    ra.coefR = nullptr;  // the row kernel reads U, not the coefficients
    ra.M = P.M;
    ra.K = P.K;
    ra.row_begin = 0;
    ra.row_end = (long long)R->n[0] * R->n[1] * R->n[2];
    ra.lines = nullptr;
    ra.line0 = 0;
    ra.Ug = base + u_off[i];
    ra.status = B->dev_status;
    wq::UArgs &ua = B->base_uargs[i];
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
    ua.coef = P.coef;
    ua.coefR = nullptr;
    if (P.coef) {
      const long long nco = (long long)R->nc[0] * R->nc[1] * R->nc[2];
      BCoef C;
      C.c = P.coef;
      C.c32 = prec == WQ_MIXED ? reinterpret_cast<float *>(base + c_off[i]) : nullptr;
      C.cdd = prec == WQ_DF64 ? reinterpret_cast<float2 *>(base + c_off[i]) : nullptr;
      C.start = B->coef_total;
      C.n = nco;
      B->coef_total += nco;
      coefs.push_back(C);
      ua.coefR = prec == WQ_FP64 ? (const void *)P.coef : (const void *)(base + c_off[i]);
    }
    ua.U = base + u_off[i];
    ua.line_lo = 0;
    ua.line_hi = R->n[1] * R->n[2] - 1;
    ua.r3_lo = 0;
    ua.nblk2 = (R->n[1] + wq::kULines - 1) / wq::kULines;
    ua.nblk1 = (R->nc[0] + wq::kUCols - 1) / wq::kUCols;
    ua.status = B->dev_status;
  }
  B->nfold = (int)folds.size();
  B->fold_total = start;
  B->ncoefseg = (int)coefs.size();
  bool ok = cudaMemcpy(B->dev_fold, folds.data(), folds.size() * sizeof(BFold), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && (coefs.empty() || cudaMemcpy(B->dev_coef, coefs.data(), coefs.size() * sizeof(BCoef),
                                          cudaMemcpyHostToDevice) == cudaSuccess);
  ok = ok && cudaMemset(B->dev_counter, 0, 5 * sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&B->aux_stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    destroy(B);
    return WQ_ERR_CUDA;
  }
  const int cfg[4] = {wq::kUGChunk, B->max_uctas, B->max_ctas, 1};
  st = apply_config(B, cfg);
  if (st != WQ_OK) {
    destroy(B);
    return st;
  }
  *out = B;
  return WQ_OK;
}

void wq_batch_free(wq_batch *batch) {
  if (!batch) return;
  const int dev = batch->device;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  destroy(batch);
  if (cur >= 0 && cur != dev) cudaSetDevice(cur);
}

wq_status wq_batch_launch(wq_batch *B, void *stream) {
  wq::TraceRange trace("wq_batch_launch");
  if (!B || !B->exec) return WQ_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != B->device) return WQ_ERR_ARG;
  return cudaGraphLaunch(B->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? WQ_OK : WQ_ERR_CUDA;
}

wq_status wq_batch_status(wq_batch *B, void *stream) {
  if (!B) return WQ_ERR_ARG;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return WQ_ERR_CUDA;
  unsigned bits = 0;
  if (cudaMemcpy(&bits, B->dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return WQ_ERR_CUDA;
  if (cudaMemset(B->dev_status, 0, sizeof(unsigned)) != cudaSuccess) return WQ_ERR_CUDA;
  if (bits & wq::kBitChecked) return WQ_ERR_CHECK;
  if (bits & wq::kBitNonFinite) return WQ_ERR_NONFINITE;
  if (bits & wq::kBitGeometry) return WQ_ERR_GEOMETRY;
  return WQ_OK;
}

wq_status wq_batch_get_config(const wq_batch *B, int *config) {
  if (!B || !config) return WQ_ERR_ARG;
  std::memcpy(config, B->config, sizeof(B->config));
  config[4] = B->max_uctas;
  config[5] = B->max_ctas;
  return WQ_OK;
}

wq_status wq_batch_set_config(wq_batch *B, const int *config) {
  if (!B || !config) return WQ_ERR_ARG;
  return apply_config(B, config);
}

wq_status wq_batch_tune(wq_batch *B, void *stream, int reps, double *best_ms) {
  if (!B || reps < 1) return WQ_ERR_ARG;
  const char *cache = std::getenv("WQ_AUTOTUNE_CACHE");
  std::string key;
  if (cache && *cache) {
    key = cache_key(B);
    int cfg[4];
    double ms = 0.0;
    // a cached configuration the plan cannot take (another build's CTA
    // limits, a chunk its tables do not fit) is timed again
    if (!key.empty() && wq::tune_cache_lookup(cache, key, cfg, &ms) && apply_config(B, cfg) == WQ_OK) {
      if (best_ms) *best_ms = ms;
      return WQ_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int chunks[] = {32, 24, 16};
  std::vector<int> ctas, uctas;
  for (int c = B->max_ctas; c >= 1 && (int)ctas.size() < 2; c--) ctas.push_back(c);
  for (int c = B->max_uctas; c >= 1 && (int)uctas.size() < 2; c--) uctas.push_back(c);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return WQ_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return WQ_ERR_CUDA;
  }
  int best[4];
  std::memcpy(best, B->config, sizeof(best));
  float best_t = -1.0f;
  wq_status st = WQ_OK;
  for (int sched = 0; sched < 2 && st == WQ_OK; sched++)
    for (int uc : uctas)
      for (int c : ctas)
        for (int t : chunks) {
          if (st != WQ_OK) break;
          const int cfg[4] = {t, uc, c, sched};
          std::memcpy(B->config, cfg, sizeof(cfg));
          if (build_segments(B) != WQ_OK) continue;  // a chunk length this batch's tables do not fit
          st = enqueue(B, s);  // warm-up
          float tsum = 0.0f;
          for (int r = 0; r < reps && st == WQ_OK; r++) {
            cudaEventRecord(e0, s);
            st = enqueue(B, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = WQ_ERR_CUDA;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            tsum += ms;
          }
          if (st == WQ_OK && (best_t < 0.0f || tsum / reps < best_t)) {
            best_t = tsum / reps;
            std::memcpy(best, cfg, sizeof(best));
          }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != WQ_OK) return st;
  if (best_ms) *best_ms = best_t;
  st = apply_config(B, best);
  if (st == WQ_OK && !key.empty()) wq::tune_cache_store(cache, key, best, best_t);  // best effort
  return st;
}

wq_status wq_assemble_batch(const wq_patch *patches, int npatch, wq_precision prec, void *stream) {
  wq_batch *B = nullptr;
  wq_status st = wq_batch_create(patches, npatch, prec, &B);
  if (st != WQ_OK) return st;
  st = wq_batch_launch(B, stream);
  if (st == WQ_OK) st = wq_batch_status(B, stream);
  wq_batch_free(B);
  return st;
}

}  // extern "C"
