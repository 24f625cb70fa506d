// Internal data structures of libwq (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/wq.h"
#include "checked.cuh"

namespace wq {

// A named NVTX range around one entry point's host work and launches (for
// profilers that filter by range; a no-op when no tool is attached).
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

constexpr int kMaxP = 3;
constexpr int kMaxDim = 3;
constexpr int kMaxRowPts = kMaxP * (kMaxP + 1);  // most points of one row in one direction
constexpr int kCoefDeg = 3;                      // the coefficient field is a cubic spline
constexpr int kMaxNel = 1 << 16;

// Rule modes (wq_rules_build flags): the method, and the two comparison rules.
constexpr int kModeWQ = 0, kModeGL = 1, kModeNC = 2;

// Status bits raised by the kernels: checked.cuh.

// One direction and one kind (mass or stiffness) of the 1D row rules.
// Point q of row r lies in element elem[q]; the p+1 B-splines acting there
// are B_{elem+i}, i = 0..p; the cubic coefficient splines acting there are
// B3_{elem+i}, i = 0..3.
struct HostDirKind {
  std::vector<int> off;      // n+1 offsets into the point arrays
  std::vector<int> elem;     // npts
  std::vector<double> x;     // npts
  std::vector<double> w;     // npts: W = h * omega * B_r^(nu)(x)
  std::vector<double> t0;    // npts*(p+1): B_{elem+i}(x)
  std::vector<double> t1;    // npts*(p+1): B'_{elem+i}(x)
  std::vector<double> beta;  // npts*4: B3_{elem+i}(x)
  std::vector<double> tl;    // npts*p: B_{elem+1+j, p-1}(x), degree p-1 on the same knots
};

// One direction of the mixed-derivative kinds (kind 2: weight B_r', tests
// B_s; kind 3: weight B_r, tests B_s'), which share their points; offsets,
// point counts and elements per row equal the mass kind's.
struct HostCross {
  std::vector<int> off, elem;
  std::vector<double> x;
  std::vector<double> w2, w3;  // combined weights of kinds 2 and 3
  std::vector<double> t0, t1;  // npts*(p+1): B_{elem+i}(x), B'_{elem+i}(x)
  std::vector<double> beta;    // npts*4: B3_{elem+i}(x)
  std::vector<double> tl;      // npts*p: B_{elem+1+j, p-1}(x)
};

struct DevCross {
  const int *elem;
  const double *w2, *w3, *t0, *t1, *beta, *tl;
  int npts;
};

// Derived tables of one direction for maps given by a full control net:
// per point set (m, s, x) the degree-p values, degree p-1 values and cubic
// values in FP32 (the FP32 Jacobian reads no double), and per weight-test
// kind 0..3 the products W(q) T(q, i) of each point's weight and its p+1
// test values, in FP64 and FP32.
struct GmDevTab {
  const float *t0f[3], *tlf[3], *betaf[3];
  const double *wt64[4];
  const float *wt32[4];
};

// Device view of one direction and kind (all arrays in device memory).
struct DevDirKind {
  const int *off;
  const int *elem;
  const double *w;
  const double *t0;
  const double *t1;
  const double *beta;
  double *v64;  // folded tables, npts*(p+1): W*|J| B (mass), W/|J| B' (stiffness)
  float *v32;   // the same rounded to float
  float *beta32;
  float2 *vdd;     // the folded tables as double-float pairs (hi, lo)
  float2 *betadd;  // the cubic values as double-float pairs
  const double *tl;  // npts*p: degree p-1 values (non-separable maps, FP32 Jacobian)
  int npts;
};

struct Lines {
  std::vector<int> interior, boundary;  // sorted line ids (r2 + n2*r3, or r2 for dim 2)
};

}  // namespace wq

struct wq_rules {
  wq_mesh mesh;
  int p = 0, dim = 0;
  int mode = 0;  // 0: weighted Gaussian rules; 1: Gauss-Legendre rows; 2: Newton-Cotes-type rows
  // mode 0 with weighted Gaussian rules for the boundary rows as well
  // (WQ_RULES_BOUNDARY_WEIGHTED): their points are padded per element so that
  // both kinds have the same elements point by point
  bool bnd_weighted = false;
  int nel[3] = {1, 1, 1};
  int n[3] = {1, 1, 1};
  int nc[3] = {1, 1, 1};
  double tau[2][wq::kMaxP + 1] = {};
  double omega[2][wq::kMaxP + 1] = {};
  wq::HostDirKind host[3][2];
  wq::HostCross hostx[3];  // mode 0 without boundary weighted rules only
  wq::Lines lines;
  // device side
  bool on_device = false;
  int device = -1;
  void *dev_block = nullptr;
  size_t dev_bytes = 0;
  wq::DevDirKind dev[3][2] = {};
  const int *dev_lines_interior = nullptr;
  const int *dev_lines_boundary = nullptr;
  unsigned *dev_status = nullptr;
  float *dev_coef32 = nullptr;   // the coefficients rounded to float (mixed mode)
  float2 *dev_coefdd = nullptr;  // the coefficients as double-float pairs (df64 mode)
  void *dev_U = nullptr;         // 3D: the partial contractions U of every line, [line][2][nc1][(2p+1)^2], 8-byte
                                 // elements (the split assembly path; its own allocation)
  wq::DevCross devx[3] = {};      // device copy of hostx (its own allocation, dev_cross)
  void *dev_cross = nullptr;
  wq::GmDevTab gmt[3] = {};       // derived tables of the non-separable path (allocation dev_gmtab)
  void *dev_gmtab = nullptr;
  // scratch of the non-separable assembly (the metric factors of a slab of
  // rows), allocated by the first call that needs it, grown when needed
  mutable void *dev_gm = nullptr;
  mutable size_t dev_gm_bytes = 0;
  // the adjoint's per-chunk coefficient blocks (FP64), allocated by the first
  // wq_assemble_adjoint call that needs them and grown when a call needs more
  mutable double *dev_adj = nullptr;
  mutable size_t dev_adj_bytes = 0;
};

namespace wq {
// rules.cpp
wq_status solve_rule(int p, int kind, const double *start, double *tau, double *omega);
wq_status default_rule(int p, int kind, double *tau, double *omega);
wq_status build_host_tables(wq_rules *R);
wq_status nc_rule(int p, int kind, double *y, double *v);
// Chunk length for lines of n1 rows and a capacity of tmax rows: the even
// split ceil(n1 / ceil(n1 / tmax)).
int chunk_length(const wq_rules *R, int tmax);
// Most x1 points one chunk holds when lines are cut into chunks of T rows
// (the last one ragged), as the launches cut them.
int max_chunk_points(const wq_rules *R, int T);
// Boundary row r < p of kind: the weighted Gaussian rule in units of h (x =
// t h from the low end, W = Wl h^(1-kind)); WQ_ERR_UNSUPPORTED where none is
// defined (Gauss-Legendre is used there).
wq_status boundary_rule(int p, int kind, int r, double *t, double *Wl, int *npts);
// The mixed-derivative rules on the cardinal support: nodes y, kind 2
// weights w (weight N', tests N), kind 3 weights v (weight N, tests N').
wq_status mixed_rule(int p, double *y, double *w, double *v);
// tune_cache.cpp: the batch autotuner's cache file (one JSON entry per line)
std::string tune_cache_clean_key(const std::string &raw);
bool tune_cache_lookup(const char *path, const std::string &key, int cfg[4], double *ms);
bool tune_cache_store(const char *path, const std::string &key, const int cfg[4], double ms);
double flop_count(const wq_rules *R, int want_m, int want_k, int64_t row_begin, int64_t row_end,
                  double *coef_flops);
}  // namespace wq
