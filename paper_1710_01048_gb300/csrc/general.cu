// Assembly for maps given by a full control net (Eq. Gmap1): the metric
// C = c |det J| J^-1 J^-T (Eq. Stiffness) is no longer diagonal, nor a
// product of 1D factors, so it is evaluated point by point.
//
// K_rs = sum over a, b of int dB_r/dxhat_a C_ab dB_s/dxhat_b, each term with
// the tensor product of one 1D rule per direction d: the stiffness rule
// where d = a = b (Eq. GaussQuadSysStiff), the mixed rule of kind 2 (weight
// B_r', tests B_s) where d = a != b, that of kind 3 (weight B_r, tests B_s')
// where d = b != a, the mass rule (Eq. GaussQuadSys) elsewhere; M with the
// mass rule in every direction and the factor c |det J|.  Kinds 2 and 3
// share their points, so the terms live on seven point grids (five in 2D):
//   g0 (m,m,m): c|det J|   g1 (s,m,m): C11   g2 (m,s,m): C22   g3 (m,m,s): C33
//   g4 (x,x,m): C12        g5 (x,m,x): C13   g6 (m,x,x): C23
// (m, s, x: the mass, stiffness and mixed point sets of a direction).  Every
// point of a grid belongs to exactly one row (each row has its own points),
// so no work is shared between rows except the map's partial contractions.
//
// gm_metric3_kernel evaluates the factors of one slab of x3 planes into a
// scratch array: a CTA takes one x3 point q3, one x2 row r2 and a chunk of
// x1 points of one (x2, x3) point-kind pair, contracts the control net over
// x3 (H, shared by the row's x2 points) and x2 (E), then forms the Jacobian,
// the coefficient and the metric entry at every point of the chunk.
// gm_rows_kernel assembles one row per warp from its points' factors by sum
// factorisation, x3 first: per term X = F A3, Y += X A2 over the terms of
// equal direction-1 kind, band += Y A1 (Eq. Decompo).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <type_traits>
#include <cstring>
#include <vector>

#include "checked.cuh"
#include "wq_internal.h"

namespace wq {
namespace {

constexpr int kGmChunk = 128;                   // x1 points per metric item
// x1 control / coefficient columns one chunk of kGmChunk points can touch:
// every row has at least p+1 points (its weighted rule, or p+1 Gauss-Legendre
// points per element), so a chunk spans at most ceil((kGmChunk-1)/(p+1)) + 1
// rows r_a..r_b, whose points lie in elements r_a-p .. r_b; their control
// columns are r_a-p .. r_b+p and coefficient columns r_a-p .. r_b+3
template <int P> constexpr int gm_cols() { return kGmChunk / (P + 1) + 2 * P + 5; }
constexpr int kGmWarps = 4;                     // rows (warps) per CTA of the row kernel
constexpr int kGmGrids = 7;
constexpr int kGmRows64 = 2, kGmRows32 = 4;  // x2 rows per 3D metric item (FP64, FP32)

struct GmTab {  // one direction, one point set (m, s, x): what the metric reads
  const int *elem;
  const double *t0, *t1, *beta, *tl;
  const float *t0f, *tlf, *betaf;  // the same in FP32 (the FP32 Jacobian)
};

struct GmArgs {
  int dim;
  int n[3], N[3], nc[3], np[3];
  const int *off[3];        // row offsets into the point lists (equal for every kind)
  GmTab tab[3][3];          // [direction][point set m, s, x]
  // [direction][weight-test kind 0..3]: W(q) T(q, i), the combined weight
  // times each of the point's p+1 test values (FP64 and FP32)
  const double *WT64[3][4];
  const float *WT32[3][4];
  const double *net;        // dim components of ntot control values
  long long ntot;
  const double *coef;       // may be null: c = 1
  void *F;                  // kGmGrids factor arrays of fstride values (double or float)
  const float *D;           // FP32 path: scaled differences of the net, [b][a][ntot]
  const float *coef32;      // FP32 path: the coefficients in FP32 (null: c = 1)
  long long fstride;
  int slab_lo, slab_n;      // 3D: x3 points [slab_lo, slab_lo + slab_n); 2D: x2 points
  int bp_lo, bp_hi;         // the slab's planes (2D: lines) [bp_lo, bp_hi]
  long long row_begin, row_end, out_row0, out_rows;  // slab rows; the call's first row and row count
  void *M, *K;              // bands, double or float
  unsigned *status;
};

// Point-set pairs (x2, x3) of the metric groups and, per group, the x1 point
// sets and the grid each feeds.  Component codes: 0 = c|det J|, else 1 + 3a + b.
struct GmGroup {
  int k2, k3, ng;
  int k1[2], grid[2], comp[2];
};
__constant__ GmGroup c_groups3[6] = {
    {0, 0, 2, {0, 1}, {0, 1}, {0, 1 + 0}},  // (m,m): g0 mass, g1 C11
    {1, 0, 1, {0, 0}, {2, 2}, {1 + 4, 0}},  // (s,m): g2 C22
    {0, 1, 1, {0, 0}, {3, 3}, {1 + 8, 0}},  // (m,s): g3 C33
    {2, 0, 1, {2, 0}, {4, 4}, {1 + 1, 0}},  // (x,m): g4 C12
    {0, 2, 1, {2, 0}, {5, 5}, {1 + 2, 0}},  // (m,x): g5 C13
    {2, 2, 1, {0, 0}, {6, 6}, {1 + 5, 0}},  // (x,x): g6 C23
};
__constant__ GmGroup c_groups2[3] = {
    {0, 0, 2, {0, 1}, {0, 1}, {0, 1 + 0}},  // (m): g0 mass, g1 C11
    {1, 0, 1, {0, 0}, {2, 2}, {1 + 4, 0}},  // (s): g2 C22
    {2, 0, 1, {2, 0}, {4, 4}, {1 + 1, 0}},  // (x): g4 C12
};

// Terms of K (and M): grid and weight-test kind per direction; grouped by the
// direction-1 kind so that each group shares the last contraction.
struct GmTerm {
  int grid, k[3];
};
__constant__ GmTerm c_terms3[10] = {
    {0, {0, 0, 0}},                                 // M
    {2, {0, 1, 0}}, {3, {0, 0, 1}}, {6, {0, 2, 3}}, {6, {0, 3, 2}},  // direction-1 kind 0: K22 K33 K23 K32
    {1, {1, 0, 0}},                                 // kind 1: K11
    {4, {2, 3, 0}}, {5, {2, 0, 3}},                 // kind 2: K12 K13
    {4, {3, 2, 0}}, {5, {3, 0, 2}},                 // kind 3: K21 K31
};
__constant__ int c_group_start3[6] = {0, 1, 5, 6, 8, 10};
__constant__ GmTerm c_terms2[5] = {
    {0, {0, 0, 0}},  // M
    {2, {0, 1, 0}},  // K22
    {1, {1, 0, 0}},  // K11
    {4, {2, 3, 0}},  // K12
    {4, {3, 2, 0}},  // K21
};
__constant__ int c_group_start2[6] = {0, 1, 2, 3, 4, 5};

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 cross3(const V3 &u, const V3 &v) {
  return V3{fma(u.y, v.z, -u.z * v.y), fma(u.z, v.x, -u.x * v.z), fma(u.x, v.y, -u.y * v.x)};
}
__device__ __forceinline__ double dot3(const V3 &u, const V3 &v) { return fma(u.x, v.x, fma(u.y, v.y, u.z * v.z)); }

// The metric entry `comp` at one point from the Jacobian columns j0..j2
// (3D): the rows of det * J^-1 are j1 x j2, j2 x j0, j0 x j1, so
// c |det J| (J^-1 J^-T)_ab = c (row_a . row_b) / |det J|.  comp is uniform
// over the CTA (one group per CTA).
__device__ __forceinline__ double metric3(int comp, const V3 &j0, const V3 &j1, const V3 &j2, double c,
                                          unsigned &bits) {
  const V3 a0 = cross3(j1, j2);
  const double det = dot3(j0, a0);
  if (!(det > 0.0)) bits |= isfinite(det) ? kBitGeometry : kBitNonFinite;
  const double adet = fabs(det);
  if (comp == 0) return c * adet;
  const int a = (comp - 1) / 3, b = (comp - 1) % 3;
  V3 ra, rb;
  if (a == 0)
    ra = a0;
  else if (a == 1)
    ra = cross3(j2, j0);
  else
    ra = cross3(j0, j1);
  if (b == a)
    rb = ra;
  else if (b == 1)
    rb = cross3(j2, j0);
  else
    rb = cross3(j0, j1);
  return c * dot3(ra, rb) / adet;
}

// 2D: J = [j0 j1] (columns), det J^-1 rows r0 = (j1.y, -j1.x), r1 = (-j0.y, j0.x).
__device__ __forceinline__ double metric2(int comp, const double *j0, const double *j1, double c, unsigned &bits) {
  const double det = fma(j0[0], j1[1], -j1[0] * j0[1]);
  if (!(det > 0.0)) bits |= isfinite(det) ? kBitGeometry : kBitNonFinite;
  const double adet = fabs(det);
  if (comp == 0) return c * adet;
  const int a = (comp - 1) / 3, b = (comp - 1) % 3;
  const double ra[2] = {a == 0 ? j1[1] : -j0[1], a == 0 ? -j1[0] : j0[0]};
  const double rb[2] = {b == 0 ? j1[1] : -j0[1], b == 0 ? -j1[0] : j0[0]};
  return c * fma(ra[0], rb[0], ra[1] * rb[1]) / adet;
}

// Smallest of vlo and largest of vhi over the CTA (every thread takes part).
__device__ __forceinline__ void block_minmax(int vlo, int vhi, int &vmin, int &vmax, int *sred) {
  int lo = __reduce_min_sync(0xffffffffu, vlo), hi = __reduce_max_sync(0xffffffffu, vhi);
  if (threadIdx.x == 0) {
    sred[0] = 0x7fffffff;
    sred[1] = -1;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&sred[0], lo);
    atomicMax(&sred[1], hi);
  }
  __syncthreads();
  vmin = sred[0];
  vmax = sred[1];
}

// Shared memory of the 3D metric kernel (doubles): H of the two x3 patterns
// [2][3][R2B+2P][kGmCols], the coefficient's Hc [R2B+P+3][kGmCols], E [10][kGmCols].
template <int P> constexpr int metric3_smem_doubles() {
  constexpr int kGmCols = gm_cols<P>();
  return 2 * 3 * (kGmRows64 + 2 * P) * kGmCols + (kGmRows64 + P + 3) * kGmCols + 10 * kGmCols;
}

template <int P> __global__ void __launch_bounds__(kGmChunk) gm_metric3_kernel(const GmArgs A) {
  constexpr int kGmCols = gm_cols<P>();
  constexpr int NP = P + 1, R2B = kGmRows64, NI2 = R2B + 2 * P, NL2 = R2B + P + 3, NT = kGmChunk;
  extern __shared__ double sm[];
  double *sHv = sm;                      // [a][i2][col]
  double *sHd = sHv + 3 * NI2 * kGmCols;  // [a][i2][col]
  double *sHc = sHd + 3 * NI2 * kGmCols;  // [l2][col]
  double *sE = sHc + NL2 * kGmCols;       // [vv0..2, dv0..2, vd0..2, c][col]
  __shared__ int sred[2];
  const int tid = threadIdx.x;
  const int np1 = A.np[0], np2 = A.np[1];
  const int nch1 = (np1 + NT - 1) / NT;
  long long item = blockIdx.x;
  const int c1 = (int)(item % nch1);
  item /= nch1;
  const int nb2 = (A.n[1] + R2B - 1) / R2B;
  const int r2a = (int)(item % nb2) * R2B, r2b = min(A.n[1], r2a + R2B) - 1;
  item /= nb2;
  const int q3l = (int)(item % A.slab_n);
  const GmGroup &grp = c_groups3[(int)(item / A.slab_n)];  // read in place (no local copy)
  const int q3 = A.slab_lo + q3l;

  // the x3 point: element and basis values
  const GmTab &T3 = A.tab[2][grp.k3];
  const int e3 = T3.elem[q3];
  double b3v[NP], b3d[NP], c3[4];
#pragma unroll
  for (int i = 0; i < NP; i++) {
    b3v[i] = T3.t0[(size_t)q3 * NP + i];
    b3d[i] = T3.t1[(size_t)q3 * NP + i];
  }
#pragma unroll
  for (int l = 0; l < 4; l++) c3[l] = T3.beta[(size_t)q3 * 4 + l];

  // the chunk's x1 points and the columns they touch (all point sets share elements)
  const int qa = c1 * NT, qb = min(np1, qa + NT);
  const int *elem1 = A.tab[0][0].elem;
  const int myq = qa + tid;
  int emin, emax;
  block_minmax(myq < qb ? elem1[myq] : 0x7fffffff, myq < qb ? elem1[myq] : -1, emin, emax, sred);
  const int ni1 = emax + P - emin + 1, nl1 = emax + 3 - emin + 1;
  if (ni1 > kGmCols || nl1 > kGmCols) {  // cannot happen (see gm_cols); reported, nothing written
    if (tid == 0) atomicOr(A.status, kBitInternal);
    return;
  }
  // the x2 rows' elements and the control / coefficient rows they touch
  const int e2lo = max(0, r2a - P), e2hi = min(A.N[1] - 1, r2b);
  const int ni2 = e2hi + P - e2lo + 1, nl2 = e2hi + 3 - e2lo + 1;
  const int n1 = A.n[0], n2 = A.n[1], nc1 = A.nc[0], nc2 = A.nc[1];

  // H: contraction of the net over the x3 point's p+1 control layers
  for (int t = tid; t < ni2 * ni1; t += NT) {
    const int i2 = e2lo + t / ni1, col = t % ni1, i1 = emin + col;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const double *g = A.net + a * A.ntot + i1 + (long long)n1 * i2;
      double hv = 0.0, hd = 0.0;
#pragma unroll
      for (int i = 0; i < NP; i++) {
        const double x = g[(long long)n1 * n2 * (e3 + i)];
        hv = fma(x, b3v[i], hv);
        hd = fma(x, b3d[i], hd);
      }
      sHv[(a * NI2 + (i2 - e2lo)) * kGmCols + col] = hv;
      sHd[(a * NI2 + (i2 - e2lo)) * kGmCols + col] = hd;
    }
  }
  if (A.coef)
    for (int t = tid; t < nl2 * nl1; t += NT) {
      const int l2 = e2lo + t / nl1, col = t % nl1, l1 = emin + col;
      const double *g = A.coef + l1 + (long long)nc1 * l2;
      double hc = 0.0;
#pragma unroll
      for (int l = 0; l < 4; l++) hc = fma(g[(long long)nc1 * nc2 * (e3 + l)], c3[l], hc);
      sHc[(l2 - e2lo) * kGmCols + col] = hc;
    }
  __syncthreads();

  unsigned bits = 0;
  const GmTab &T2 = A.tab[1][grp.k2];
  const int q2a = A.off[1][r2a], q2b = A.off[1][r2b + 1];
  for (int q2 = q2a; q2 < q2b; q2++) {
    const int e2 = T2.elem[q2];
    double b2v[NP], b2d[NP], c2[4];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      b2v[i] = T2.t0[(size_t)q2 * NP + i];
      b2d[i] = T2.t1[(size_t)q2 * NP + i];
    }
#pragma unroll
    for (int l = 0; l < 4; l++) c2[l] = T2.beta[(size_t)q2 * 4 + l];
    // E: the x2 contraction at this x2 point, one (component, column) per
    // thread, then the coefficient's columns
    const int nE = 3 * ni1 + (A.coef ? nl1 : 0);
    for (int t = tid; t < nE; t += NT) {
      if (t < 3 * ni1) {
        const int a = t / ni1, col = t - a * ni1;
        double vv = 0.0, dv = 0.0, vd = 0.0;
#pragma unroll
        for (int i = 0; i < NP; i++) {
          const int row = (a * NI2 + (e2 - e2lo + i)) * kGmCols + col;
          vv = fma(sHv[row], b2v[i], vv);
          dv = fma(sHv[row], b2d[i], dv);
          vd = fma(sHd[row], b2v[i], vd);
        }
        sE[a * kGmCols + col] = vv;
        sE[(3 + a) * kGmCols + col] = dv;
        sE[(6 + a) * kGmCols + col] = vd;
      } else {
        const int col = t - 3 * ni1;
        double ec = 0.0;
#pragma unroll
        for (int l = 0; l < 4; l++) ec = fma(sHc[(e2 - e2lo + l) * kGmCols + col], c2[l], ec);
        sE[9 * kGmCols + col] = ec;
      }
    }
    __syncthreads();
    if (myq < qb) {
      const int e1 = elem1[myq], o = e1 - emin;
      for (int gi = 0; gi < grp.ng; gi++) {
        const GmTab &T1 = A.tab[0][grp.k1[gi]];
        double bv[NP], bd[NP];
#pragma unroll
        for (int i = 0; i < NP; i++) {
          bv[i] = T1.t0[(size_t)myq * NP + i];
          bd[i] = T1.t1[(size_t)myq * NP + i];
        }
        double jc[3][3];  // jc[b][a] = d x_a / d xhat_b
#pragma unroll
        for (int a = 0; a < 3; a++) {
          double d1 = 0.0, d2 = 0.0, d3 = 0.0;
#pragma unroll
          for (int i = 0; i < NP; i++) {
            d1 = fma(sE[a * kGmCols + o + i], bd[i], d1);
            d2 = fma(sE[(3 + a) * kGmCols + o + i], bv[i], d2);
            d3 = fma(sE[(6 + a) * kGmCols + o + i], bv[i], d3);
          }
          jc[0][a] = d1;
          jc[1][a] = d2;
          jc[2][a] = d3;
        }
        const V3 j0{jc[0][0], jc[0][1], jc[0][2]}, j1{jc[1][0], jc[1][1], jc[1][2]}, j2{jc[2][0], jc[2][1], jc[2][2]};
        double c = 1.0;
        if (A.coef) {
          c = 0.0;
#pragma unroll
          for (int l = 0; l < 4; l++) c = fma(sE[9 * kGmCols + o + l], T1.beta[(size_t)myq * 4 + l], c);
          if (!isfinite(c)) bits |= kBitNonFinite;
        }
        const double f = metric3(grp.comp[gi], j0, j1, j2, c, bits);
        {
          const long long fi = grp.grid[gi] * A.fstride + myq + (long long)np1 * (q2 + (long long)np2 * q3l);
          if (check_range(A.status, fi, 1, (long long)kGmGrids * A.fstride)) static_cast<double *>(A.F)[fi] = f;
        }
      }
    }
    __syncthreads();
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((tid & 31) == 0 && bits) atomicOr(A.status, bits);
}

// 2D: a CTA takes one x2 point (of the group's x2 set) and a chunk of x1
// points; E is the net's contraction over that point's p+1 control rows.
template <int P> __global__ void __launch_bounds__(kGmChunk) gm_metric2_kernel(const GmArgs A) {
  constexpr int kGmCols = gm_cols<P>();
  constexpr int NP = P + 1, NT = kGmChunk;
  __shared__ double sE[5 * kGmCols];  // [v0, v1, d0, d1, c][col]
  __shared__ int sred[2];
  const int tid = threadIdx.x;
  const int np1 = A.np[0];
  const int nch1 = (np1 + NT - 1) / NT;
  long long item = blockIdx.x;
  const int c1 = (int)(item % nch1);
  item /= nch1;
  const int q2l = (int)(item % A.slab_n);
  const GmGroup &grp = c_groups2[(int)(item / A.slab_n)];
  const int q2 = A.slab_lo + q2l;
  const GmTab &T2 = A.tab[1][grp.k2];
  const int e2 = T2.elem[q2];
  double b2v[NP], b2d[NP], c2[4];
#pragma unroll
  for (int i = 0; i < NP; i++) {
    b2v[i] = T2.t0[(size_t)q2 * NP + i];
    b2d[i] = T2.t1[(size_t)q2 * NP + i];
  }
#pragma unroll
  for (int l = 0; l < 4; l++) c2[l] = T2.beta[(size_t)q2 * 4 + l];
  const int qa = c1 * NT, qb = min(np1, qa + NT);
  const int *elem1 = A.tab[0][0].elem;
  const int myq = qa + tid;
  int emin, emax;
  block_minmax(myq < qb ? elem1[myq] : 0x7fffffff, myq < qb ? elem1[myq] : -1, emin, emax, sred);
  const int ni1 = emax + P - emin + 1, nl1 = emax + 3 - emin + 1;
  if (ni1 > kGmCols || nl1 > kGmCols) {  // cannot happen (see gm_cols); reported, nothing written
    if (tid == 0) atomicOr(A.status, kBitInternal);
    return;
  }
  const int n1 = A.n[0], nc1 = A.nc[0];
  for (int col = tid; col < ni1; col += NT) {
#pragma unroll
    for (int a = 0; a < 2; a++) {
      const double *g = A.net + a * A.ntot + emin + col;
      double v = 0.0, d = 0.0;
#pragma unroll
      for (int i = 0; i < NP; i++) {
        const double x = g[(long long)n1 * (e2 + i)];
        v = fma(x, b2v[i], v);
        d = fma(x, b2d[i], d);
      }
      sE[a * kGmCols + col] = v;
      sE[(2 + a) * kGmCols + col] = d;
    }
  }
  if (A.coef)
    for (int col = tid; col < nl1; col += NT) {
      const double *g = A.coef + emin + col;
      double ec = 0.0;
#pragma unroll
      for (int l = 0; l < 4; l++) ec = fma(g[(long long)nc1 * (e2 + l)], c2[l], ec);
      sE[4 * kGmCols + col] = ec;
    }
  __syncthreads();
  unsigned bits = 0;
  if (myq < qb) {
    const int o = elem1[myq] - emin;
    for (int gi = 0; gi < grp.ng; gi++) {
      const GmTab &T1 = A.tab[0][grp.k1[gi]];
      double j0[2], j1[2];
#pragma unroll
      for (int a = 0; a < 2; a++) {
        double d1 = 0.0, d2 = 0.0;
#pragma unroll
        for (int i = 0; i < NP; i++) {
          d1 = fma(sE[a * kGmCols + o + i], T1.t1[(size_t)myq * NP + i], d1);
          d2 = fma(sE[(2 + a) * kGmCols + o + i], T1.t0[(size_t)myq * NP + i], d2);
        }
        j0[a] = d1;
        j1[a] = d2;
      }
      double c = 1.0;
      if (A.coef) {
        c = 0.0;
#pragma unroll
        for (int l = 0; l < 4; l++) c = fma(sE[4 * kGmCols + o + l], T1.beta[(size_t)myq * 4 + l], c);
        if (!isfinite(c)) bits |= kBitNonFinite;
      }
      {
        const long long fi = grp.grid[gi] * A.fstride + myq + (long long)np1 * q2l;
        if (check_range(A.status, fi, 1, (long long)kGmGrids * A.fstride)) static_cast<double *>(A.F)[fi] = metric2(grp.comp[gi], j0, j1, c, bits);
      }
    }
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((tid & 31) == 0 && bits) atomicOr(A.status, bits);
}

// ------------------------------------------------------------------ FP32 metric
// The FP32 form (WQ_MIXED) takes the Jacobian from the scaled differences of
// the net, D_b[i] = p (P_i - P_{i-e_b}) / (t_{i_b+p} - t_{i_b}) (formed in
// FP64, rounded once), and the degree p-1 basis of direction b: each column
// of J is then a sum of terms of one sign pattern without the cancellation
// of sum_i P_i B_i'(x) (whose terms are ~1/h larger than the result), so
// FP32 arithmetic keeps ~1e-7 relative accuracy at any mesh size.

__global__ void gm_diff_kernel(const double *__restrict__ net, float *__restrict__ D, int dim, int p, int n0, int n1,
                               int N0, int N1, int N2, long long ntot, const double *__restrict__ coef,
                               float *__restrict__ coef32, long long ncoef, unsigned *status) {
  unsigned bad = 0;
  if (coef)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncoef;
         i += (long long)gridDim.x * blockDim.x) {
      const float v = (float)coef[i];
      if (!isfinite(v)) bad = 1;
      coef32[i] = v;
    }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(status, kBitNonFinite);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ntot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i[3] = {(int)(idx % n0), (int)((idx / n0) % n1), (int)(idx / ((long long)n0 * n1))};
    const int Nn[3] = {N0, N1, N2};
    const long long stride[3] = {1, n0, (long long)n0 * n1};
    for (int b = 0; b < dim; b++) {
      const int ib = i[b];
      const double sc = ib >= 1 ? (double)p * Nn[b] / (double)(min(ib, Nn[b]) - max(ib - p, 0)) : 0.0;
      for (int a = 0; a < dim; a++)
        D[(b * dim + a) * ntot + idx] =
            ib >= 1 ? (float)((net[a * ntot + idx] - net[a * ntot + idx - stride[b]]) * sc) : 0.0f;
    }
  }
}

struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 cross3f(const F3 &u, const F3 &v) {
  return F3{fmaf(u.y, v.z, -u.z * v.y), fmaf(u.z, v.x, -u.x * v.z), fmaf(u.x, v.y, -u.y * v.x)};
}
__device__ __forceinline__ float dot3f(const F3 &u, const F3 &v) { return fmaf(u.x, v.x, fmaf(u.y, v.y, u.z * v.z)); }

__device__ __forceinline__ float metric3f(int comp, const F3 &j0, const F3 &j1, const F3 &j2, float c,
                                          unsigned &bits) {
  const F3 a0 = cross3f(j1, j2);
  const float det = dot3f(j0, a0);
  if (!(det > 0.0f)) bits |= isfinite(det) ? kBitGeometry : kBitNonFinite;
  const float adet = fabsf(det);
  if (comp == 0) return c * adet;
  const int a = (comp - 1) / 3, b = (comp - 1) % 3;
  F3 ra, rb;
  if (a == 0)
    ra = a0;
  else if (a == 1)
    ra = cross3f(j2, j0);
  else
    ra = cross3f(j0, j1);
  if (b == a)
    rb = ra;
  else if (b == 1)
    rb = cross3f(j2, j0);
  else
    rb = cross3f(j0, j1);
  return c * dot3f(ra, rb) / adet;
}

// Shared memory of the 3D FP32 metric kernel (floats): H of the three
// Jacobian columns [3][3][2P+1][kGmCols], Hc [P+4][kGmCols], E [10][kGmCols].
template <int P> constexpr int metric3f_smem_floats() {
  constexpr int kGmCols = gm_cols<P>();
  return 9 * (kGmRows32 + 2 * P) * kGmCols + (kGmRows32 + P + 3) * kGmCols + 10 * kGmCols;
}

// As gm_metric3_kernel, in FP32 from the difference nets: column b of J
// contracts D_b with the degree p-1 basis in direction b and the degree-p
// basis in the others (H: over x3, E: over x2, then x1 at each point).
template <int P> __global__ void __launch_bounds__(kGmChunk, 5) gm_metric3f_kernel(const GmArgs A) {
  constexpr int kGmCols = gm_cols<P>();
  constexpr int NP = P + 1, R2B = kGmRows32, NI2 = R2B + 2 * P, NL2 = R2B + P + 3, NT = kGmChunk;
  extern __shared__ float smf[];
  float *sH = smf;                      // [column b][a][i2][col]
  float *sHc = sH + 9 * NI2 * kGmCols;  // [l2][col]
  float *sE = sHc + NL2 * kGmCols;      // [E0 a, E1 a, E2 a, c][col]
  __shared__ int sred[2];
  const int tid = threadIdx.x;
  const int np1 = A.np[0], np2 = A.np[1];
  const int nch1 = (np1 + NT - 1) / NT;
  long long item = blockIdx.x;
  const int c1 = (int)(item % nch1);
  item /= nch1;
  const int nb2 = (A.n[1] + R2B - 1) / R2B;
  const int r2a = (int)(item % nb2) * R2B, r2b = min(A.n[1], r2a + R2B) - 1;
  item /= nb2;
  const int q3l = (int)(item % A.slab_n);
  const GmGroup &grp = c_groups3[(int)(item / A.slab_n)];
  const int q3 = A.slab_lo + q3l;
  const GmTab &T3 = A.tab[2][grp.k3];
  const int e3 = T3.elem[q3];
  float b3v[NP], b3l[P], c3[4];
#pragma unroll
  for (int i = 0; i < NP; i++) b3v[i] = T3.t0f[(size_t)q3 * NP + i];
#pragma unroll
  for (int j = 0; j < P; j++) b3l[j] = T3.tlf[(size_t)q3 * P + j];
#pragma unroll
  for (int l = 0; l < 4; l++) c3[l] = T3.betaf[(size_t)q3 * 4 + l];
  const int qa = c1 * NT, qb = min(np1, qa + NT);
  const int *elem1 = A.tab[0][0].elem;
  const int myq = qa + tid;
  int emin, emax;
  block_minmax(myq < qb ? elem1[myq] : 0x7fffffff, myq < qb ? elem1[myq] : -1, emin, emax, sred);
  const int ni1 = emax + P - emin + 1, nl1 = emax + 3 - emin + 1;
  if (ni1 > kGmCols || nl1 > kGmCols) {  // cannot happen (see gm_cols); reported, nothing written
    if (tid == 0) atomicOr(A.status, kBitInternal);
    return;
  }
  const int e2lo = max(0, r2a - P), e2hi = min(A.N[1] - 1, r2b);
  const int ni2 = e2hi + P - e2lo + 1, nl2 = e2hi + 3 - e2lo + 1;
  const int n1 = A.n[0], n2 = A.n[1], nc1 = A.nc[0], nc2 = A.nc[1];
  const long long nt = A.ntot, s3 = (long long)n1 * n2;
  for (int t = tid; t < ni2 * ni1; t += NT) {
    const int i2 = e2lo + t / ni1, col = t % ni1;
    const long long base = emin + col + (long long)n1 * i2;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const float *d0 = A.D + (0 * 3 + a) * nt + base, *d1 = A.D + (1 * 3 + a) * nt + base,
                  *d2 = A.D + (2 * 3 + a) * nt + base;
      float h0 = 0.0f, h1 = 0.0f, h2 = 0.0f;
#pragma unroll
      for (int i = 0; i < NP; i++) {
        h0 = fmaf(d0[s3 * (e3 + i)], b3v[i], h0);
        h1 = fmaf(d1[s3 * (e3 + i)], b3v[i], h1);
      }
#pragma unroll
      for (int j = 0; j < P; j++) h2 = fmaf(d2[s3 * (e3 + 1 + j)], b3l[j], h2);
      const int row = (a * NI2 + (i2 - e2lo)) * kGmCols + col;
      sH[row] = h0;
      sH[3 * NI2 * kGmCols + row] = h1;
      sH[6 * NI2 * kGmCols + row] = h2;
    }
  }
  if (A.coef32)
    for (int t = tid; t < nl2 * nl1; t += NT) {
      const int l2 = e2lo + t / nl1, col = t % nl1, l1 = emin + col;
      const float *g = A.coef32 + l1 + (long long)nc1 * l2;
      float hc = 0.0f;
#pragma unroll
      for (int l = 0; l < 4; l++) hc = fmaf(g[(long long)nc1 * nc2 * (e3 + l)], c3[l], hc);
      sHc[(l2 - e2lo) * kGmCols + col] = hc;
    }
  __syncthreads();
  unsigned bits = 0;
  const GmTab &T2 = A.tab[1][grp.k2];
  const int q2a = A.off[1][r2a], q2b = A.off[1][r2b + 1];
  // this thread's x1 point: its basis values for each x1 point set of the group
  float pv[2][NP], pl[2][P], pc[2][4];
  const int ng = grp.ng;
  if (myq < qb)
#pragma unroll
    for (int gi = 0; gi < 2; gi++) {
      if (gi >= ng) break;
      const GmTab &T1 = A.tab[0][grp.k1[gi]];
#pragma unroll
      for (int i = 0; i < NP; i++) pv[gi][i] = T1.t0f[(size_t)myq * NP + i];
#pragma unroll
      for (int j = 0; j < P; j++) pl[gi][j] = T1.tlf[(size_t)myq * P + j];
#pragma unroll
      for (int l = 0; l < 4; l++) pc[gi][l] = T1.betaf[(size_t)myq * 4 + l];
    }
  for (int q2 = q2a; q2 < q2b; q2++) {
    const int e2 = T2.elem[q2];
    float b2v[NP], b2l[P], c2[4];
#pragma unroll
    for (int i = 0; i < NP; i++) b2v[i] = T2.t0f[(size_t)q2 * NP + i];
#pragma unroll
    for (int j = 0; j < P; j++) b2l[j] = T2.tlf[(size_t)q2 * P + j];
#pragma unroll
    for (int l = 0; l < 4; l++) c2[l] = T2.betaf[(size_t)q2 * 4 + l];
    const int nE = 3 * ni1 + (A.coef32 ? nl1 : 0);
    for (int t = tid; t < nE; t += NT) {
      if (t < 3 * ni1) {
        const int a = t / ni1, col = t - a * ni1;
        float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f;
#pragma unroll
        for (int i = 0; i < NP; i++) {
          const int row = (a * NI2 + (e2 - e2lo + i)) * kGmCols + col;
          v0 = fmaf(sH[row], b2v[i], v0);
          v2 = fmaf(sH[6 * NI2 * kGmCols + row], b2v[i], v2);
        }
#pragma unroll
        for (int j = 0; j < P; j++)
          v1 = fmaf(sH[3 * NI2 * kGmCols + (a * NI2 + (e2 - e2lo + 1 + j)) * kGmCols + col], b2l[j], v1);
        sE[a * kGmCols + col] = v0;
        sE[(3 + a) * kGmCols + col] = v1;
        sE[(6 + a) * kGmCols + col] = v2;
      } else {
        const int col = t - 3 * ni1;
        float ec = 0.0f;
#pragma unroll
        for (int l = 0; l < 4; l++) ec = fmaf(sHc[(e2 - e2lo + l) * kGmCols + col], c2[l], ec);
        sE[9 * kGmCols + col] = ec;
      }
    }
    __syncthreads();
    if (myq < qb) {
      const int o = elem1[myq] - emin;
#pragma unroll
      for (int gi = 0; gi < 2; gi++) {
        if (gi >= ng) break;
        const float *bv = pv[gi], *bl = pl[gi];
        float jc[3][3];  // jc[b][a] = d x_a / d xhat_b
#pragma unroll
        for (int a = 0; a < 3; a++) {
          float d1 = 0.0f, d2 = 0.0f, d3 = 0.0f;
#pragma unroll
          for (int j = 0; j < P; j++) d1 = fmaf(sE[a * kGmCols + o + 1 + j], bl[j], d1);
#pragma unroll
          for (int i = 0; i < NP; i++) {
            d2 = fmaf(sE[(3 + a) * kGmCols + o + i], bv[i], d2);
            d3 = fmaf(sE[(6 + a) * kGmCols + o + i], bv[i], d3);
          }
          jc[0][a] = d1;
          jc[1][a] = d2;
          jc[2][a] = d3;
        }
        const F3 j0{jc[0][0], jc[0][1], jc[0][2]}, j1{jc[1][0], jc[1][1], jc[1][2]}, j2{jc[2][0], jc[2][1], jc[2][2]};
        float c = 1.0f;
        if (A.coef32) {
          c = 0.0f;
#pragma unroll
          for (int l = 0; l < 4; l++) c = fmaf(sE[9 * kGmCols + o + l], pc[gi][l], c);
          if (!isfinite(c)) bits |= kBitNonFinite;
        }
        const float f = metric3f(grp.comp[gi], j0, j1, j2, c, bits);
        {
          const long long fi = grp.grid[gi] * A.fstride + myq + (long long)np1 * (q2 + (long long)np2 * q3l);
          if (check_range(A.status, fi, 1, (long long)kGmGrids * A.fstride)) static_cast<float *>(A.F)[fi] = f;
        }
      }
    }
    __syncthreads();
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((tid & 31) == 0 && bits) atomicOr(A.status, bits);
}

// 2D FP32: E0 = D0 contracted with the x2 point's degree-p basis, E1 = D1
// with its degree p-1 basis; J's columns at each x1 point.
template <int P> __global__ void __launch_bounds__(kGmChunk) gm_metric2f_kernel(const GmArgs A) {
  constexpr int kGmCols = gm_cols<P>();
  constexpr int NP = P + 1, NT = kGmChunk;
  __shared__ float sE[5 * kGmCols];  // [E0 a0, a1, E1 a0, a1, c][col]
  __shared__ int sred[2];
  const int tid = threadIdx.x;
  const int np1 = A.np[0];
  const int nch1 = (np1 + NT - 1) / NT;
  long long item = blockIdx.x;
  const int c1 = (int)(item % nch1);
  item /= nch1;
  const int q2l = (int)(item % A.slab_n);
  const GmGroup &grp = c_groups2[(int)(item / A.slab_n)];
  const int q2 = A.slab_lo + q2l;
  const GmTab &T2 = A.tab[1][grp.k2];
  const int e2 = T2.elem[q2];
  float b2v[NP], b2l[P], c2[4];
#pragma unroll
  for (int i = 0; i < NP; i++) b2v[i] = T2.t0f[(size_t)q2 * NP + i];
#pragma unroll
  for (int j = 0; j < P; j++) b2l[j] = T2.tlf[(size_t)q2 * P + j];
#pragma unroll
  for (int l = 0; l < 4; l++) c2[l] = T2.betaf[(size_t)q2 * 4 + l];
  const int qa = c1 * NT, qb = min(np1, qa + NT);
  const int *elem1 = A.tab[0][0].elem;
  const int myq = qa + tid;
  int emin, emax;
  block_minmax(myq < qb ? elem1[myq] : 0x7fffffff, myq < qb ? elem1[myq] : -1, emin, emax, sred);
  const int ni1 = emax + P - emin + 1, nl1 = emax + 3 - emin + 1;
  if (ni1 > kGmCols || nl1 > kGmCols) {  // cannot happen (see gm_cols); reported, nothing written
    if (tid == 0) atomicOr(A.status, kBitInternal);
    return;
  }
  const int n1 = A.n[0], nc1 = A.nc[0];
  const long long nt = A.ntot;
  for (int t = tid; t < 2 * ni1; t += NT) {
    const int a = t / ni1, col = t - a * ni1;
    const float *d0 = A.D + (0 * 2 + a) * nt + emin + col, *d1 = A.D + (1 * 2 + a) * nt + emin + col;
    float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
    for (int i = 0; i < NP; i++) v0 = fmaf(d0[(long long)n1 * (e2 + i)], b2v[i], v0);
#pragma unroll
    for (int j = 0; j < P; j++) v1 = fmaf(d1[(long long)n1 * (e2 + 1 + j)], b2l[j], v1);
    sE[a * kGmCols + col] = v0;
    sE[(2 + a) * kGmCols + col] = v1;
  }
  if (A.coef32)
    for (int col = tid; col < nl1; col += NT) {
      const float *g = A.coef32 + emin + col;
      float ec = 0.0f;
#pragma unroll
      for (int l = 0; l < 4; l++) ec = fmaf(g[(long long)nc1 * (e2 + l)], c2[l], ec);
      sE[4 * kGmCols + col] = ec;
    }
  __syncthreads();
  unsigned bits = 0;
  if (myq < qb) {
    const int o = elem1[myq] - emin;
    for (int gi = 0; gi < grp.ng; gi++) {
      const GmTab &T1 = A.tab[0][grp.k1[gi]];
      float j0[2], j1[2];
#pragma unroll
      for (int a = 0; a < 2; a++) {
        float d1 = 0.0f, d2 = 0.0f;
#pragma unroll
        for (int j = 0; j < P; j++) d1 = fmaf(sE[a * kGmCols + o + 1 + j], T1.tlf[(size_t)myq * P + j], d1);
#pragma unroll
        for (int i = 0; i < NP; i++) d2 = fmaf(sE[(2 + a) * kGmCols + o + i], T1.t0f[(size_t)myq * NP + i], d2);
        j0[a] = d1;
        j1[a] = d2;
      }
      float c = 1.0f;
      if (A.coef32) {
        c = 0.0f;
#pragma unroll
        for (int l = 0; l < 4; l++) c = fmaf(sE[4 * kGmCols + o + l], T1.betaf[(size_t)myq * 4 + l], c);
        if (!isfinite(c)) bits |= kBitNonFinite;
      }
      const float det = fmaf(j0[0], j1[1], -j1[0] * j0[1]);
      if (!(det > 0.0f)) bits |= isfinite(det) ? kBitGeometry : kBitNonFinite;
      const float adet = fabsf(det);
      const int comp = grp.comp[gi];
      float f;
      if (comp == 0) {
        f = c * adet;
      } else {
        const int a = (comp - 1) / 3, b = (comp - 1) % 3;
        const float ra0 = a == 0 ? j1[1] : -j0[1], ra1 = a == 0 ? -j1[0] : j0[0];
        const float rb0 = b == 0 ? j1[1] : -j0[1], rb1 = b == 0 ? -j1[0] : j0[0];
        f = c * fmaf(ra0, rb0, ra1 * rb1) / adet;
      }
      {
        const long long fi = grp.grid[gi] * A.fstride + myq + (long long)np1 * q2l;
        if (check_range(A.status, fi, 1, (long long)kGmGrids * A.fstride)) static_cast<float *>(A.F)[fi] = f;
      }
    }
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((tid & 31) == 0 && bits) atomicOr(A.status, bits);
}

// Per-warp shared memory of the row kernel (elements of R): the weight-test
// tables [DIM][4][LM][NBP] (rows padded to NBP), X [LM][LM][NB] (3D),
// Y [LM][NB^(DIM-1)] and the band row being written [NB^DIM]; LM = the most
// points of a row in one direction (LC when the row class fixes it).
template <int P> constexpr int nb_pad() { return ((2 * P + 1) + 3) / 4 * 4; }

// Row classes of the row kernel: 0 interior (p+1 points in every
// direction); 1, 2, 3: a face row, direction 0, 1 or 2 on Gauss-Legendre and
// the others interior; 4: the rest (two or more directions on
// Gauss-Legendre).  Points per row in direction d: p+1 where the class fixes
// it, else read from the tables (at most p(p+1)).
constexpr int kClsInt = 0, kClsRest = 4;
template <int P, int CLS> constexpr int cls_l(int d) { return CLS == kClsRest ? 0 : (CLS == 1 + d ? 0 : P + 1); }
template <int P, int CLS> constexpr int cls_lm(int d) { return cls_l<P, CLS>(d) ? P + 1 : P * (P + 1); }

// Per-warp shared memory of the row kernel (elements of R): the weight-test
// tables [d][4][LM_d][NBP] (rows padded to NBP), X [LM_0][LM_1][NB] (3D),
// Y [LM_0][NB^(DIM-1)] and the band row being written [NB^DIM].
template <int P, int DIM, int CLS> constexpr int rows_warp_elems() {
  constexpr int NB = 2 * P + 1, NY = DIM == 3 ? NB * NB : NB;
  constexpr int L0 = cls_lm<P, CLS>(0), L1 = cls_lm<P, CLS>(1), L2 = DIM == 3 ? cls_lm<P, CLS>(2) : 0;
  return 4 * (L0 + L1 + L2) * nb_pad<P>() + (DIM == 3 ? L0 * L1 * NB : 0) + L0 * NY + NY * NB;
}

// Rows of class CLS in the slab's planes (2D: lines) [bp_lo, bp_hi], item
// idx of a gap-free enumeration; false past the end.  With the slab
// direction's interior planes I = [max(bp_lo, p), min(bp_hi, N_s - 1)] and
// the others B (those below p, then those from max(p, N_s) on), and in the
// earlier directions the interior rows p .. N-1 (b of them) and the rest
// (k -> k < p ? k : k + b):
//   3D  interior: I x I1 x I2;  face 0: I x B1 x I2;  face 1: I x I1 x B2;
//       face 2: B x I1 x I2;  rest: B x (rows with r1 or r2 outside), then
//       I x B1 x B2;
//   2D  interior: I x I1;  face 0: I x B1;  face 1: B x I1;  rest: B x B1.
template <int P, int DIM, int CLS>
__device__ __forceinline__ bool class_row(const GmArgs &A, long long j, int (&r)[3]) {
  constexpr int SD = DIM - 1;
  const int n1 = A.n[0], b1 = max(0, A.N[0] - P), o1 = n1 - b1;
  const int n2 = A.n[1], b2 = DIM == 3 ? max(0, A.N[1] - P) : 0, o2 = n2 - b2;
  const int pl0 = A.bp_lo, pl1 = A.bp_hi, Ns = A.N[SD];
  const int nA = max(0, min(pl1, P - 1) - pl0 + 1);
  const int bLo = max(pl0, P), nI = max(0, min(pl1, Ns - 1) - bLo + 1);
  const int cLo = max(pl0, max(P, Ns)), nC = max(0, pl1 - cLo + 1);
  auto bplane = [&](long long k) { return (int)(k < nA ? pl0 + k : cLo + (k - nA)); };
  auto outer = [&](int k, int b) { return k < P ? k : k + b; };
  r[0] = r[1] = r[2] = 0;
  if constexpr (DIM == 3) {
    if (CLS == kClsInt) {
      const long long per = (long long)b1 * b2;
      if (j >= per * nI) return false;
      r[0] = P + (int)(j % b1);
      r[1] = P + (int)((j / b1) % b2);
      r[2] = bLo + (int)(j / per);
    } else if (CLS == 1) {
      const long long per = (long long)o1 * b2;
      if (j >= per * nI) return false;
      r[0] = outer((int)(j % o1), b1);
      r[1] = P + (int)((j / o1) % b2);
      r[2] = bLo + (int)(j / per);
    } else if (CLS == 2) {
      const long long per = (long long)b1 * o2;
      if (j >= per * nI) return false;
      r[0] = P + (int)(j % b1);
      r[1] = outer((int)((j / b1) % o2), b2);
      r[2] = bLo + (int)(j / per);
    } else if (CLS == 3) {
      const long long per = (long long)b1 * b2;
      if (j >= per * (nA + nC)) return false;
      r[0] = P + (int)(j % b1);
      r[1] = P + (int)((j / b1) % b2);
      r[2] = bplane(j / per);
    } else {
      const long long part = (long long)o2 * n1 + (long long)b2 * o1;
      if (j < part * (nA + nC)) {
        r[2] = bplane(j / part);
        long long k = j % part;
        if (k < (long long)o2 * n1) {
          r[1] = outer((int)(k / n1), b2);
          r[0] = (int)(k % n1);
        } else {
          k -= (long long)o2 * n1;
          r[1] = P + (int)(k / o1);
          r[0] = outer((int)(k % o1), b1);
        }
      } else {
        j -= part * (nA + nC);
        const long long per = (long long)o1 * o2;
        if (j >= per * nI) return false;
        r[0] = outer((int)(j % o1), b1);
        r[1] = outer((int)((j / o1) % o2), b2);
        r[2] = bLo + (int)(j / per);
      }
    }
  } else {
    if (CLS == kClsInt) {
      if (j >= (long long)b1 * nI) return false;
      r[0] = P + (int)(j % b1);
      r[1] = bLo + (int)(j / b1);
    } else if (CLS == 1) {
      if (j >= (long long)o1 * nI) return false;
      r[0] = outer((int)(j % o1), b1);
      r[1] = bLo + (int)(j / o1);
    } else if (CLS == 2) {
      if (j >= (long long)b1 * (nA + nC)) return false;
      r[0] = P + (int)(j % b1);
      r[1] = bplane(j / b1);
    } else {
      if (j >= (long long)o1 * (nA + nC)) return false;
      r[0] = outer((int)(j % o1), b1);
      r[1] = bplane(j / o1);
    }
  }
  return true;
}

// Rows of each class in the slab (host; the counts class_row enumerates).
inline void class_counts(int dim, int P, const int *n, const int *N, int pl0, int pl1, long long cnt[5]) {
  const long long n1 = n[0], b1 = std::max(0, N[0] - P), o1 = n1 - b1;
  const long long n2 = n[1], b2 = dim == 3 ? std::max(0, N[1] - P) : 0, o2 = n2 - b2;
  const int Ns = N[dim - 1];
  const long long nA = std::max(0, std::min(pl1, P - 1) - pl0 + 1);
  const int bLo = std::max(pl0, P);
  const long long nI = std::max(0, std::min(pl1, Ns - 1) - bLo + 1);
  const int cLo = std::max(pl0, std::max(P, Ns));
  const long long nB = nA + std::max(0, pl1 - cLo + 1);
  for (int c = 0; c < 5; c++) cnt[c] = 0;
  if (dim == 3) {
    cnt[0] = b1 * b2 * nI;
    cnt[1] = o1 * b2 * nI;
    cnt[2] = b1 * o2 * nI;
    cnt[3] = b1 * b2 * nB;
    cnt[4] = (o2 * n1 + b2 * o1) * nB + o1 * o2 * nI;
  } else {
    cnt[0] = b1 * nI;
    cnt[1] = o1 * nI;
    cnt[2] = b1 * nB;
    cnt[4] = o1 * nB;
  }
}

// One row per warp, rows of class CLS (compile-time point counts where the
// class fixes them).  Each lane owns a run of outputs of every contraction
// (a row of NB columns, or half of one), so the weight-test row of the
// contracted point is read once for them all: X[q1][q2][.] = sum_q3
// F[q1,q2,q3] A3[q3][.], then Y[q1][.][s3] += sum_q2 X[q1][q2][s3] A2[q2][.]
// over the terms of one direction-1 kind, then band[.][s23] += sum_q1
// Y[q1][s23] A1[q1][.]; the band row is staged in shared memory and written
// with consecutive lanes on consecutive entries.
template <int P, int DIM, int CLS, int WARPS, typename R>
__global__ void __launch_bounds__(32 * WARPS) gm_rows_kernel(const GmArgs A) {
  constexpr int NB = 2 * P + 1, NP = P + 1, NBP = nb_pad<P>();
  constexpr int LC0 = cls_l<P, CLS>(0), LC1 = cls_l<P, CLS>(1), LC2 = DIM == 3 ? cls_l<P, CLS>(2) : 1;
  constexpr int LM0 = cls_lm<P, CLS>(0), LM1 = cls_lm<P, CLS>(1), LM2 = DIM == 3 ? cls_lm<P, CLS>(2) : 0;
  constexpr int NY = DIM == 3 ? NB * NB : NB;  // columns of Y (s2, s3)
  constexpr int NBAND = NY * NB;
  constexpr int NK = (NY + 31) / 32;  // band columns s23 per lane
  constexpr int H1 = (NB + 1) / 2;    // the first half of the x3 columns
  // unroll a row loop only where its bound is compile-time
  constexpr int U0 = LC0 ? 64 : 1, U1 = LC1 ? 64 : 1, U2 = LC2 ? 64 : 1, U01 = (LC0 && LC1) ? 64 : 1;
  extern __shared__ __align__(16) unsigned char smrows[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R *sA = reinterpret_cast<R *>(smrows) + warp * rows_warp_elems<P, DIM, CLS>();  // [d][k][q][NBP]
  R *sX = sA + 4 * (LM0 + LM1 + LM2) * NBP;
  R *sY = sX + (DIM == 3 ? LM0 * LM1 * NB : 0);
  R *sO = sY + LM0 * NY;
  const int aoff[3] = {0, 4 * LM0 * NBP, 4 * (LM0 + LM1) * NBP};
  const int lmd[3] = {LM0, LM1, LM2};
  int r[3];
  if (!class_row<P, DIM, CLS>(A, (long long)blockIdx.x * WARPS + warp, r)) return;
  const long long row = r[0] + (long long)A.n[0] * (r[1] + (long long)A.n[1] * r[2]);
  if (row < A.row_begin || row >= A.row_end) return;
  int off[3], L[3];
  const int lc[3] = {LC0, LC1, LC2};
#pragma unroll
  for (int d = 0; d < DIM; d++) {
    off[d] = A.off[d][r[d]];
    L[d] = lc[d] ? lc[d] : A.off[d][r[d] + 1] - off[d];
  }
  if (DIM == 2) L[2] = 1;
  // weight-test tables: A_d^k[q][j] = W(q) T(q, j - o), o = elem(q) - r + P
#pragma unroll
  for (int d = 0; d < DIM; d++) {
    const int *elem = A.tab[d][0].elem;
    for (int t = lane; t < 4 * L[d]; t += 32) {
      const int k = t / L[d], q = t - k * L[d];
      const int o = elem[off[d] + q] - r[d] + P;
      const R *wt = (std::is_same<R, float>::value ? (const R *)A.WT32[d][k] : (const R *)A.WT64[d][k]) +
                    (size_t)(off[d] + q) * NP;
      R v[NP];
#pragma unroll
      for (int i = 0; i < NP; i++) v[i] = wt[i];
      R *rowp = sA + aoff[d] + (k * lmd[d] + q) * NBP;
#pragma unroll
      for (int j = 0; j < NBP; j++) {
        R x = 0;
#pragma unroll
        for (int i = 0; i < NP; i++)
          if (j == o + i) x = v[i];
        rowp[j] = x;
      }
    }
  }
  __syncwarp();
  R outK[NK][NB];
#pragma unroll
  for (int c = 0; c < NK; c++)
#pragma unroll
    for (int s = 0; s < NB; s++) outK[c][s] = 0;
  const GmTerm *terms = DIM == 3 ? c_terms3 : c_terms2;
  const int *gstart = DIM == 3 ? c_group_start3 : c_group_start2;
  const long long ob = (row - A.out_row0) * NBAND;
  const long long s2 = A.np[0], s3 = (long long)A.np[0] * A.np[1];
  // the row's factor box, first to last point, in every grid
  if (!check_range(A.status, off[0] + s2 * off[1] + (DIM == 3 ? s3 * (off[2] - A.slab_lo) : -s2 * A.slab_lo),
                   (L[0] - 1) + s2 * (L[1] - 1) + (DIM == 3 ? s3 * (L[2] - 1) : 0) + 1, A.fstride) ||
      !check_range(A.status, ob, NBAND, A.out_rows * NBAND))
    return;
  // interior class in 3D: a lane's x3 stage item is the same (q1, q2, half) in
  // every term, so the factors of the next term are loaded while the
  // current one is contracted (the terms run in one contiguous range)
  constexpr bool PF = DIM == 3 && LC0 && LC1 && LC2 && 2 * LC0 * LC1 <= 32;
  const int t_first = A.M ? gstart[0] : gstart[1], t_end = A.K ? gstart[5] : gstart[1];
  const bool pf_act = lane < 2 * LC0 * LC1;
  const int pf_q1 = (lane >> 1) % (LC0 ? LC0 : 1), pf_q2 = (lane >> 1) / (LC0 ? LC0 : 1);
  R fcur[PF ? LC2 : 1], fnxt[PF ? LC2 : 1];
  auto load_f = [&](int ti, R (&v)[PF ? LC2 : 1]) {
    if constexpr (PF) {
      const R *f = static_cast<const R *>(A.F) + terms[ti].grid * A.fstride + off[0] + s2 * off[1] +
                   s3 * (off[2] - A.slab_lo) + pf_q1 + s2 * pf_q2;
#pragma unroll
      for (int q3 = 0; q3 < LC2; q3++) v[q3] = pf_act ? f[s3 * q3] : R(0);
    }
  };
  if (PF && t_first < t_end) load_f(t_first, fcur);
  for (int grp = 0; grp < 5; grp++) {
    if (grp == 0 ? !A.M : !A.K) continue;
#pragma unroll U0
    for (int t = lane; t < L[0] * NY; t += 32) sY[t] = 0;
    __syncwarp();
    int k1 = 0;
    for (int ti = gstart[grp]; ti < gstart[grp + 1]; ti++) {
      const GmTerm &tm = terms[ti];
      k1 = tm.k[0];
      const R *F = static_cast<const R *>(A.F) + tm.grid * A.fstride;
      const R *A2 = sA + aoff[1] + (tm.k[1] * LM1) * NBP;
      if (DIM == 3) {
        const R *A3 = sA + aoff[2] + (tm.k[2] * LM2) * NBP;
        const R *F0 = F + off[0] + s2 * off[1] + s3 * (off[2] - A.slab_lo);
        if constexpr (PF) {
          if (ti + 1 < t_end) load_f(ti + 1, fnxt);
          if (pf_act) {
            const int c0 = (lane & 1) * H1;
            R acc[H1];
#pragma unroll
            for (int h = 0; h < H1; h++) acc[h] = 0;
#pragma unroll
            for (int q3 = 0; q3 < LC2; q3++) {
              const R *a = A3 + q3 * NBP + c0;
#pragma unroll
              for (int h = 0; h < H1; h++) acc[h] = fma(fcur[q3], a[h], acc[h]);
            }
            R *x = sX + (lane >> 1) * NB + c0;
#pragma unroll
            for (int h = 0; h < H1; h++)
              if (c0 + h < NB) x[h] = acc[h];
          }
#pragma unroll
          for (int q3 = 0; q3 < LC2; q3++) fcur[q3] = fnxt[q3];
        } else
        // X: items (q1, q2, half of the x3 columns)
#pragma unroll U01
        for (int it = lane; it < 2 * L[0] * L[1]; it += 32) {
          const int pr = it >> 1, c0 = (it & 1) * H1;
          const int q1 = pr % L[0], q2 = pr / L[0];
          const R *f = F0 + q1 + s2 * q2;
          R acc[H1];
#pragma unroll
          for (int h = 0; h < H1; h++) acc[h] = 0;
#pragma unroll U2
          for (int q3 = 0; q3 < L[2]; q3++) {
            const R fv = f[s3 * q3];
            const R *a = A3 + q3 * NBP + c0;
#pragma unroll
            for (int h = 0; h < H1; h++) acc[h] = fma(fv, a[h], acc[h]);
          }
          R *x = sX + pr * NB + c0;
#pragma unroll
          for (int h = 0; h < H1; h++)
            if (c0 + h < NB) x[h] = acc[h];
        }
        __syncwarp();
        // Y: items (q1, s3), all x2 columns
#pragma unroll U0
        for (int it = lane; it < L[0] * NB; it += 32) {
          const int q1 = it % L[0], c3 = it / L[0];
          R acc[NB];
#pragma unroll
          for (int c = 0; c < NB; c++) acc[c] = 0;
#pragma unroll U1
          for (int q2 = 0; q2 < L[1]; q2++) {
            const R xv = sX[(q1 + L[0] * q2) * NB + c3];
            const R *a = A2 + q2 * NBP;
#pragma unroll
            for (int c = 0; c < NB; c++) acc[c] = fma(xv, a[c], acc[c]);
          }
          R *y = sY + q1 * NY + NB * c3;
#pragma unroll
          for (int c = 0; c < NB; c++) y[c] += acc[c];
        }
        __syncwarp();
      } else {
        const R *F0 = F + off[0] + s2 * (off[1] - A.slab_lo);
        // Y: items q1, all x2 columns
#pragma unroll U0
        for (int it = lane; it < L[0]; it += 32) {
          R acc[NB];
#pragma unroll
          for (int c = 0; c < NB; c++) acc[c] = 0;
#pragma unroll U1
          for (int q2 = 0; q2 < L[1]; q2++) {
            const R fv = F0[it + s2 * q2];
            const R *a = A2 + q2 * NBP;
#pragma unroll
            for (int c = 0; c < NB; c++) acc[c] = fma(fv, a[c], acc[c]);
          }
          R *y = sY + it * NY;
#pragma unroll
          for (int c = 0; c < NB; c++) y[c] += acc[c];
        }
        __syncwarp();
      }
    }
    // band: items s23, all x1 columns
    const R *A1 = sA + aoff[0] + (k1 * LM0) * NBP;
#pragma unroll
    for (int c = 0; c < NK; c++) {
      const int s23 = lane + 32 * c;
      if (s23 < NY) {
        R acc[NB];
#pragma unroll
        for (int s = 0; s < NB; s++) acc[s] = 0;
#pragma unroll U0
        for (int q1 = 0; q1 < L[0]; q1++) {
          const R yv = sY[q1 * NY + s23];
          const R *a = A1 + q1 * NBP;
#pragma unroll
          for (int s = 0; s < NB; s++) acc[s] = fma(yv, a[s], acc[s]);
        }
        if (grp == 0) {
#pragma unroll
          for (int s = 0; s < NB; s++) sO[s23 * NB + s] = acc[s];
        } else {
#pragma unroll
          for (int s = 0; s < NB; s++) outK[c][s] += acc[s];
        }
      }
    }
    __syncwarp();
    if (grp == 0) {
      R *M = static_cast<R *>(A.M) + ob;
      for (int e = lane; e < NBAND; e += 32) M[e] = sO[e];
      __syncwarp();
    }
  }
  if (A.K) {
#pragma unroll
    for (int c = 0; c < NK; c++) {
      const int s23 = lane + 32 * c;
      if (s23 < NY)
#pragma unroll
        for (int s = 0; s < NB; s++) sO[s23 * NB + s] = outK[c][s];
    }
    __syncwarp();
    R *K = static_cast<R *>(A.K) + ob;
    for (int e = lane; e < NBAND; e += 32) K[e] = sO[e];
  }
}

constexpr int kGmWarpsInt = 8;  // rows (warps) per CTA of the interior-row kernel

template <int P, int DIM, int CLS, typename R> wq_status launch_rows_class(const GmArgs &a, long long n, cudaStream_t s) {
  if (n <= 0) return WQ_OK;
  constexpr int W = CLS == kClsInt ? kGmWarpsInt : kGmWarps;
  const size_t smem = sizeof(R) * (size_t)rows_warp_elems<P, DIM, CLS>() * W;
  gm_rows_kernel<P, DIM, CLS, W, R><<<(unsigned)((n + W - 1) / W), 32 * W, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? WQ_OK : WQ_ERR_CUDA;
}

template <int P, int DIM, typename R>
wq_status launch_slab(const GmArgs &a, long long nitems, const long long *ncls, cudaStream_t s) {
  constexpr bool F32 = std::is_same<R, float>::value;
  if (nitems > 0) {
    if (DIM == 3) {
      if (F32)
        gm_metric3f_kernel<P><<<(unsigned)nitems, kGmChunk, sizeof(float) * (size_t)metric3f_smem_floats<P>(), s>>>(a);
      else
        gm_metric3_kernel<P><<<(unsigned)nitems, kGmChunk, sizeof(double) * (size_t)metric3_smem_doubles<P>(), s>>>(a);
    } else {
      if (F32)
        gm_metric2f_kernel<P><<<(unsigned)nitems, kGmChunk, 0, s>>>(a);
      else
        gm_metric2_kernel<P><<<(unsigned)nitems, kGmChunk, 0, s>>>(a);
    }
    if (cudaGetLastError() != cudaSuccess) return WQ_ERR_CUDA;
  }
  wq_status st = launch_rows_class<P, DIM, 0, R>(a, ncls[0], s);
  if (st == WQ_OK) st = launch_rows_class<P, DIM, 1, R>(a, ncls[1], s);
  if (st == WQ_OK) st = launch_rows_class<P, DIM, 2, R>(a, ncls[2], s);
  if (st == WQ_OK && DIM == 3) st = launch_rows_class<P, DIM, 3, R>(a, ncls[3], s);
  if (st == WQ_OK) st = launch_rows_class<P, DIM, kClsRest, R>(a, ncls[4], s);
  return st;
}

template <int P, int DIM, int CLS, typename R> cudaError_t set_rows_limit() {
  constexpr int W = CLS == kClsInt ? kGmWarpsInt : kGmWarps;
  return cudaFuncSetAttribute(gm_rows_kernel<P, DIM, CLS, W, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(R) * rows_warp_elems<P, DIM, CLS>() * W));
}

template <int P, int DIM, typename R> cudaError_t set_smem_limits() {
  cudaError_t e = cudaSuccess;
  if (DIM == 3)
    e = std::is_same<R, float>::value
            ? cudaFuncSetAttribute(gm_metric3f_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(float) * metric3f_smem_floats<P>()))
            : cudaFuncSetAttribute(gm_metric3_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(double) * metric3_smem_doubles<P>()));
  if (e == cudaSuccess) e = set_rows_limit<P, DIM, 0, R>();
  if (e == cudaSuccess) e = set_rows_limit<P, DIM, 1, R>();
  if (e == cudaSuccess) e = set_rows_limit<P, DIM, 2, R>();
  if (e == cudaSuccess && DIM == 3) e = set_rows_limit<P, DIM, 3, R>();
  if (e == cudaSuccess) e = set_rows_limit<P, DIM, kClsRest, R>();
  return e;
}

template <typename R> cudaError_t set_limits(int p, int dim) {
  return p == 2 ? (dim == 3 ? set_smem_limits<2, 3, R>() : set_smem_limits<2, 2, R>())
                : (dim == 3 ? set_smem_limits<3, 3, R>() : set_smem_limits<3, 2, R>());
}

template <typename R>
wq_status launch_any(int p, int dim, const GmArgs &a, long long nitems, const long long *ncls, cudaStream_t s) {
  return p == 2 ? (dim == 3 ? launch_slab<2, 3, R>(a, nitems, ncls, s) : launch_slab<2, 2, R>(a, nitems, ncls, s))
                : (dim == 3 ? launch_slab<3, 3, R>(a, nitems, ncls, s) : launch_slab<3, 2, R>(a, nitems, ncls, s));
}

// Scratch budget of one slab's factor arrays.
constexpr size_t kGmScratchBytes = size_t(1) << 30;

}  // namespace
}  // namespace wq

extern "C" wq_status wq_assemble_general(const wq_rules *R, const double *net, const double *coef,
                                         wq_precision prec, void *M, void *K, int64_t row_begin, int64_t row_end,
                                         void *stream) {
  using namespace wq;
  TraceRange trace("wq_assemble_general");
  if (!R || !R->on_device) return WQ_ERR_ARG;
  const long long nrows = (long long)R->n[0] * R->n[1] * R->n[2];
  if (row_begin < 0 || row_end > nrows || row_begin > row_end) return WQ_ERR_ARG;
  if (row_begin == row_end) return WQ_OK;
  if (!net || (!M && !K)) return WQ_ERR_ARG;
  if (prec != WQ_FP64 && prec != WQ_MIXED) return WQ_ERR_UNSUPPORTED;
  const bool f32 = prec == WQ_MIXED;
  const size_t elt = f32 ? sizeof(float) : sizeof(double);
  if (R->mode != kModeWQ || R->bnd_weighted || !R->dev_cross) return WQ_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != R->device) return WQ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int dim = R->dim, p = R->p;

  GmArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dim = dim;
  a.ntot = 1;
  for (int d = 0; d < 3; d++) {
    a.n[d] = R->n[d];
    a.N[d] = R->nel[d];
    a.nc[d] = R->nc[d];
    a.np[d] = d < dim ? R->dev[d][0].npts : 1;
    if (d < dim) a.ntot *= R->n[d];
  }
  for (int d = 0; d < dim; d++) {
    const DevDirKind &Dm = R->dev[d][0], &Ds = R->dev[d][1];
    const DevCross &Dx = R->devx[d];
    a.off[d] = Dm.off;
    a.tab[d][0] = GmTab{Dm.elem, Dm.t0, Dm.t1, Dm.beta, Dm.tl, nullptr, nullptr, nullptr};
    a.tab[d][1] = GmTab{Ds.elem, Ds.t0, Ds.t1, Ds.beta, Ds.tl, nullptr, nullptr, nullptr};
    a.tab[d][2] = GmTab{Dx.elem, Dx.t0, Dx.t1, Dx.beta, Dx.tl, nullptr, nullptr, nullptr};
    const GmDevTab &G = R->gmt[d];
    for (int k = 0; k < 3; k++) {
      a.tab[d][k].t0f = G.t0f[k];
      a.tab[d][k].tlf = G.tlf[k];
      a.tab[d][k].betaf = G.betaf[k];
    }
    for (int k = 0; k < 4; k++) {
      a.WT64[d][k] = G.wt64[k];
      a.WT32[d][k] = G.wt32[k];
    }
  }
  a.net = net;
  a.coef = coef;
  a.M = M;
  a.K = K;
  a.out_row0 = row_begin;
  a.out_rows = row_end - row_begin;
  a.status = R->dev_status;

  // slabs of whole x3 planes (3D) or x2 lines (2D), their points' factors at most kGmScratchBytes
  const int sd = dim - 1;                      // slab direction
  const long long plane = dim == 3 ? (long long)R->n[0] * R->n[1] : R->n[0];
  const int pl0 = (int)(row_begin / plane), pl1 = (int)((row_end - 1) / plane);
  const std::vector<int> &offs = R->host[sd][0].off;
  const long long per_point = (long long)kGmGrids * a.np[0] * (dim == 3 ? a.np[1] : 1) * (long long)elt;
  // FP32: the scaled difference nets ([b][a], dim^2 arrays of the net's size) precede the factors
  const long long ncoef = (long long)R->nc[0] * R->nc[1] * R->nc[2];
  const long long dnet = f32 ? (long long)((dim * dim * a.ntot * sizeof(float) + 255) / 256 * 256) : 0;
  const long long dbytes = f32 ? dnet + (long long)((ncoef * sizeof(float) + 255) / 256 * 256) : 0;
  int most = 0;
  for (int r = pl0; r <= pl1; r++) most = std::max(most, offs[r + 1] - offs[r]);
  // (WQ_GENERAL_SLAB_BYTES lowers the bound, down to one plane per slab: a
  // hook for testing the slab loop on small meshes)
  long long budget = (long long)kGmScratchBytes;
  if (const char *env = std::getenv("WQ_GENERAL_SLAB_BYTES")) {
    const long long v = std::atoll(env);
    if (v > 0 && v < budget) budget = v;
  }
  budget = std::max(budget, per_point * most);
  // grow the scratch to the largest slab of this call
  std::vector<std::pair<int, int>> slabs;
  long long need = 0;
  for (int r = pl0; r <= pl1;) {
    int e = r;
    while (e + 1 <= pl1 && per_point * (offs[e + 2] - offs[r]) <= budget) e++;
    slabs.push_back({r, e});
    need = std::max(need, per_point * (long long)(offs[e + 1] - offs[r]));
    r = e + 1;
  }
  need += dbytes;
  if ((size_t)need > R->dev_gm_bytes) {
    if (R->dev_gm) {
      if (cudaStreamSynchronize(s) != cudaSuccess) return WQ_ERR_CUDA;
      cudaFree(R->dev_gm);
      R->dev_gm = nullptr;
      R->dev_gm_bytes = 0;
    }
    if (cudaMalloc(&R->dev_gm, (size_t)need) != cudaSuccess) {
      cudaGetLastError();
      return WQ_ERR_OOM;
    }
    R->dev_gm_bytes = (size_t)need;
  }
  a.F = static_cast<char *>(R->dev_gm) + dbytes;
  a.D = f32 ? static_cast<const float *>(R->dev_gm) : nullptr;
  float *coef32 = f32 ? reinterpret_cast<float *>(static_cast<char *>(R->dev_gm) + dnet) : nullptr;
  a.coef32 = f32 && coef ? coef32 : nullptr;
  cudaError_t e = f32 ? set_limits<float>(p, dim) : set_limits<double>(p, dim);
  if (e != cudaSuccess) return WQ_ERR_CUDA;
  if (f32) {
    const long long blocks = std::min<long long>((std::max(a.ntot, ncoef) + 255) / 256, 8192);
    gm_diff_kernel<<<(unsigned)blocks, 256, 0, s>>>(net, static_cast<float *>(R->dev_gm), dim, p, a.n[0], a.n[1],
                                                    a.N[0], a.N[1], a.N[2], a.ntot, coef, coef32, ncoef,
                                                    R->dev_status);
    if (cudaGetLastError() != cudaSuccess) return WQ_ERR_CUDA;
  }
  for (const auto &sl : slabs) {
    a.slab_lo = offs[sl.first];
    a.slab_n = offs[sl.second + 1] - offs[sl.first];
    a.fstride = (long long)a.np[0] * (dim == 3 ? a.np[1] : 1) * a.slab_n;
    a.row_begin = std::max((long long)row_begin, sl.first * plane);
    a.row_end = std::min((long long)row_end, (sl.second + 1) * plane);
    const long long nch1 = (a.np[0] + kGmChunk - 1) / kGmChunk;
    const int r2b = f32 ? kGmRows32 : kGmRows64;
    const long long nitems = dim == 3 ? 6LL * a.slab_n * ((R->n[1] + r2b - 1) / r2b) * nch1 : 3LL * a.slab_n * nch1;
    if (nitems > 0x7fffffffLL) return WQ_ERR_UNSUPPORTED;
    // the rows of each class in the slab's planes (the row kernels enumerate them)
    a.bp_lo = sl.first;
    a.bp_hi = sl.second;
    long long ncls[5];
    class_counts(dim, p, R->n, R->nel, sl.first, sl.second, ncls);
    wq_status st = f32 ? launch_any<float>(p, dim, a, nitems, ncls, s) : launch_any<double>(p, dim, a, nitems, ncls, s);
    if (st != WQ_OK) return st;
  }
  return WQ_OK;
}
