// Row-wise weighted-quadrature assembly kernel (sum factorisation into the
// band), templated on degree P, dimension D, point capacity LM of the inner
// directions, chunk length TMAX, the terms (DO_M, DO_K) and the arithmetic
// type R (double; float for the mixed mode; dd, double-float on the FP32
// pipe, for FP64 accuracy at FP32 throughput).
//
// A CTA owns a chunk of consecutive rows along x1 that share (r2, r3), one
// "line" of rows; their rules in directions 2..D coincide.  Writing term g's
// band entries as
//   A_g[j1][j2][j3] = sum_{q1} V1[q1][j1] sum_{l1} b1_{q1}[l1] U_g[l1][j2][j3],
//   U_g[l1][j2][j3] = sum_{q2,q3} c_{l1}(x_q2, x_q3) V2[q2][j2] V3[q3][j3],
// where c_{l1}(.,.) = sum_{l2,l3} C[l1][l2][l3] b2(.)[l2] b3(.)[l3] is the
// coefficient spline's column l1 and b the cubic B-spline values at the
// points (Eq. Decompo applied to the weighted sums of Eq. GaussQuadSys and
// Eq. GaussQuadSysStiff, with c as the integrand's factor), U depends only on
// the line.  Phase A builds U for the chunk's coefficient columns, one
// direction at a time (x3 then x2), for the two combinations the terms need:
//   U0: mass kind in x2 and x3           (terms M and K1)
//   U1: stiffness kind in x2 + in x3     (K2 + K3, summed)
// one warp per column.  Phase B spreads (row, band fibre (j2, j3)) items
// over the CTA's threads, a group of rows at a time; at each x1 point of its
// row a thread forms
//   y_M = b1M . U0,  y_K = b1M . U1,  y_S = b1S . U0
// and accumulates A_M += V1M y_M, A_K += V1M y_K + V1S y_S over the 2P+1
// entries j1 of the fibre; the group's bands are staged in shared memory and
// written with consecutive threads on consecutive addresses.  The folded 1D
// tables hold W * |J_aa| (mass kind) or W / |J_aa| (stiffness kind), so no
// other per-point factor remains.  Rows whose x1 rule is the weighted Gaussian
// one (P+1 points, one per element) take an unrolled path; boundary rows
// (Gauss-Legendre per element) a general one.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "checked.cuh"
#include "dd.cuh"

namespace wq {

struct RowsArgs {
  const int *off[3][2];
  const int *elem[3][2];
  const void *V[3][2];     // folded tables in the arithmetic type R, npts*(P+1)
  const void *beta[3][2];  // cubic coefficient-spline values in R, npts*4
  int n[3], N[3], nc[3];
  const double *coef;  // may be null: c = 1
  const void *coefR;   // the same already in the arithmetic type R (and checked), or null
  void *M, *K;         // band outputs, OutT<R> (double for R = double or dd)
  long long row_begin, row_end;
  const int *lines;  // line ids of this launch, or null: lines line0, line0+1, ...
  int line0;
  int nch, T;        // chunks per line and chunk length
  const void *Ug;    // U of every line, [line][2][nc1][(2P+1)^2] in R (split 3D path)
  unsigned *status;
  float zero;  // 0.0f, read at run time by the packed double-float path (dd2_fma)
  // matrix-free apply (rows_phase_b with APPLY): M and K above then receive
  // y = M x and y = K x, one OutT<R> value per row of [row_begin, row_end);
  // x holds one OutT<R> value per row of the whole mesh, or is null for x = 1
  const void *x;
  // 1: every boundary x1 row holds P+1 points per element of its support in
  // element order (Gauss-Legendre), processed element by element; 0: the
  // general per-point form
  int bnd_grouped;
};

// Asynchronous global -> shared copies of one 4- or 8-byte element
// (cp.async): complete in the issuing thread after cp_async_wait_all(),
// visible to the CTA after a barrier.
template <typename T> __device__ __forceinline__ void cp_async_el(T *sdst, const T *gsrc) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
// n consecutive elements, strided over the threads tid, tid + nt, ...
template <typename T> __device__ __forceinline__ void cp_async_n(T *sdst, const T *gsrc, int n, int tid, int nt) {
  for (int i = tid; i < n; i += nt) cp_async_el(sdst + i, gsrc + i);
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bulk asynchronous shared -> global copy (cp.async.bulk, bulk-group
// completion): both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_store_s2g(void *gdst, const void *ssrc, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst),
               "r"((unsigned)__cvta_generic_to_shared(ssrc)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// Waits until the committed bulk copies of this thread have read their source.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// Makes this thread's shared-memory writes visible to the bulk copies.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Writes n floats of a stage to g: the 16-byte-aligned middle by one bulk
// copy (thread `issuer`), the at most three entries on either side by plain
// stores (threads helper0 ..); s is positioned so that s[i] and g[i] agree
// modulo 16 bytes.  The caller fences, synchronises and commits.
__device__ __forceinline__ void stage_out(float *g, const float *s, int n, int tid, int issuer, int helper0) {
  const int head = min((int)((4 - (((uintptr_t)g >> 2) & 3)) & 3), n);
  const int mid = (n - head) / 4 * 4;
  const int tail = n - head - mid;
  if (tid == issuer && mid > 0) bulk_store_s2g(g + head, s + head, (unsigned)mid * 4u);
  const int h = tid - helper0;
  if (h >= 0 && h < head) g[h] = s[h];
  if (h >= head && h < head + tail) g[mid + h] = s[mid + h];  // entries head + mid .. n - 1
}

// acc[o + i] += x * v[i], i = 0..P, with a compile-time register index in
// each case.
template <int P, int O, typename R, typename VT>
__device__ __forceinline__ void fiber_at(R (&acc)[2 * P + 1], R x, VT v) {
#pragma unroll
  for (int i = 0; i <= P; i++) acc[O + i] = r_fma(x, v[i], acc[O + i]);
}

template <int P, typename R, typename VT>
__device__ __forceinline__ void fiber_add(R (&acc)[2 * P + 1], R x, VT v, int o) {
  switch (o) {
    case 0: fiber_at<P, 0>(acc, x, v); break;
    case 1: fiber_at<P, 1>(acc, x, v); break;
    case 2: fiber_at<P, 2>(acc, x, v); break;
    default:
      if constexpr (P >= 3) fiber_at<P, (P >= 3 ? 3 : 0)>(acc, x, v);
      break;
  }
}

constexpr int kRowsWarps = 8;

// acc[j] += x * vd[j] over the whole band width, vd zero outside the point's
// P+1 columns (used where the band offset varies from point to point).
template <int NB, typename R>
__device__ __forceinline__ void fiber_dense(R (&acc)[NB], R x, const R *__restrict__ vd) {
#pragma unroll
  for (int j = 0; j < NB; j++) acc[j] = r_fma(x, vd[j], acc[j]);
}

// One point's update of a band fibre whose offset o varies from point to
// point: for double, P+1 multiply-adds through a switch on o (the FP64 pipe
// is the bound); for float and double-float, the dense NB-wide form (a
// little more arithmetic, no branching or code replication).
template <int P, typename R>
__device__ __forceinline__ void fiber_point(R (&acc)[2 * P + 1], R x, const R *__restrict__ v,
                                            const R *__restrict__ vd, int o) {
  if constexpr (sizeof(R) == 8 && !std::is_same<R, dd>::value) fiber_add<P>(acc, x, v, o);
  else fiber_dense<2 * P + 1>(acc, x, vd);
}

// acc[o + i] += x * v[i], i = 0..P, for a runtime offset o in [0, P]: the
// switch form for double and float (every call site has o uniform across a
// warp, or nearly so), the dense NB-wide form with the point's P+1 columns
// selected by comparison for double-float.  The two forms give the same
// values: the dense form's extra terms add x * 0 to entries that start at +0
// and never become -0.
template <int P, typename R, typename VT>
__device__ __forceinline__ void fiber_shift(R (&acc)[2 * P + 1], R x, VT v, int o) {
  if constexpr (!std::is_same<R, dd>::value) {
    fiber_add<P>(acc, x, v, o);
  } else {
#pragma unroll
    for (int j = 0; j < 2 * P + 1; j++) {
      const int i = j - o;
      const R vv = v[i < 0 ? 0 : (i > P ? P : i)];
      acc[j] = r_fma(x, (i >= 0 && i <= P) ? vv : r_zero<R>(), acc[j]);
    }
  }
}

// Double-float mass and stiffness updates of one point at band offset O,
// packed: (aM, aK)[O+i] += (y, yk) vm[i], then aK[O+i] += ys vs[i], with
// yy = (y, yk) and aMK[j] = (aM[j], aK[j]); the operand order of every
// multiply-add is fiber_shift's, so the bits are those of the unpacked path.
template <int P, int O, typename VT>
__device__ __forceinline__ void fiber_mk_at(dd2 (&aMK)[2 * P + 1], dd2 yy, dd ys, VT vm, VT vs, unsigned long long z) {
#pragma unroll
  for (int i = 0; i <= P; i++) {
    const dd v = vm[i];
    const dd2 t = dd2_fma(yy, dd2_pack(v, v), aMK[O + i], z);
    aMK[O + i] = dd2_with_second(t, dd_fma(ys, vs[i], dd2_second(t)));
  }
}

// Rounds a region size up to whole 16-byte units of R.
template <typename R> constexpr int pad16(int n) {
  return (n * (int)sizeof(R) + 15) / 16 * 16 / (int)sizeof(R);
}

// Per-warp band stage of phase B, in values of R: for float one buffer per
// matrix, each one run of kBulkSub x 32 items plus three entries of alignment slack, written
// to global memory by bulk copies; otherwise one buffer for both matrices in
// turn, written by the warp's lanes.
template <typename R, int NB, bool APPLY> constexpr bool bulk_stage() {
  return std::is_same<R, float>::value && !APPLY;
}
constexpr int kBulkSub = 2;  // 32-item sub-runs per bulk run
template <typename R, int NB> constexpr int stage_run() { return pad16<R>(32 * kBulkSub * NB + 3); }
template <typename R, int NB, bool APPLY> constexpr int stage_per_warp() {
  return bulk_stage<R, NB, APPLY>() ? 2 * stage_run<R, NB>() : pad16<R>(32 * NB);
}

template <int P, int D, int LM, int TMAX, bool DO_M, bool DO_K, typename R, bool APPLY = false>
struct RowsLayout {
  static constexpr int NP = P + 1;             // points of a weighted Gaussian rule
  static constexpr int NB = 2 * P + 1;         // band width per direction
  static constexpr int NPAIR = (D == 3) ? NB * NB : NB;  // (j2, j3) fibres of a row
  static constexpr int BAND = NPAIR * NB;
  static constexpr int NSLOT = (NPAIR + 31) / 32;       // fibres per lane
  static constexpr int LS = NPAIR;             // U's stride between coefficient columns
  static constexpr int NU = DO_K ? 2 : 1;
  static constexpr int NK3 = (D == 3) ? (DO_K ? 2 : 1) : 0;  // kinds in x3
  static constexpr int NCOMBO = DO_K ? D : 1;  // (kind2, kind3) combinations
  static constexpr int NL1 = TMAX + P + 3;     // coefficient columns of a chunk
  static constexpr int NL = P + 4;             // coefficient indices of one row per direction
  static constexpr int NL3 = (D == 3) ? NL : 1;
  static constexpr int NW = kRowsWarps;
  static constexpr int NT = 32 * NW;
  // general class (the comparison rules): up to (P+1)^2 points per row and
  // direction, every row through the general x1 path
  static constexpr bool GENERAL = (LM > P * (P + 1));
  static constexpr int MAXPTS1 = GENERAL ? TMAX * NP * NP : TMAX * NP + P * NP * (P - 1);  // x1 points of a chunk
  // per-warp scratch: phase A's column work (Z/Cq, then T3) or phase B's band stage
  static constexpr int WZ = (D == 3) ? NK3 * NL * LM : 0;
  static constexpr int WC = (D == 3) ? NCOMBO * LM * NB : NCOMBO * LM;
  static constexpr int WX = WZ > WC ? WZ : WC;
  static constexpr int WT = (D == 3) ? NK3 * NL * NB : 0;
  static constexpr int WA = WX + WT;
  static constexpr int WS = pad16<R>(WA);  // phase A, per half-warp
  // phase B: per-warp stage of 32 items' fibres, one matrix at a time
  static constexpr int WST = stage_per_warp<R, NB, APPLY>();
  static constexpr int SCRATCH0 = (2 * NW * WS) > (NW * WST) ? (2 * NW * WS) : (NW * WST);
  // apply: phase B's per-fibre partial sums share the scratch; x gets its own region
  static constexpr int PART = pad16<R>(2 * TMAX * NPAIR);
  static constexpr int SCRATCH = (APPLY && PART > SCRATCH0) ? PART : SCRATCH0;
  static constexpr int XS = APPLY ? pad16<R>(NPAIR * (TMAX + 2 * P)) : 0;
  // R region
  static constexpr bool INNER_GAUSS = (LM == P + 1);  // interior line: o = q in x2, x3
  // every region is a whole number of 16-byte units, so 4-wide float rows stay aligned
  static constexpr int V23 = pad16<R>(2 * 2 * LM * NP);  // [dir2/3][kind][q][i]
  static constexpr int V23D = INNER_GAUSS ? 0 : pad16<R>(2 * 2 * LM * NB);  // zero-padded [..][q][j]
  static constexpr int B23 = pad16<R>(2 * 2 * LM * 4);
  static constexpr int V1 = pad16<R>(2 * MAXPTS1 * NP);  // [kind][point][i]
  static constexpr int B1 = pad16<R>(2 * MAXPTS1 * 4);
  static constexpr int CB = pad16<R>(NL3 * NL * NL1);    // [l3][l2][l1]
  static constexpr int US = pad16<R>(NU * NL1 * LS);     // [u][l1][j3*NB+j2]
  static constexpr int R_TOTAL = V23 + V23D + B23 + V1 + B1 + CB + US + SCRATCH + XS;
  // int region: E23[2][LM], O23[2][LM], E1[MAXPTS1], OFF1[TMAX+1]
  static constexpr int I_TOTAL = 4 * LM + MAXPTS1 + TMAX + 1;
  static constexpr size_t BYTES = sizeof(R) * (size_t)R_TOTAL + sizeof(int) * (size_t)I_TOTAL;
};

// Resident CTAs per SM the compiler is asked to allow (caps registers at
// 65536 / (threads * minblocks)): four for float, three for double-float,
// two for double.
#ifndef WQ_ROWS_MIN_BLOCKS_F32
#define WQ_ROWS_MIN_BLOCKS_F32 4
#endif
#ifndef WQ_ROWS_MIN_BLOCKS
#define WQ_ROWS_MIN_BLOCKS 2
#endif
#ifndef WQ_ROWS_MIN_BLOCKS_DD
#define WQ_ROWS_MIN_BLOCKS_DD 3
#endif
template <typename R> constexpr int rows_min_blocks() {
  return sizeof(R) == 4 ? WQ_ROWS_MIN_BLOCKS_F32 : std::is_same<R, dd>::value ? WQ_ROWS_MIN_BLOCKS_DD : WQ_ROWS_MIN_BLOCKS;
}

// Position of entry i of kind k (0: mass factors, 1: stiffness factors) of
// point q in an x1 table with W entries per point.  For double the two kinds
// are interleaved entry by entry, so that an (M, S) pair is one 16-byte load
// (the FP64 row kernel measured 3 % faster so); float and double-float keep
// one block per kind, whose runs of four entries their 16-byte loads take.
template <typename R, int MAXPTS1, int W> __device__ __forceinline__ int x1_idx(int q, int i, int k) {
  if constexpr (std::is_same<R, double>::value) return 2 * (q * W + i) + k;
  else return (k * MAXPTS1 + q) * W + i;
}

// Entries 0.. of one kind of one point of an x1 table, indexable like a pointer.
template <typename R, int MAXPTS1, int W> struct X1Row {
  static constexpr int S = std::is_same<R, double>::value ? 2 : 1;  // entry stride
  const R *v;
  __device__ __forceinline__ X1Row(const R *t, int q, int k) : v(t + x1_idx<R, MAXPTS1, W>(q, 0, k)) {}
  __device__ __forceinline__ R operator[](int i) const { return v[i * S]; }
};

// The chunk's x1 tables (rows [a, a+T) hold one contiguous range of points):
// point offsets per row, folded values and cubic coefficient-spline values of
// both kinds, elements, by asynchronous copies: the caller waits for them
// (cp_async_wait_all) and synchronises.
template <int P, int MAXPTS1, typename R>
__device__ __forceinline__ void load_x1_tables(const RowsArgs &A, const int a, const int T, R *sV1, R *sB1, int *sE1,
                                               int *sOff1) {
  constexpr int NP = P + 1, NT = 32 * kRowsWarps;
  const int tid = threadIdx.x;
  const int p1lo = A.off[0][0][a], p1hi = A.off[0][0][a + T];
  const int np1 = p1hi - p1lo;
  for (int t = tid; t <= T; t += NT) sOff1[t] = A.off[0][0][a + t] - p1lo;
  for (int t = tid; t < 2 * np1; t += NT) {
    const int kind = t >= np1 ? 1 : 0, q = t - kind * np1;
    const int gq = (kind ? A.off[0][1][a] : p1lo) + q;
    const R *Vg = static_cast<const R *>(A.V[0][kind]);
    const R *Bg = static_cast<const R *>(A.beta[0][kind]);
#pragma unroll
    for (int i = 0; i < NP; i++) cp_async_el(&sV1[x1_idx<R, MAXPTS1, NP>(q, i, kind)], &Vg[(size_t)gq * NP + i]);
#pragma unroll
    for (int i = 0; i < 4; i++) cp_async_el(&sB1[x1_idx<R, MAXPTS1, 4>(q, i, kind)], &Bg[(size_t)gq * 4 + i]);
    if (kind == 0) cp_async_el(&sE1[q], &A.elem[0][0][p1lo + q]);
  }
}

// The P+1 Gauss-Legendre points q .. q+P of one element, at band offset O,
// of a boundary x1 row: per point y_M = b1M . u0, y_K = b1M . u1,
// y_S = b1S . u0 and the updates of fiber_shift, in the same order.
template <int P, int O, int MAXPTS1, bool DO_M, bool DO_K, typename R>
__device__ __forceinline__ void gl_element(R (&accM)[2 * P + 1], R (&accK)[2 * P + 1], const R (&u0)[4],
                                           const R (&u1)[4], const R *sB1, const R *sV1, const int q) {
  constexpr int NP = P + 1;
#pragma unroll
  for (int qq = 0; qq < NP; qq++) {
    R bm[4], bs[4], vm[NP], vs[NP];
    if constexpr (std::is_same<R, float>::value && NP == 4) {
      const float4 b4m = reinterpret_cast<const float4 *>(&sB1[(0 * MAXPTS1 + q + qq) * 4])[0];
      const float4 b4s = reinterpret_cast<const float4 *>(&sB1[(1 * MAXPTS1 + q + qq) * 4])[0];
      const float4 v4m = reinterpret_cast<const float4 *>(&sV1[(0 * MAXPTS1 + q + qq) * NP])[0];
      const float4 v4s = reinterpret_cast<const float4 *>(&sV1[(1 * MAXPTS1 + q + qq) * NP])[0];
      bm[0] = b4m.x; bm[1] = b4m.y; bm[2] = b4m.z; bm[3] = b4m.w;
      bs[0] = b4s.x; bs[1] = b4s.y; bs[2] = b4s.z; bs[3] = b4s.w;
      vm[0] = v4m.x; vm[1] = v4m.y; vm[2] = v4m.z; vm[3] = v4m.w;
      vs[0] = v4s.x; vs[1] = v4s.y; vs[2] = v4s.z; vs[3] = v4s.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        bm[i] = sB1[x1_idx<R, MAXPTS1, 4>(q + qq, i, 0)];
        bs[i] = sB1[x1_idx<R, MAXPTS1, 4>(q + qq, i, 1)];
      }
#pragma unroll
      for (int i = 0; i < NP; i++) {
        vm[i] = sV1[x1_idx<R, MAXPTS1, NP>(q + qq, i, 0)];
        vs[i] = sV1[x1_idx<R, MAXPTS1, NP>(q + qq, i, 1)];
      }
    }
    if constexpr (DO_M) {
      R y = r_zero<R>();
#pragma unroll
      for (int i = 0; i < 4; i++) y = r_fma(bm[i], u0[i], y);
      fiber_at<P, O>(accM, y, vm);
    }
    if constexpr (DO_K) {
      R yk = r_zero<R>(), ys = r_zero<R>();
#pragma unroll
      for (int i = 0; i < 4; i++) {
        yk = r_fma(bm[i], u1[i], yk);
        ys = r_fma(bs[i], u0[i], ys);
      }
      fiber_at<P, O>(accK, yk, vm);
      fiber_at<P, O>(accK, ys, vs);
    }
  }
}

// Phase B of the row kernel: (row, fibre) items, 32 per warp.  sU holds U0
// and U1 for the chunk's coefficient columns l1lo .. l1lo+NL1-1 ([u][NL1][NPAIR]);
// sV1, sB1, sE1, sOff1 the chunk's x1 tables; sW at least NW * 32 * pad16(2P+1)
// values of per-warp stage.
// APPLY: instead of the band, y = M x and y = K x for the chunk's rows.  sX
// holds x at the chunk's columns, [fibre][NL1 + P - 3] from column a - P (zero
// outside the mesh); sW then holds 2 * T * NPAIR per-fibre partial sums, and
// the call ends with a CTA-wide barrier.
template <int P, int D, int MAXPTS1, int NL1, bool GENERAL, bool DO_M, bool DO_K, typename R, bool APPLY = false>
__device__ __forceinline__ void rows_phase_b(const RowsArgs &A, const R *sU, const R *sV1, const R *sB1,
                                             const int *sE1, const int *sOff1, R *sW, const int a, const int T,
                                             const int l1lo, const long long base, const R *sX = nullptr) {
  using O = typename OutT<R>::type;
  constexpr int NP = P + 1, NB = 2 * P + 1, NT = 32 * kRowsWarps;
  constexpr int NPAIR = (D == 3) ? NB * NB : NB, BAND = NPAIR * NB, LS = NPAIR;
  constexpr bool BULK = bulk_stage<R, NB, APPLY>();
  constexpr int WST = stage_per_warp<R, NB, APPLY>(), WSTB = stage_run<R, NB>();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ------------------------------------------------ phase B: (row, fibre) items, 32 per warp
  // Item i of the chunk is fibre i % NPAIR of row i / NPAIR; its 2P+1 band
  // entries sit at offset i * NB of the chunk's output rows, so a warp's 32
  // consecutive items own one contiguous run of 32 * NB entries per matrix.
  // The warp stages that run in shared memory; in float (BULK) one lane
  // writes its 16-byte-aligned middle with a bulk asynchronous copy per
  // matrix and lanes store the ends, otherwise the warp's lanes write it
  // with consecutive lanes on consecutive addresses, converting to the
  // output type there.  No CTA-wide barrier is needed.
  const R *U0 = sU;
  const R *U1 = sU + NL1 * LS;
  R *wst = sW + warp * WST;  // [32][NB]
  const int nitems = T * NPAIR;
  const long long ochunk = (base + a - A.row_begin) * BAND;
  // in float a warp's consecutive iterations take consecutive 32-item
  // sub-runs (kBulkSub per run, written out together)
  constexpr int SUB = BULK ? kBulkSub : 1;
  for (int it = 0;; it++) {
    const int ib = warp * 32 * SUB + (it / SUB) * NT * SUB + (it % SUB) * 32;
    if (ib >= nitems) break;
    const int item = ib + lane;
    R oM[NB], oK[NB];
    if (item < nitems) {
      const int rl = item / NPAIR, pr = item - rl * NPAIR;
      const int r1 = a + rl;
      const int q0 = sOff1[rl], q1end = sOff1[rl + 1];
      if (!GENERAL && r1 >= P && r1 <= A.N[0] - 1) {
        // weighted Gaussian rule in x1: point q in element r1-P+q, band
        // offset q; the row's coefficient columns kb .. kb+P+3
        const int kb = (r1 - P) - l1lo;
        if constexpr (std::is_same<R, dd>::value && DO_M && DO_K && NP == 4) {
          // double-float with M and K side by side in packed pairs: the terms
          // sharing an operand (b1M with U0 and U1; V1M with y_M and y_K) run as
          // one packed multiply-add, the rest (y_S, V1S y_S) as before
          const unsigned long long z = f2_pack(A.zero, A.zero);
          dd2 w01[NP + 3], aMK[NB];
#pragma unroll
          for (int i = 0; i < NP + 3; i++) w01[i] = dd2_pack(U0[(kb + i) * LS + pr], U1[(kb + i) * LS + pr]);
#pragma unroll
          for (int j = 0; j < NB; j++) aMK[j] = dd2{z, z};
          const float4 *b4m = reinterpret_cast<const float4 *>(&sB1[(0 * MAXPTS1 + q0) * 4]);
          const float4 *b4s = reinterpret_cast<const float4 *>(&sB1[(1 * MAXPTS1 + q0) * 4]);
          const float4 *v4m = reinterpret_cast<const float4 *>(&sV1[(0 * MAXPTS1 + q0) * NP]);
          const float4 *v4s = reinterpret_cast<const float4 *>(&sV1[(1 * MAXPTS1 + q0) * NP]);
#pragma unroll
          for (int q = 0; q < NP; q++) {
            dd bm[4], bs[4], vm[4], vs[4];
#pragma unroll
            for (int h = 0; h < 2; h++) {
              const float4 x = b4m[2 * q + h], y = b4s[2 * q + h], z = v4m[2 * q + h], w = v4s[2 * q + h];
              bm[2 * h] = dd{x.x, x.y}; bm[2 * h + 1] = dd{x.z, x.w};
              bs[2 * h] = dd{y.x, y.y}; bs[2 * h + 1] = dd{y.z, y.w};
              vm[2 * h] = dd{z.x, z.y}; vm[2 * h + 1] = dd{z.z, z.w};
              vs[2 * h] = dd{w.x, w.y}; vs[2 * h + 1] = dd{w.z, w.w};
            }
            dd2 yMK{z, z};
            dd ys = r_zero<dd>();
#pragma unroll
            for (int i = 0; i < 4; i++) {
              yMK = dd2_fma(dd2_pack(bm[i], bm[i]), w01[q + i], yMK, z);
              ys = dd_fma(bs[i], dd2_first(w01[q + i]), ys);
            }
#pragma unroll
            for (int i = 0; i < NP; i++) {
              const dd2 t = dd2_fma(dd2_pack(vm[i], vm[i]), yMK, aMK[q + i], z);
              aMK[q + i] = dd2_with_second(t, dd_fma(vs[i], ys, dd2_second(t)));
            }
          }
#pragma unroll
          for (int j = 0; j < NB; j++) {
            oM[j] = dd2_first(aMK[j]);
            oK[j] = dd2_second(aMK[j]);
          }
        } else if constexpr (std::is_same<R, float>::value && DO_M && DO_K && NP == 4) {
          // float with M and K side by side in packed pairs: (y_M, y_K) share
          // b1M and (A_M, A_K) share V1M, one fma.rn.f32x2 each; y_S and the
          // V1S y_S update stay scalar.  Every lane performs the scalar path's
          // multiply-adds in its order (16 instead of 24 instructions a point).
          const unsigned long long z = f2_pack(A.zero, A.zero);
          unsigned long long w01[NP + 3], aMK[NB];
          float w0[NP + 3];
#pragma unroll
          for (int i = 0; i < NP + 3; i++) {
            w0[i] = U0[(kb + i) * LS + pr];
            w01[i] = f2_pack(w0[i], U1[(kb + i) * LS + pr]);
          }
#pragma unroll
          for (int j = 0; j < NB; j++) aMK[j] = z;
          const float4 *b4m = reinterpret_cast<const float4 *>(&sB1[(0 * MAXPTS1 + q0) * 4]);
          const float4 *b4s = reinterpret_cast<const float4 *>(&sB1[(1 * MAXPTS1 + q0) * 4]);
          const float4 *v4m = reinterpret_cast<const float4 *>(&sV1[(0 * MAXPTS1 + q0) * NP]);
          const float4 *v4s = reinterpret_cast<const float4 *>(&sV1[(1 * MAXPTS1 + q0) * NP]);
#pragma unroll
          for (int q = 0; q < NP; q++) {
            const float4 xm = b4m[q], xs = b4s[q], ym = v4m[q], ys4 = v4s[q];
            const float bm[4] = {xm.x, xm.y, xm.z, xm.w}, bs[4] = {xs.x, xs.y, xs.z, xs.w};
            const float vm[4] = {ym.x, ym.y, ym.z, ym.w}, vs[4] = {ys4.x, ys4.y, ys4.z, ys4.w};
            unsigned long long yMK = z;
            float ys = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; i++) {
              yMK = f2_fma(f2_pack(bm[i], bm[i]), w01[q + i], yMK);
              ys = fmaf(bs[i], w0[q + i], ys);
            }
#pragma unroll
            for (int i = 0; i < NP; i++) {
              float m, k;
              f2_unpack(f2_fma(f2_pack(vm[i], vm[i]), yMK, aMK[q + i]), m, k);
              aMK[q + i] = f2_pack(m, fmaf(vs[i], ys, k));
            }
          }
#pragma unroll
          for (int j = 0; j < NB; j++) {
            float m, k;
            f2_unpack(aMK[j], m, k);
            oM[j] = m;
            oK[j] = k;
          }
        } else {
        R w0[NP + 3], w1[NP + 3], aM[NB], aK[NB];
#pragma unroll
        for (int i = 0; i < NP + 3; i++) {
          w0[i] = U0[(kb + i) * LS + pr];
          w1[i] = DO_K ? U1[(kb + i) * LS + pr] : r_zero<R>();
        }
#pragma unroll
        for (int j = 0; j < NB; j++) {
          aM[j] = r_zero<R>();
          aK[j] = r_zero<R>();
        }
        const R *bm0 = &sB1[(0 * MAXPTS1 + q0) * 4];
        const R *bs0 = &sB1[(1 * MAXPTS1 + q0) * 4];
        const R *vm0 = &sV1[(0 * MAXPTS1 + q0) * NP];
        const R *vs0 = &sV1[(1 * MAXPTS1 + q0) * NP];
#pragma unroll
        for (int q = 0; q < NP; q++) {
          R bm[4], vm[NP], bs[4], vs[NP];
          if constexpr (std::is_same<R, float>::value && NP == 4) {
            const float4 b4m = reinterpret_cast<const float4 *>(bm0)[q], b4s = reinterpret_cast<const float4 *>(bs0)[q];
            const float4 v4m = reinterpret_cast<const float4 *>(vm0)[q], v4s = reinterpret_cast<const float4 *>(vs0)[q];
            bm[0] = b4m.x; bm[1] = b4m.y; bm[2] = b4m.z; bm[3] = b4m.w;
            bs[0] = b4s.x; bs[1] = b4s.y; bs[2] = b4s.z; bs[3] = b4s.w;
            vm[0] = v4m.x; vm[1] = v4m.y; vm[2] = v4m.z; vm[3] = v4m.w;
            vs[0] = v4s.x; vs[1] = v4s.y; vs[2] = v4s.z; vs[3] = v4s.w;
          } else if constexpr (std::is_same<R, dd>::value && NP == 4) {
            // two double-float values per 16-byte load (rows of 4 values are 32-byte aligned)
            const float4 *b4m = reinterpret_cast<const float4 *>(bm0) + 2 * q;
            const float4 *b4s = reinterpret_cast<const float4 *>(bs0) + 2 * q;
            const float4 *v4m = reinterpret_cast<const float4 *>(vm0) + 2 * q;
            const float4 *v4s = reinterpret_cast<const float4 *>(vs0) + 2 * q;
#pragma unroll
            for (int h = 0; h < 2; h++) {
              const float4 x = b4m[h], y = b4s[h], z = v4m[h], w = v4s[h];
              bm[2 * h] = dd{x.x, x.y}; bm[2 * h + 1] = dd{x.z, x.w};
              bs[2 * h] = dd{y.x, y.y}; bs[2 * h + 1] = dd{y.z, y.w};
              vm[2 * h] = dd{z.x, z.y}; vm[2 * h + 1] = dd{z.z, z.w};
              vs[2 * h] = dd{w.x, w.y}; vs[2 * h + 1] = dd{w.z, w.w};
            }
          } else {
#pragma unroll
            for (int i = 0; i < 4; i++) {
              bm[i] = sB1[x1_idx<R, MAXPTS1, 4>(q0 + q, i, 0)];
              bs[i] = sB1[x1_idx<R, MAXPTS1, 4>(q0 + q, i, 1)];
            }
#pragma unroll
            for (int i = 0; i < NP; i++) {
              vm[i] = sV1[x1_idx<R, MAXPTS1, NP>(q0 + q, i, 0)];
              vs[i] = sV1[x1_idx<R, MAXPTS1, NP>(q0 + q, i, 1)];
            }
          }
          if constexpr (DO_M) {
            R y = r_zero<R>();
#pragma unroll
            for (int i = 0; i < 4; i++) y = r_fma(bm[i], w0[q + i], y);
#pragma unroll
            for (int i = 0; i < NP; i++) aM[q + i] = r_fma(vm[i], y, aM[q + i]);
          }
          if constexpr (DO_K) {
            R yk = r_zero<R>(), ys = r_zero<R>();
#pragma unroll
            for (int i = 0; i < 4; i++) {
              yk = r_fma(bm[i], w1[q + i], yk);
              ys = r_fma(bs[i], w0[q + i], ys);
            }
#pragma unroll
            for (int i = 0; i < NP; i++) aK[q + i] = r_fma(vs[i], ys, r_fma(vm[i], yk, aK[q + i]));
          }
        }
#pragma unroll
        for (int j = 0; j < NB; j++) {
          if constexpr (DO_M) oM[j] = aM[j];
          if constexpr (DO_K) oK[j] = aK[j];
        }
        }
      } else {
        // Gauss-Legendre on each element of supp B_r1 (or a comparison rule):
        // any number of points, each with its own band offset o
        if constexpr (std::is_same<R, dd>::value && DO_M && DO_K) {
          // double-float: the interior path's packed (M, K) pairs, P+1
          // updates per point through a switch on o (uniform across a warp's
          // items of one row; 5 % faster at 64^3 than the dense form)
          const unsigned long long z = f2_pack(A.zero, A.zero);
          dd2 aMK[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) aMK[j] = dd2{z, z};
          for (int q = q0; q < q1end; q++) {
            const int e = sE1[q];
            const int k0 = e - l1lo, o = e - r1 + P;
            const X1Row<R, MAXPTS1, 4> bm{sB1, q, 0}, bs{sB1, q, 1};
            const X1Row<R, MAXPTS1, NP> vm{sV1, q, 0}, vs{sV1, q, 1};
            dd2 yy{z, z};
            dd ys = r_zero<dd>();
#pragma unroll
            for (int i = 0; i < 4; i++) {
              const dd w0 = U0[(k0 + i) * LS + pr], w1 = U1[(k0 + i) * LS + pr];
              const dd b = bm[i];
              yy = dd2_fma(dd2_pack(b, b), dd2_pack(w0, w1), yy, z);
              ys = dd_fma(bs[i], w0, ys);
            }
            switch (o) {
              case 0: fiber_mk_at<P, 0>(aMK, yy, ys, vm, vs, z); break;
              case 1: fiber_mk_at<P, 1>(aMK, yy, ys, vm, vs, z); break;
              case 2: fiber_mk_at<P, 2>(aMK, yy, ys, vm, vs, z); break;
              default:
                if constexpr (P >= 3) fiber_mk_at<P, (P >= 3 ? 3 : 0)>(aMK, yy, ys, vm, vs, z);
                break;
            }
          }
#pragma unroll
          for (int j = 0; j < NB; j++) {
            oM[j] = dd2_first(aMK[j]);
            oK[j] = dd2_second(aMK[j]);
          }
        } else if (!GENERAL && A.bnd_grouped) {
          // Gauss-Legendre rows: P+1 points in each element of the support,
          // in element order; per element its four coefficient columns are
          // loaded once and its band offset selects compile-time indices
          // (the per-point order of the general form below is kept)
          R accM[NB], accK[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) { accM[j] = r_zero<R>(); accK[j] = r_zero<R>(); }
          for (int q = q0; q < q1end; q += NP) {
            const int e = sE1[q];
            const int k0 = e - l1lo, o = e - r1 + P;
            R u0[4], u1[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
              u0[i] = U0[(k0 + i) * LS + pr];
              u1[i] = DO_K ? U1[(k0 + i) * LS + pr] : r_zero<R>();
            }
            switch (o) {
              case 0: gl_element<P, 0, MAXPTS1, DO_M, DO_K>(accM, accK, u0, u1, sB1, sV1, q); break;
              case 1: gl_element<P, 1, MAXPTS1, DO_M, DO_K>(accM, accK, u0, u1, sB1, sV1, q); break;
              case 2: gl_element<P, 2, MAXPTS1, DO_M, DO_K>(accM, accK, u0, u1, sB1, sV1, q); break;
              default:
                if constexpr (P >= 3) gl_element<P, (P >= 3 ? 3 : 0), MAXPTS1, DO_M, DO_K>(accM, accK, u0, u1, sB1, sV1, q);
                break;
            }
          }
#pragma unroll
          for (int j = 0; j < NB; j++) {
            if constexpr (DO_M) oM[j] = accM[j];
            if constexpr (DO_K) oK[j] = accK[j];
          }
        } else {
          R accM[NB], accK[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) { accM[j] = r_zero<R>(); accK[j] = r_zero<R>(); }
          for (int q = q0; q < q1end; q++) {
            const int e = sE1[q];
            const int k0 = e - l1lo, o = e - r1 + P;
            const X1Row<R, MAXPTS1, 4> bm{sB1, q, 0};
            const X1Row<R, MAXPTS1, NP> vm{sV1, q, 0};
            if constexpr (DO_M) {
              R y = r_zero<R>();
#pragma unroll
              for (int i = 0; i < 4; i++) y = r_fma(bm[i], U0[(k0 + i) * LS + pr], y);
              fiber_shift<P>(accM, y, vm, o);
            }
            if constexpr (DO_K) {
              const X1Row<R, MAXPTS1, 4> bs{sB1, q, 1};
              R yk = r_zero<R>(), ys = r_zero<R>();
#pragma unroll
              for (int i = 0; i < 4; i++) {
                yk = r_fma(bm[i], U1[(k0 + i) * LS + pr], yk);
                ys = r_fma(bs[i], U0[(k0 + i) * LS + pr], ys);
              }
              fiber_shift<P>(accK, yk, vm, o);
              fiber_shift<P>(accK, ys, X1Row<R, MAXPTS1, NP>{sV1, q, 1}, o);
            }
          }
#pragma unroll
          for (int j = 0; j < NB; j++) {
            if constexpr (DO_M) oM[j] = accM[j];
            if constexpr (DO_K) oK[j] = accK[j];
          }
        }
      }
    }
    if constexpr (APPLY) {
      // this fibre's share of y: its NB entries times x at their columns
      // (r1 - P + j of the row's x1 index), kept per fibre for the row sums
      if (item < nitems) {
        constexpr int XL = NL1 + P - 3;
        const int rl = item / NPAIR, pr = item - rl * NPAIR;
        const R *xr = sX + pr * XL + rl;
        R pm = r_zero<R>(), pk = r_zero<R>();
        if constexpr (std::is_same<R, dd>::value && DO_M && DO_K) {
          // both sums as one packed pair, each lane dd_fma's bits
          const unsigned long long z = f2_pack(A.zero, A.zero);
          dd2 pmk{z, z};
#pragma unroll
          for (int j = 0; j < NB; j++) pmk = dd2_fma(dd2_pack(oM[j], oK[j]), dd2_pack(xr[j], xr[j]), pmk, z);
          pm = dd2_first(pmk);
          pk = dd2_second(pmk);
        } else {
#pragma unroll
          for (int j = 0; j < NB; j++) {
            if constexpr (DO_M) pm = r_fma(oM[j], xr[j], pm);
            if constexpr (DO_K) pk = r_fma(oK[j], xr[j], pk);
          }
        }
        sW[2 * item] = pm;
        sW[2 * item + 1] = pk;
      }
      continue;
    }
    const int nent = ((nitems - ib) < 32 ? (nitems - ib) : 32) * NB;
    if constexpr (BULK) {
      const int h = it % SUB, ib0 = ib - h * 32;  // sub-run h of the run starting at item ib0
      float *gM = DO_M ? static_cast<float *>(A.M) + ochunk + (long long)ib0 * NB : nullptr;
      float *gK = DO_K ? static_cast<float *>(A.K) + ochunk + (long long)ib0 * NB : nullptr;
      float *sM = wst + (DO_M ? (int)(((uintptr_t)gM >> 2) & 3) : 0);
      float *sK = wst + WSTB + (DO_K ? (int)(((uintptr_t)gK >> 2) & 3) : 0);
      if (h == 0) {
        if (lane == 0) bulk_wait_read();  // the previous run's copies have read the stage
        __syncwarp();
      }
      if (item < nitems) {
#pragma unroll
        for (int j = 0; j < NB; j++) {
          if constexpr (DO_M) sM[(h * 32 + lane) * NB + j] = oM[j];
          if constexpr (DO_K) sK[(h * 32 + lane) * NB + j] = oK[j];
        }
      }
      if (h == SUB - 1 || ib + 32 >= nitems) {
        const int nent = ((nitems - ib0) < 32 * SUB ? (nitems - ib0) : 32 * SUB) * NB;
        fence_proxy_async();
        __syncwarp();
        const bool inb = check_range(A.status, ochunk + (long long)ib0 * NB, nent, (A.row_end - A.row_begin) * BAND);
        if constexpr (DO_M) if (inb) stage_out(gM, sM, nent, lane, 0, 1);
        if constexpr (DO_K) if (inb) stage_out(gK, sK, nent, lane, 0, 8);
        if (lane == 0) bulk_commit();
      }
    } else {
      if constexpr (DO_M) {
        if (item < nitems) {
#pragma unroll
          for (int j = 0; j < NB; j++) wst[lane * NB + j] = oM[j];
        }
        __syncwarp();
        O *gM = static_cast<O *>(A.M) + ochunk + (long long)ib * NB;
        if (check_range(A.status, ochunk + (long long)ib * NB, nent, (A.row_end - A.row_begin) * BAND))
          for (int i = lane; i < nent; i += 32) gM[i] = r_out(wst[i]);
        __syncwarp();
      }
      if constexpr (DO_K) {
        if (item < nitems) {
#pragma unroll
          for (int j = 0; j < NB; j++) wst[lane * NB + j] = oK[j];
        }
        __syncwarp();
        O *gK = static_cast<O *>(A.K) + ochunk + (long long)ib * NB;
        if (check_range(A.status, ochunk + (long long)ib * NB, nent, (A.row_end - A.row_begin) * BAND))
          for (int i = lane; i < nent; i += 32) gK[i] = r_out(wst[i]);
        __syncwarp();
      }
    }
  }
  // the stage is read before the caller may reuse the shared memory
  if constexpr (BULK) {
    if (lane == 0) bulk_wait_read();
    __syncwarp();
  }
  if constexpr (APPLY) {
    // y of each row: the sum of its NPAIR fibre partials, formed by one warp
    // in a fixed order (lane-strided sums, then a butterfly)
    __syncthreads();
    for (int rl = warp; rl < T; rl += kRowsWarps) {
      R sm = r_zero<R>(), sk = r_zero<R>();
      for (int pr = lane; pr < NPAIR; pr += 32) {
        sm = r_add(sm, sW[2 * (rl * NPAIR + pr)]);
        sk = r_add(sk, sW[2 * (rl * NPAIR + pr) + 1]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sm = r_add(sm, r_shfl_xor(sm, o));
        sk = r_add(sk, r_shfl_xor(sk, o));
      }
      if (lane == 0) {
        const long long yi = base + a + rl - A.row_begin;
        if (check_range(A.status, yi, 1, A.row_end - A.row_begin)) {
          if (DO_M && A.M) static_cast<O *>(A.M)[yi] = r_out(sm);
          if (DO_K && A.K) static_cast<O *>(A.K)[yi] = r_out(sk);
        }
      }
    }
  }
}

// x at the band columns of rows a .. a+T-1 of a line (apply): sX[pr][c] =
// x at column (a - P + c) in x1 and, across the line, at the fibre pr's offset
// rows (r2 - P + j2 and, in 3D, r3 - P + j3; pr = j3 (2P+1) + j2); zero
// outside the mesh; x null means x = 1.  XL = T_max + 2P columns per fibre.
template <int P, int D, int XL, typename R>
__device__ __forceinline__ void stage_x(const RowsArgs &A, const int line, const int a, const int T, R *sX) {
  using O = typename OutT<R>::type;
  constexpr int NB = 2 * P + 1, NPAIR = (D == 3) ? NB * NB : NB, NT = 32 * kRowsWarps;
  const O *xg = static_cast<const O *>(A.x);
  const int n1 = A.n[0], n2 = A.n[1], n3 = (D == 3) ? A.n[2] : 1;
  const int r2 = (D == 3) ? line % n2 : line, r3 = (D == 3) ? line / n2 : 0;
  for (int t = threadIdx.x; t < NPAIR * XL; t += NT) {
    const int pr = t / XL, c = t - pr * XL;
    const int c1 = a - P + c, c2 = r2 - P + pr % NB, c3 = (D == 3) ? r3 - P + pr / NB : 0;
    R v = r_zero<R>();
    if (c < T + 2 * P && c1 >= 0 && c1 < n1 && c2 >= 0 && c2 < n2 && c3 >= 0 && c3 < n3)
      v = xg ? r_from_out<R>(xg[c1 + (long long)n1 * (c2 + (long long)n2 * c3)]) : r_from_double<R>(1.0);
    sX[t] = v;
  }
}

// The work of one CTA: chunk `bid` of the launch's line list (line
// bid / nch, chunk bid % nch), in the dynamic shared memory `smem_raw`
// (RowsLayout::BYTES).  Called by rows_kernel with bid = blockIdx.x and by
// the persistent batch kernel once per work item.
template <int P, int D, int LM, int TMAX, bool DO_M, bool DO_K, typename R, bool APPLY = false>
__device__ __forceinline__ void rows_block(const RowsArgs &A, const int bid, unsigned char *smem_raw) {
  using L = RowsLayout<P, D, LM, TMAX, DO_M, DO_K, R, APPLY>;
  using O = typename OutT<R>::type;
  static_assert(sizeof(O) == sizeof(R), "the band stage shares the R region");
  constexpr int NP = L::NP, NB = L::NB, NT = L::NT, NW = L::NW, LS = L::LS, NL = L::NL, NL1 = L::NL1;

  R *sV23 = reinterpret_cast<R *>(smem_raw);  // [di][kind][LM][NP]
  R *sV23d = sV23 + L::V23;                   // [di][kind][LM][NB] (boundary lines)
  R *sB23 = sV23d + L::V23D;                  // [di][kind][LM][4]
  R *sV1 = sB23 + L::B23;                     // 2 x MAXPTS1 x NP (x1_idx)
  R *sB1 = sV1 + L::V1;                       // 2 x MAXPTS1 x 4 (x1_idx)
  R *sCb = sB1 + L::B1;                       // [l3][l2][l1]
  R *sU = sCb + L::CB;                        // [u][NL1][LS]
  R *sW = sU + L::US;                         // phase A: [warp][WS]; phase B: the row stage
  R *sX = sW + L::SCRATCH;                    // apply: x at the chunk's band columns
  int *sE23 = reinterpret_cast<int *>(smem_raw + sizeof(R) * (size_t)L::R_TOTAL);  // [di][LM]
  int *sO23 = sE23 + 2 * LM;                  // [di][LM]
  int *sE1 = sO23 + 2 * LM;                   // [MAXPTS1]
  int *sOff1 = sE1 + L::MAXPTS1;              // [TMAX+1]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int line = A.lines ? A.lines[bid / A.nch] : A.line0 + bid / A.nch;
  const int ch = bid % A.nch;
  const int n1 = A.n[0];
  const int r2 = (D == 3) ? line % A.n[1] : line;
  const int r3 = (D == 3) ? line / A.n[1] : 0;
  const long long base = (long long)line * n1;
  long long lo = (long long)ch * A.T, hi = lo + A.T;
  if (hi > n1) hi = n1;
  if (lo < A.row_begin - base) lo = A.row_begin - base;
  if (hi > A.row_end - base) hi = A.row_end - base;
  if (lo >= hi) return;
  const int a = (int)lo, b = (int)hi, T = b - a;

  // ------------------------------------------------ tables and the coefficient block
  const int rr[2] = {r2, r3};
  int L23[2] = {1, 1}, l23lo[2] = {0, 0}, nl23[2] = {1, 1};
#pragma unroll
  for (int di = 0; di < D - 1; di++) {
    const int dir = di + 1, r = rr[di];
    const int off0 = A.off[dir][0][r];
    const int off1 = A.off[dir][1][r];
    L23[di] = (LM == P + 1) ? P + 1 : A.off[dir][0][r + 1] - off0;
    const int elo = r - P < 0 ? 0 : r - P;
    const int ehi = r > A.N[dir] - 1 ? A.N[dir] - 1 : r;
    l23lo[di] = elo;
    nl23[di] = ehi - elo + 4;
    for (int t = tid; t < 2 * LM; t += NT) {
      const int kind = t / LM, q = t % LM;
      if (q < L23[di]) {
        const int gq = (kind ? off1 : off0) + q;
        const R *Vg = static_cast<const R *>(A.V[dir][kind]);
        const R *Bg = static_cast<const R *>(A.beta[dir][kind]);
#pragma unroll
        for (int i = 0; i < NP; i++) sV23[((di * 2 + kind) * LM + q) * NP + i] = Vg[(size_t)gq * NP + i];
#pragma unroll
        for (int i = 0; i < 4; i++) sB23[((di * 2 + kind) * LM + q) * 4 + i] = Bg[(size_t)gq * 4 + i];
        const int e = A.elem[dir][0][gq];
        if constexpr (!L::INNER_GAUSS) {
          const int o = e - r + P;
#pragma unroll
          for (int j = 0; j < NB; j++)
            sV23d[((di * 2 + kind) * LM + q) * NB + j] =
                (j >= o && j <= o + P) ? Vg[(size_t)gq * NP + (j - o)] : r_zero<R>();
        }
        if (kind == 0) {
          sE23[di * LM + q] = e;
          sO23[di * LM + q] = e - r + P;
        }
      }
    }
  }
  load_x1_tables<P, L::MAXPTS1, R>(A, a, T, sV1, sB1, sE1, sOff1);
  const int elo1 = a - P < 0 ? 0 : a - P;
  const int ehi1 = (b - 1) > A.N[0] - 1 ? A.N[0] - 1 : (b - 1);
  const int l1lo = elo1, nl1 = ehi1 - elo1 + 4;
  const int L2 = L23[0], L3 = L23[1];
  const int nl2 = nl23[0], nl3 = (D == 3) ? nl23[1] : 1;
  {
    unsigned bad = 0;
    const double *cg = A.coef;
    const R *cr = static_cast<const R *>(A.coefR);
    for (int t = tid; t < L::NL3 * NL * NL1; t += NT) {
      const int l1 = t % NL1, l2 = (t / NL1) % NL, l3 = t / (NL1 * NL);
      if (l1 < nl1 && l2 < nl2 && l3 < nl3) {
        const long long g = (long long)(l1lo + l1) +
                            (long long)A.nc[0] * ((long long)(l23lo[0] + l2) +
                                                  (long long)A.nc[1] * (D == 3 ? (long long)(l23lo[1] + l3) : 0LL));
        if (cr) {
          sCb[t] = cr[g];
        } else if (cg) {
          const double v = cg[g];
          if (!isfinite(v)) bad = 1;
          sCb[t] = r_from_double<R>(v);
        } else {
          sCb[t] = r_from_double<R>(1.0);
        }
      }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && lane == 0) atomicOr(A.status, 2u);
  }
  cp_async_wait_all();  // the x1 tables
  __syncthreads();

  // ------------------------------------------------ phase A: U, two coefficient columns per warp
  // (16 lanes each; a half-warp past the last column idles through the
  // same loop trip counts, so every __syncwarp is reached by all lanes)
  const int half = lane >> 4, hl = lane & 15;
  R *wx = sW + (2 * warp + half) * L::WS;  // Z, later Cq
  R *wt = wx + L::WX;                      // T3
  for (int l1b = 2 * warp; l1b < nl1; l1b += 2 * NW) {
    const int l1 = l1b + half;
    const bool act = l1 < nl1;
    if constexpr (D == 3) {
      // Z[k3][l2][q3] = sum_i Cb[e3(q3)+i][l2][l1] * b3[k3][q3][i]
      for (int t = hl; t < L::NK3 * NL * LM; t += 16) {
        const int q3 = t % LM, l2 = (t / LM) % NL, k3 = t / (LM * NL);
        if (act && q3 < L3 && l2 < nl2) {
          const int e = sE23[LM + q3] - l23lo[1];
          const R *bb = &sB23[((1 * 2 + k3) * LM + q3) * 4];
          R s = r_zero<R>();
#pragma unroll
          for (int i = 0; i < 4; i++) s = r_fma(sCb[((e + i) * NL + l2) * NL1 + l1], bb[i], s);
          wx[t] = s;
        }
      }
      __syncwarp();
      // T3[k3][l2][j3] = sum_q3 Z[k3][l2][q3] * V3[k3][q3][j3 - o3]
      for (int t = hl; t < L::NK3 * NL; t += 16) {
        const int l2 = t % NL, k3 = t / NL;
        if (act && l2 < nl2) {
          R acc[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) acc[j] = r_zero<R>();
          if constexpr (L::INNER_GAUSS) {
            fiber_at<P, 0>(acc, wx[t * LM + 0], &sV23[((1 * 2 + k3) * LM + 0) * NP]);
            fiber_at<P, 1>(acc, wx[t * LM + 1], &sV23[((1 * 2 + k3) * LM + 1) * NP]);
            fiber_at<P, 2>(acc, wx[t * LM + 2], &sV23[((1 * 2 + k3) * LM + 2) * NP]);
            if constexpr (P >= 3) fiber_at<P, (P >= 3 ? 3 : 0)>(acc, wx[t * LM + 3], &sV23[((1 * 2 + k3) * LM + 3) * NP]);
          } else {
            for (int q3 = 0; q3 < L3; q3++)
              fiber_point<P>(acc, wx[t * LM + q3], &sV23[((1 * 2 + k3) * LM + q3) * NP],
                             &sV23d[((1 * 2 + k3) * LM + q3) * NB], sO23[LM + q3]);
          }
#pragma unroll
          for (int j = 0; j < NB; j++) wt[t * NB + j] = acc[j];
        }
      }
      __syncwarp();
      // Cq[c][q2][j3] = sum_i T3[k3(c)][e2(q2)+i][j3] * b2[k2(c)][q2][i]; c = (kind2, kind3):
      // 0 = (M, M), 1 = (S, M), 2 = (M, S)
      for (int t = hl; t < L::NCOMBO * LM * NB; t += 16) {
        const int j3 = t % NB, q2 = (t / NB) % LM, c = t / (NB * LM);
        if (act && q2 < L2) {
          const int k2 = (c == 1) ? 1 : 0, k3 = (c == 2) ? 1 : 0;
          const int e = sE23[q2] - l23lo[0];
          const R *bb = &sB23[((0 * 2 + k2) * LM + q2) * 4];
          R s = r_zero<R>();
#pragma unroll
          for (int i = 0; i < 4; i++) s = r_fma(wt[(k3 * NL + e + i) * NB + j3], bb[i], s);
          wx[t] = s;
        }
      }
      __syncwarp();
      // U0[l1][j3*NB+j2] = sum_q2 Cq[MM][q2][j3] V2M[q2][j2-o2]
      // U1[l1][j3*NB+j2] = sum_q2 Cq[SM][q2][j3] V2S[q2][..] + Cq[MS][q2][j3] V2M[q2][..]
      for (int t = hl; t < L::NU * NB; t += 16) {
        if (!act) continue;
        const int j3 = t % NB, u = t / NB;
        R acc[NB];
#pragma unroll
        for (int j = 0; j < NB; j++) acc[j] = r_zero<R>();
        if constexpr (L::INNER_GAUSS) {
          if (u == 0) {
            fiber_at<P, 0>(acc, wx[(0 * LM + 0) * NB + j3], &sV23[(0 * LM + 0) * NP]);
            fiber_at<P, 1>(acc, wx[(0 * LM + 1) * NB + j3], &sV23[(0 * LM + 1) * NP]);
            fiber_at<P, 2>(acc, wx[(0 * LM + 2) * NB + j3], &sV23[(0 * LM + 2) * NP]);
            if constexpr (P >= 3) fiber_at<P, (P >= 3 ? 3 : 0)>(acc, wx[(0 * LM + 3) * NB + j3], &sV23[(0 * LM + 3) * NP]);
          } else {
#pragma unroll
            for (int c = 1; c <= 2; c++) {
              const int k = (c == 1) ? 1 : 0;  // kind of x2 in combination c
              fiber_at<P, 0>(acc, wx[(c * LM + 0) * NB + j3], &sV23[(k * LM + 0) * NP]);
              fiber_at<P, 1>(acc, wx[(c * LM + 1) * NB + j3], &sV23[(k * LM + 1) * NP]);
              fiber_at<P, 2>(acc, wx[(c * LM + 2) * NB + j3], &sV23[(k * LM + 2) * NP]);
              if constexpr (P >= 3) fiber_at<P, (P >= 3 ? 3 : 0)>(acc, wx[(c * LM + 3) * NB + j3], &sV23[(k * LM + 3) * NP]);
            }
          }
        } else {
          for (int q2 = 0; q2 < L2; q2++) {
            const int o = sO23[q2];
            const R *vM = &sV23[(0 * LM + q2) * NP], *vMd = &sV23d[(0 * LM + q2) * NB];
            if (u == 0) {
              fiber_point<P>(acc, wx[(0 * LM + q2) * NB + j3], vM, vMd, o);
            } else {
              fiber_point<P>(acc, wx[(1 * LM + q2) * NB + j3], &sV23[(1 * LM + q2) * NP],
                             &sV23d[(1 * LM + q2) * NB], o);
              fiber_point<P>(acc, wx[(2 * LM + q2) * NB + j3], vM, vMd, o);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < NB; j++) sU[(u * NL1 + l1) * LS + j3 * NB + j] = acc[j];
      }
    } else {
      // Cq[k2][q2] = sum_i Cb[e2(q2)+i][l1] * b2[k2][q2][i]
      for (int t = hl; t < L::NCOMBO * LM; t += 16) {
        const int q2 = t % LM, c = t / LM;
        if (act && q2 < L2) {
          const int e = sE23[q2] - l23lo[0];
          const R *bb = &sB23[((0 * 2 + c) * LM + q2) * 4];
          R s = r_zero<R>();
#pragma unroll
          for (int i = 0; i < 4; i++) s = r_fma(sCb[(e + i) * NL1 + l1], bb[i], s);
          wx[t] = s;
        }
      }
      __syncwarp();
      // U0[l1][j2] = sum_q2 Cq[M][q2] V2M[q2][..];  U1[l1][j2] = sum_q2 Cq[S][q2] V2S[q2][..]
      if (act && hl < L::NU) {
        const int u = hl;
        R acc[NB];
#pragma unroll
        for (int j = 0; j < NB; j++) acc[j] = r_zero<R>();
        if constexpr (L::INNER_GAUSS) {
          fiber_at<P, 0>(acc, wx[u * LM + 0], &sV23[(u * LM + 0) * NP]);
          fiber_at<P, 1>(acc, wx[u * LM + 1], &sV23[(u * LM + 1) * NP]);
          fiber_at<P, 2>(acc, wx[u * LM + 2], &sV23[(u * LM + 2) * NP]);
          if constexpr (P >= 3) fiber_at<P, (P >= 3 ? 3 : 0)>(acc, wx[u * LM + 3], &sV23[(u * LM + 3) * NP]);
        } else {
          for (int q2 = 0; q2 < L2; q2++)
            fiber_point<P>(acc, wx[u * LM + q2], &sV23[(u * LM + q2) * NP], &sV23d[(u * LM + q2) * NB], sO23[q2]);
        }
#pragma unroll
        for (int j = 0; j < NB; j++) sU[(u * NL1 + l1) * LS + j] = acc[j];
      }
    }
    __syncwarp();
  }
  if constexpr (APPLY) stage_x<P, D, TMAX + 2 * P>(A, line, a, T, sX);
  __syncthreads();

  rows_phase_b<P, D, L::MAXPTS1, NL1, L::GENERAL, DO_M, DO_K, R, APPLY>(A, sU, sV1, sB1, sE1, sOff1, sW, a, T, l1lo,
                                                                        base, sX);
}

template <int P, int D, int LM, int TMAX, bool DO_M, bool DO_K, typename R, bool APPLY = false>
__global__ void __launch_bounds__(32 * kRowsWarps, rows_min_blocks<R>()) rows_kernel(const RowsArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_block<P, D, LM, TMAX, DO_M, DO_K, R, APPLY>(A, blockIdx.x, smem_raw);
}

}  // namespace wq
