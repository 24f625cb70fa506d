// 3D adjoint, second stage: the x2 and x3 stages transposed, once per block
// of kAULines lines of one x3 plane and kAUCols coefficient columns l1 (the
// forward u_kernel's blocking, run backwards).
//
// Input: Ubar in the chunk slots written by adjoint_x1_kernel; a line's Ubar
// at column l1 is the sum, in chunk order, of the slots whose window holds
// l1.  Per line r2 and item (l1, j3), with o = e2(q2) - r2 + P and
// d = e2(q2) - l2lo(r2):
//   c0[q2] = sum_i Ubar0[j3][o+i] V2M[q2][i]    (transpose of U0 += Cq_MM V2M)
//   c1[q2] = sum_i Ubar1[j3][o+i] V2S[q2][i]    (U1 += Cq_SM V2S)
//   c2[q2] = sum_i Ubar1[j3][o+i] V2M[q2][i]    (U1 += Cq_MS V2M)
//   T3bar_M[d+i][j3] += c0[q2] b2M[q2][i] + c1[q2] b2S[q2][i],
//   T3bar_S[d+i][j3] += c2[q2] b2M[q2][i]        (transpose of Cq = T3 x2 b2)
// The block's lines are summed per coefficient row l2 in line order, then
// per (k3, l1, l2), with o3 = e3(q3) - r3 + P and d3 = e3(q3) - l3lo:
//   z[q3] = sum_i T3bar_k3[l2][o3+i] V3_k3[q3][i],
//   Cbar[l1][l2][d3+i] += z[q3] b3_k3[q3][i]     (transpose of the x3 stage)
// summed over k3 = M, S.  The block's Cbar ([l1][l2 - l2lo][l3 - l3lo],
// double) goes to its own slot; adjoint_gather3_kernel adds the slots that
// hold each coefficient in a fixed order.
#pragma once

#include "assemble.cuh"

namespace wq {

constexpr int kAULines = 8, kAUCols = 4;

struct AdjUArgs {
  const int *off[3][2];
  const int *elem[3][2];
  const void *V[3][2];
  const void *beta[3][2];
  int n[3], N[3], nc[3];
  const void *ubar;       // chunk slots of Ubar in R (adjoint_x1_kernel)
  long long ubar_slot;    // values per slot
  int nch_max, nl1max;    // slots per line; the column extent of a slot
  int T_int, T_bnd;       // chunk lengths of interior and boundary lines
  long long row_begin, row_end;
  int line_lo, line_hi;   // lines of the call
  int r3_lo;              // plane of the launch's first CTA
  int nblk2, nblk1;       // line blocks per plane, column blocks
  double *cbar;           // one slot of CBAR values per CTA
  unsigned *status;
};

template <int P, typename R> struct AdjULayout {
  static constexpr int NP = P + 1, NB = 2 * P + 1, NPAIR = NB * NB;
  static constexpr int LM = P * (P + 1);             // most points of one row in one direction
  static constexpr int NL = P + 4;                   // coefficient rows of one row's support
  static constexpr int NL2 = kAULines + P + 3;       // x2 coefficient rows of a line block
  static constexpr int CBAR = kAUCols * NL2 * NL;    // doubles per block
  static constexpr int V3 = pad16<R>(2 * LM * NP);
  static constexpr int B3 = pad16<R>(2 * LM * 4);
  static constexpr int V2 = pad16<R>(kAULines * 2 * LM * NP);
  static constexpr int B2 = pad16<R>(kAULines * 2 * LM * 4);
  // per line: Ubar [u][l1][pair], then (same place) T3bar [k3][l1][l2 - l2lo(r2)][j3]
  static constexpr int UWA = 2 * kAUCols * NPAIR, UWB = 2 * kAUCols * NL * NB;
  static constexpr int UW = pad16<R>(UWA > UWB ? UWA : UWB);
  static constexpr int UB = kAULines * UW;
  static constexpr int TB = pad16<R>(2 * kAUCols * NL2 * NB);  // the lines' sum [k3][l1][l2][j3]
  static constexpr int CK = pad16<R>(2 * CBAR);                 // [k3][l1][l2][l3]
  static constexpr int R_TOTAL = V3 + B3 + V2 + B2 + UB + TB + CK;
  // int region: e3[LM], L2[kAULines], ok[kAULines], e2[kAULines][LM], db[kAULines]
  static constexpr int I_TOTAL = LM + 2 * kAULines + kAULines * LM + kAULines;
  // the Ubar sources of each (line, column): up to two slot offsets, -1 for none
  static constexpr int SRC = kAULines * kAUCols * 2;
  static constexpr size_t BYTES =
      sizeof(R) * (size_t)R_TOTAL + sizeof(long long) * (size_t)SRC + sizeof(int) * (size_t)I_TOTAL;
};

// c = sum_i u[O + i] v[i], i = 0..P.
template <int P, int O, int N, typename R>
__device__ __forceinline__ R adj_dot_at(const R (&u)[N], const R *v) {
  R c = r_zero<R>();
#pragma unroll
  for (int i = 0; i <= P; i++) c = r_fma(u[O + i], v[i], c);
  return c;
}
// The same for a runtime offset o in [0, P] (compile-time register indices).
template <int P, int N, typename R>
__device__ __forceinline__ R adj_dot(const R (&u)[N], const R *v, int o) {
  switch (o) {
    case 0: return adj_dot_at<P, 0>(u, v);
    case 1: return adj_dot_at<P, 1>(u, v);
    case 2: return adj_dot_at<P, 2>(u, v);
    default:
      if constexpr (P >= 3) return adj_dot_at<P, (P >= 3 ? 3 : 0)>(u, v);
      return r_zero<R>();
  }
}
// acc[D + i] += x b[i] (+ y c[i]), i = 0..3.
template <int D, int N, typename R>
__device__ __forceinline__ void adj_spread_at(R (&acc)[N], R x, const R *b, R y, const R *c, bool two) {
#pragma unroll
  for (int i = 0; i < 4; i++) {
    R t = r_fma(x, b[i], acc[D + i]);
    if (two) t = r_fma(y, c[i], t);
    acc[D + i] = t;
  }
}
// The same for a runtime offset d in [0, P].
template <int P, int N, typename R>
__device__ __forceinline__ void adj_spread(R (&acc)[N], R x, const R *b, R y, const R *c, bool two, int d) {
  switch (d) {
    case 0: adj_spread_at<0>(acc, x, b, y, c, two); break;
    case 1: adj_spread_at<1>(acc, x, b, y, c, two); break;
    case 2: adj_spread_at<2>(acc, x, b, y, c, two); break;
    default:
      if constexpr (P >= 3) adj_spread_at<(P >= 3 ? 3 : 0)>(acc, x, b, y, c, two);
      break;
  }
}

// Resident CTAs per SM the register allocation is sized for (four for
// float, three for double and double-float).
#ifndef WQ_ADJU_MIN_BLOCKS
#define WQ_ADJU_MIN_BLOCKS 3
#endif
#ifndef WQ_ADJU_MIN_BLOCKS_F32
#define WQ_ADJU_MIN_BLOCKS_F32 4
#endif
template <typename R> constexpr int adju_min_blocks() {
  return sizeof(R) == 4 ? WQ_ADJU_MIN_BLOCKS_F32 : WQ_ADJU_MIN_BLOCKS;
}
template <int P, typename R>
__global__ void __launch_bounds__(256, adju_min_blocks<R>()) adjoint_u_kernel(const AdjUArgs A) {
  using L = AdjULayout<P, R>;
  constexpr int NP = L::NP, NB = L::NB, NPAIR = L::NPAIR, LM = L::LM, NL = L::NL, NL2 = L::NL2;
  constexpr int NT = 256;
  static_assert(kAULines * 32 == NT, "one warp per line of the block");
  static_assert(kAUCols * NB <= 32, "one item per lane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sV3 = reinterpret_cast<R *>(smem_raw);
  R *sB3 = sV3 + L::V3;
  R *sV2 = sB3 + L::B3;
  R *sB2 = sV2 + L::V2;
  R *sUw = sB2 + L::B2;
  R *sTb = sUw + L::UB;
  R *sCk = sTb + L::TB;
  long long *sSrc = reinterpret_cast<long long *>(smem_raw + sizeof(R) * (size_t)L::R_TOTAL);
  int *sE3 = reinterpret_cast<int *>(sSrc + L::SRC);
  int *sL2 = sE3 + LM;
  int *sOk = sL2 + kAULines;
  int *sE2 = sOk + kAULines;
  int *sDb = sE2 + kAULines * LM;  // a line's first coefficient row minus the block's; large: no line

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n1 = A.n[0], n2 = A.n[1], N1 = A.N[0], nc1 = A.nc[0];
  int bid = blockIdx.x;
  const int b1 = bid % A.nblk1;
  bid /= A.nblk1;
  const int b2 = bid % A.nblk2;
  const int r3 = A.r3_lo + bid / A.nblk2;
  const int r2a = b2 * kAULines;
  const int nlines = (n2 - r2a) < kAULines ? (n2 - r2a) : kAULines;
  const int lid0 = r2a + n2 * r3;
  const int l1a = b1 * kAUCols;
  const int ncols = (nc1 - l1a) < kAUCols ? (nc1 - l1a) : kAUCols;
  const bool in3 = r3 >= P && r3 <= A.N[2] - 1;
  const int l2lo = (r2a - P) > 0 ? (r2a - P) : 0;
  const int l3lo = (r3 - P) > 0 ? (r3 - P) : 0;

  // ------------------------------------------------ tables
  const int off30 = A.off[2][0][r3], off31 = A.off[2][1][r3];
  const int L3 = A.off[2][0][r3 + 1] - off30;
#pragma unroll
  for (int kind = 0; kind < 2; kind++) {
    const int o = kind ? off31 : off30;
    cp_async_n(&sV3[kind * LM * NP], static_cast<const R *>(A.V[2][kind]) + (size_t)o * NP, L3 * NP, tid, NT);
    cp_async_n(&sB3[kind * LM * 4], static_cast<const R *>(A.beta[2][kind]) + (size_t)o * 4, L3 * 4, tid, NT);
  }
  cp_async_n(sE3, A.elem[2][0] + off30, L3, tid, NT);
  for (int t = tid; t < kAULines * 2 * LM; t += NT) {
    const int b = t / (2 * LM), kind = (t / LM) % 2, q = t % LM;
    if (b < nlines) {
      const int r2 = r2a + b;
      const int off0 = A.off[1][0][r2];
      const int L2b = A.off[1][0][r2 + 1] - off0;
      if (kind == 0 && q == 0) {
        sL2[b] = L2b;
        sOk[b] = (lid0 + b >= A.line_lo && lid0 + b <= A.line_hi) ? 1 : 0;
        sDb[b] = sOk[b] ? ((r2 - P) > 0 ? (r2 - P) : 0) - l2lo : (1 << 20);
      }
      if (q < L2b) {
        const int gq = (kind ? A.off[1][1][r2] : off0) + q;
        const R *Vg = static_cast<const R *>(A.V[1][kind]);
        const R *Bg = static_cast<const R *>(A.beta[1][kind]);
#pragma unroll
        for (int i = 0; i < NP; i++) cp_async_el(&sV2[((b * 2 + kind) * LM + q) * NP + i], &Vg[(size_t)gq * NP + i]);
#pragma unroll
        for (int i = 0; i < 4; i++) cp_async_el(&sB2[((b * 2 + kind) * LM + q) * 4 + i], &Bg[(size_t)gq * 4 + i]);
        if (kind == 0) cp_async_el(&sE2[b * LM + q], &A.elem[1][0][gq]);
      }
    } else if (kind == 0 && q == 0) {
      sL2[b] = 0;
      sOk[b] = 0;
      sDb[b] = 1 << 20;
    }
  }
  // the chunk slots whose window holds each (line, column), in chunk order,
  // as the offset of the column's u = 0 run (a column lies in at most two
  // windows when the chunk length is at least P + 3; more sets kBitInternal)
  if (tid < kAULines * kAUCols) {
    const int b = tid / kAUCols, l1 = tid % kAUCols;
    long long src0 = -1, src1 = -1;
    int ns = 0;
    const int r2 = r2a + b;
    const long long line = (long long)lid0 + b;
    if (b < nlines && l1 < ncols && line >= A.line_lo && line <= A.line_hi) {
      const int col = l1a + l1;
      const bool in2 = r2 >= P && r2 <= A.N[1] - 1;
      const int T = (in2 && in3) ? A.T_int : A.T_bnd;
      const int nch = (n1 + T - 1) / T;
      const long long base = line * n1;
      int chlo = (col - 2) / T - 1, chhi = (col + P) / T;
      if (chlo < 0) chlo = 0;
      if (chhi > nch - 1) chhi = nch - 1;
      for (int ch = chlo; ch <= chhi; ch++) {
        long long lo = (long long)ch * T, hi = lo + T;
        if (hi > n1) hi = n1;
        if (lo < A.row_begin - base) lo = A.row_begin - base;
        if (hi > A.row_end - base) hi = A.row_end - base;
        if (lo >= hi) continue;
        const int ca = (int)lo - P > 0 ? (int)lo - P : 0;
        const int cb = ((int)hi - 1 < N1 - 1 ? (int)hi - 1 : N1 - 1) + 3;
        if (col < ca || col > cb) continue;
        const long long off = (line * A.nch_max + ch) * A.ubar_slot + (long long)(col - ca) * NPAIR;
        if (ns == 0) src0 = off;
        else if (ns == 1) src1 = off;
        else atomicOr(A.status, kBitInternal);
        ns++;
      }
    }
    sSrc[tid * 2] = src0;
    sSrc[tid * 2 + 1] = src1;
  }
  __syncthreads();
  // Ubar of the block's lines at its columns: the sum of those slots' values;
  // a warp per (line, u, column) run of NPAIR values, lanes along the run
  {
    const R *Ug = static_cast<const R *>(A.ubar);
    const long long total = (long long)n2 * A.n[2] * A.nch_max * A.ubar_slot;
    const long long uoff = (long long)A.nl1max * NPAIR;
    for (int c = warp; c < kAULines * 2 * kAUCols; c += NT / 32) {
      const int b = c / (2 * kAUCols), u = (c / kAUCols) & 1, l1 = c % kAUCols;
      const long long sb0 = sSrc[(b * kAUCols + l1) * 2], sb1 = sSrc[(b * kAUCols + l1) * 2 + 1];
      const long long o0 = sb0 + u * uoff, o1 = sb1 + u * uoff;
      R *dst = sUw + b * L::UW + (u * kAUCols + l1) * NPAIR;
      for (int pr = lane; pr < NPAIR; pr += 32) {
        // the first source's value, plus the second's where the column has
        // two (no addition of a zero: the FP64 pipe is this kernel's bound)
        R v = r_zero<R>();
        if (sb0 >= 0 && check_range(A.status, o0 + pr, 1, total)) v = Ug[o0 + pr];
        if (sb1 >= 0 && check_range(A.status, o1 + pr, 1, total)) v = r_add(v, Ug[o1 + pr]);
        dst[pr] = v;
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // ------------------------------------------------ x2 stage transposed: warp = line, lane = (l1, j3)
  {
    const int b = warp, r2 = r2a + b;
    R *w = sUw + b * L::UW;
    const int l1 = lane / NB, j3 = lane - (lane / NB) * NB;
    const bool act = lane < kAUCols * NB && sOk[b] && l1 < ncols;
    R u0[NB], u1[NB];
#pragma unroll
    for (int j = 0; j < NB; j++) {
      u0[j] = act ? w[(0 * kAUCols + l1) * NPAIR + j3 * NB + j] : r_zero<R>();
      u1[j] = act ? w[(1 * kAUCols + l1) * NPAIR + j3 * NB + j] : r_zero<R>();
    }
    __syncwarp();  // the line's Ubar is read: its place takes T3bar
    R tm[NL], ts[NL];
#pragma unroll
    for (int j = 0; j < NL; j++) {
      tm[j] = r_zero<R>();
      ts[j] = r_zero<R>();
    }
    if (act) {
      const R *v2 = &sV2[(b * 2) * LM * NP];
      const R *bb2 = &sB2[(b * 2) * LM * 4];
      const int l2lo_r = (r2 - P) > 0 ? (r2 - P) : 0;
      const bool in2 = r2 >= P && r2 <= A.N[1] - 1;
      if (in2 && sE2[b * LM] == l2lo_r) {
        // interior line: point q2 in element r2 - P + q2, band offset q2
#pragma unroll
        for (int q2 = 0; q2 < NP; q2++) {
          const R *vm = &v2[(0 * LM + q2) * NP], *vs = &v2[(1 * LM + q2) * NP];
          const R *bm = &bb2[(0 * LM + q2) * 4], *bs = &bb2[(1 * LM + q2) * 4];
          R c0 = r_zero<R>(), c1 = r_zero<R>(), c2 = r_zero<R>();
#pragma unroll
          for (int i = 0; i < NP; i++) {
            c0 = r_fma(u0[q2 + i], vm[i], c0);
            c1 = r_fma(u1[q2 + i], vs[i], c1);
            c2 = r_fma(u1[q2 + i], vm[i], c2);
          }
#pragma unroll
          for (int i = 0; i < 4; i++) {
            tm[q2 + i] = r_fma(c1, bs[i], r_fma(c0, bm[i], tm[q2 + i]));
            ts[q2 + i] = r_fma(c2, bm[i], ts[q2 + i]);
          }
        }
      } else {
        const int L2 = sL2[b];
        for (int q2 = 0; q2 < L2; q2++) {
          const int e = sE2[b * LM + q2];
          const int o = e - r2 + P, d = e - l2lo_r;
          const R *vm = &v2[(0 * LM + q2) * NP], *vs = &v2[(1 * LM + q2) * NP];
          const R *bm = &bb2[(0 * LM + q2) * 4], *bs = &bb2[(1 * LM + q2) * 4];
          const R c0 = adj_dot<P>(u0, vm, o), c1 = adj_dot<P>(u1, vs, o), c2 = adj_dot<P>(u1, vm, o);
          adj_spread<P>(tm, c0, bm, c1, bs, true, d);
          adj_spread<P>(ts, c2, bm, c2, bm, false, d);
        }
      }
    }
    if (lane < kAUCols * NB) {
#pragma unroll
      for (int j = 0; j < NL; j++) {
        w[((0 * kAUCols + l1) * NL + j) * NB + j3] = tm[j];
        w[((1 * kAUCols + l1) * NL + j) * NB + j3] = ts[j];
      }
    }
  }
  __syncthreads();

  // ------------------------------------------------ the lines' sum (line order), items (k3, l1, l2, j3)
  for (int t = tid; t < 2 * kAUCols * NL2 * NB; t += NT) {
    const int j = t % NB, m = (t / NB) % NL2, l1 = (t / (NB * NL2)) % kAUCols, k3 = t / (NB * NL2 * kAUCols);
    R v = r_zero<R>();
    bool first = true;
    const R *src = sUw + (k3 * kAUCols + l1) * NL * NB + j;
    for (int b = 0; b < nlines; b++) {
      const int k = m - sDb[b];
      if ((unsigned)k < (unsigned)NL) {
        const R x = src[b * L::UW + k * NB];
        v = first ? x : r_add(v, x);
        first = false;
      }
    }
    sTb[t] = v;
  }
  __syncthreads();

  // ------------------------------------------------ x3 stage transposed, items (k3, l1, l2)
  for (int t = tid; t < 2 * kAUCols * NL2; t += NT) {
    const int m = t % NL2, l1 = (t / NL2) % kAUCols, k3 = t / (NL2 * kAUCols);
    R tb[NB];
#pragma unroll
    for (int j = 0; j < NB; j++) tb[j] = sTb[t * NB + j];
    R cb[NL];
#pragma unroll
    for (int j = 0; j < NL; j++) cb[j] = r_zero<R>();
    if (in3 && sE3[0] == l3lo) {
#pragma unroll
      for (int q3 = 0; q3 < NP; q3++) {
        const R *v = &sV3[(k3 * LM + q3) * NP];
        const R *bb = &sB3[(k3 * LM + q3) * 4];
        R z = r_zero<R>();
#pragma unroll
        for (int i = 0; i < NP; i++) z = r_fma(tb[q3 + i], v[i], z);
#pragma unroll
        for (int i = 0; i < 4; i++) cb[q3 + i] = r_fma(z, bb[i], cb[q3 + i]);
      }
    } else {
      for (int q3 = 0; q3 < L3; q3++) {
        const int e = sE3[q3];
        const R z = adj_dot<P>(tb, &sV3[(k3 * LM + q3) * NP], e - r3 + P);
        adj_spread<P>(cb, z, &sB3[(k3 * LM + q3) * 4], z, &sB3[(k3 * LM + q3) * 4], false, e - l3lo);
      }
    }
#pragma unroll
    for (int j = 0; j < NL; j++) sCk[((k3 * kAUCols + l1) * NL2 + m) * NL + j] = cb[j];
  }
  __syncthreads();
  const long long cslot = (long long)blockIdx.x * L::CBAR;
  const long long ctotal = (long long)gridDim.x * L::CBAR;
  for (int t = tid; t < L::CBAR; t += NT) {
    const R v = r_add(sCk[t], sCk[L::CBAR + t]);
    if (check_range(A.status, cslot + t, 1, ctotal)) A.cbar[cslot + t] = r_to_double(v);
  }
}

template <int P, typename R> cudaError_t launch_adjoint_u(const AdjUArgs &a, int nblocks, cudaStream_t s) {
  using L = AdjULayout<P, R>;
  auto kern = adjoint_u_kernel<P, R>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  kern<<<nblocks, 256, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wq
