// Row-wise weighted-quadrature assembly kernel (sum factorisation into the
// band), templated on degree P, dimension D, point capacity of the inner
// directions LM, and the arithmetic type R (double, or float for the mixed
// mode).
//
// Work decomposition.  A CTA owns a chunk of consecutive rows along x1 that
// share (r2, r3) -- one "line" of rows.  Rows of a line share their rule
// points in directions 2..D, so the coefficient spline c is contracted over
// directions D..2 once per chunk (phase A), leaving c on the (q2, q3) point
// grid for every coefficient column l1.  Each warp then takes one row at a
// time (phase B) and streams over blocks of P+1 points of direction 1 (an
// interior row is one block, a boundary row one block per element):
//   C1: c at the block's points of each grid, from the phase-A columns
//   X : contraction over q3 into the band index j3   (D = 3)
//   Y : contraction over q2 into j2
//   F : contraction over q1 into j1, accumulated in registers
// The grids are the point sets of the terms (Sec. 3.1 rule in every
// direction for M; Sec. 3.2 rule in direction a and Sec. 3.1 elsewhere for
// term a of K).  The folded 1D tables already hold W * |J_aa| (mass kind) or
// W / |J_aa| (stiffness kind), so c is the only per-point factor.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace wq {

struct RowsArgs {
  const int *off[3][2];
  const int *elem[3][2];
  const void *V[3][2];     // folded tables, R, npts*(P+1)
  const void *beta[3][2];  // cubic coefficient-spline values, R, npts*4
  int n[3], N[3], nc[3];
  const double *coef;  // may be null: c = 1
  void *M, *K;         // R band outputs
  long long row_begin, row_end;
  const int *lines;  // line ids of this launch
  int nch, T;        // chunks per line and chunk length
  unsigned *status;
};

// acc[o + i] += x * v[i], i = 0..P, with a compile-time register index in
// each case (o is uniform across the warp by construction).
template <int P, int O, typename R>
__device__ __forceinline__ void fiber_at(R (&acc)[2 * P + 1], R x, const R *__restrict__ v) {
#pragma unroll
  for (int i = 0; i <= P; i++) acc[O + i] = fma(x, v[i], acc[O + i]);
}

template <int P, typename R>
__device__ __forceinline__ void fiber_add(R (&acc)[2 * P + 1], R x, const R *__restrict__ v, int o) {
  switch (o) {
    case 0: fiber_at<P, 0>(acc, x, v); break;
    case 1: fiber_at<P, 1>(acc, x, v); break;
    case 2: fiber_at<P, 2>(acc, x, v); break;
    default:
      if constexpr (P >= 3) fiber_at<P, (P >= 3 ? 3 : 0)>(acc, x, v);
      break;
  }
}

template <int P, int D, int LM, int NW, int TMAX, bool DO_M, bool DO_K, typename R>
struct RowsLayout {
  static constexpr int NP = P + 1;             // points per direction-1 block
  static constexpr int NB = 2 * P + 1;         // band width per direction
  static constexpr int NG = (DO_M ? 1 : 0) + (DO_K ? D : 0);  // point grids
  static constexpr int NCOMBO = DO_K ? D : 1;  // (kind2, kind3) combinations of the phase-A columns
  static constexpr int NK3 = (D == 3) ? (DO_K ? 2 : 1) : 0;
  static constexpr int NL1 = TMAX + P + 3;     // coefficient columns of a chunk
  static constexpr int NL = P + 4;             // coefficient indices of one row per direction
  static constexpr int LM2 = (D == 3) ? LM * LM : LM;
  // R region
  static constexpr int P23V = 2 * 2 * LM * NP;  // [dir2/3][kind][q][i]
  static constexpr int P23B = 2 * 2 * LM * 4;
  static constexpr int CQ = NCOMBO * NL1 * LM2;
  static constexpr int CB = (D == 3 ? NL * NL : NL) * NL1;
  static constexpr int ZS = (D == 3) ? NK3 * NL1 * NL * LM : 0;
  static constexpr int PHASE_A = CB + ZS;
  static constexpr int BUFA = (D == 3) ? NG * NP * (LM * LM > NB * NB ? LM * LM : NB * NB) : NG * NP * LM;
  static constexpr int BUFB = (D == 3) ? NG * NP * LM * NB : NG * NP * NB;
  static constexpr int BLK = 2 * NP * NP + 2 * NP * 4;
  static constexpr int WARP = BLK + BUFA + BUFB;
  static constexpr int UNION = (PHASE_A > NW * WARP) ? PHASE_A : NW * WARP;
  static constexpr int R_TOTAL = P23V + P23B + CQ + UNION;
  // int region
  static constexpr int I_P23 = 2 * 2 * LM;  // elem, o per (dir2/3, q)
  static constexpr int I_WARP = 2 * NP;     // elem, o per block point
  static constexpr int I_TOTAL = I_P23 + NW * I_WARP;
  static constexpr size_t BYTES = sizeof(R) * (size_t)R_TOTAL + sizeof(int) * (size_t)I_TOTAL;
};

template <int P, int D, int LM, int NW, int TMAX, bool DO_M, bool DO_K, typename R>
__global__ void __launch_bounds__(NW * 32) rows_kernel(const RowsArgs A) {
  using L = RowsLayout<P, D, LM, NW, TMAX, DO_M, DO_K, R>;
  constexpr int NP = L::NP, NB = L::NB, NG = L::NG;
  constexpr int G_M = 0;
  constexpr int G_K1 = DO_M ? 1 : 0, G_K2 = G_K1 + 1, G_K3 = G_K1 + 2;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sR = reinterpret_cast<R *>(smem_raw);
  int *sI = reinterpret_cast<int *>(smem_raw + sizeof(R) * (size_t)L::R_TOTAL);
  R *sV23 = sR;                          // [di][kind][LM][NP]
  R *sB23 = sV23 + L::P23V;              // [di][kind][LM][4]
  R *sCq = sB23 + L::P23B;               // [combo][NL1][LM2]
  R *sU = sCq + L::CQ;                   // union
  int *sE23 = sI;                        // [di][LM]
  int *sO23 = sI + 2 * LM;               // [di][LM]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int line = A.lines[blockIdx.x / A.nch];
  const int ch = blockIdx.x % A.nch;
  const int n1 = A.n[0];
  const int r2 = (D == 3) ? line % A.n[1] : line;
  const int r3 = (D == 3) ? line / A.n[1] : 0;
  const long long base = (long long)line * n1;
  long long lo = (long long)ch * A.T, hi = lo + A.T;
  if (hi > n1) hi = n1;
  if (lo < A.row_begin - base) lo = A.row_begin - base;
  if (hi > A.row_end - base) hi = A.row_end - base;
  if (lo >= hi) return;
  const int a = (int)lo, b = (int)hi;

  // ---------------------------------------------------------------- phase A
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
    for (int t = tid; t < 2 * L23[di]; t += NW * 32) {
      const int kind = t / L23[di], q = t % L23[di];
      const int gq = (kind ? off1 : off0) + q;
      const R *Vg = static_cast<const R *>(A.V[dir][kind]);
      const R *Bg = static_cast<const R *>(A.beta[dir][kind]);
#pragma unroll
      for (int i = 0; i < NP; i++) sV23[((di * 2 + kind) * LM + q) * NP + i] = Vg[(size_t)gq * NP + i];
#pragma unroll
      for (int i = 0; i < 4; i++) sB23[((di * 2 + kind) * LM + q) * 4 + i] = Bg[(size_t)gq * 4 + i];
      if (kind == 0) {
        const int e = A.elem[dir][0][gq];
        sE23[di * LM + q] = e;
        sO23[di * LM + q] = e - r + P;
      }
    }
  }
  const int elo1 = a - P < 0 ? 0 : a - P;
  const int ehi1 = (b - 1) > A.N[0] - 1 ? A.N[0] - 1 : (b - 1);
  const int l1lo = elo1, nl1 = ehi1 - elo1 + 4;
  const int L2 = L23[0], L3 = L23[1];
  const int nl2 = nl23[0], nl3 = (D == 3) ? nl23[1] : 1;
  R *sCb = sU;             // [l3'][l2'][l1'] (runtime strides nl2, nl1)
  R *sZ = sU + L::CB;      // [k3][NL1][NL][LM]
  {
    unsigned bad = 0;
    const int tot = nl3 * nl2 * nl1;
    for (int t = tid; t < tot; t += NW * 32) {
      const int l1 = t % nl1, l2 = (t / nl1) % nl2, l3 = t / (nl1 * nl2);
      double v = 1.0;
      if (A.coef) {
        const long long g = (long long)(l1lo + l1) +
                            (long long)A.nc[0] * ((long long)(l23lo[0] + l2) + (long long)A.nc[1] * (D == 3 ? (long long)(l23lo[1] + l3) : 0LL));
        v = A.coef[g];
        if (!isfinite(v)) bad = 1;
      }
      sCb[t] = (R)v;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && lane == 0) atomicOr(A.status, 2u);
  }
  __syncthreads();
  if constexpr (D == 3) {
    // Z[k3][l1][l2][q3] = sum_i Cb[e3(q3)+i-l3lo][l2][l1] * beta3[k3][q3][i]
    const int tot = L::NK3 * nl1 * nl2 * L3;
    for (int t = tid; t < tot; t += NW * 32) {
      const int q3 = t % L3, l2 = (t / L3) % nl2, l1 = (t / (L3 * nl2)) % nl1, k3 = t / (L3 * nl2 * nl1);
      const int e = sE23[LM + q3] - l23lo[1];
      const R *bb = &sB23[((1 * 2 + k3) * LM + q3) * 4];
      R s = 0;
#pragma unroll
      for (int i = 0; i < 4; i++) s = fma(sCb[((e + i) * nl2 + l2) * nl1 + l1], bb[i], s);
      sZ[((k3 * L::NL1 + l1) * L::NL + l2) * LM + q3] = s;
    }
    __syncthreads();
    // Cq[c][l1][q2][q3]; combos: 0 = (M, M), 1 = (S, M), 2 = (M, S)
    const int tot2 = L::NCOMBO * nl1 * L2 * L3;
    for (int t = tid; t < tot2; t += NW * 32) {
      const int q3 = t % L3, q2 = (t / L3) % L2, l1 = (t / (L3 * L2)) % nl1, c = t / (L3 * L2 * nl1);
      const int k2 = (c == 1) ? 1 : 0, k3 = (c == 2) ? 1 : 0;
      const int e = sE23[q2] - l23lo[0];
      const R *bb = &sB23[((0 * 2 + k2) * LM + q2) * 4];
      R s = 0;
#pragma unroll
      for (int i = 0; i < 4; i++) s = fma(sZ[((k3 * L::NL1 + l1) * L::NL + e + i) * LM + q3], bb[i], s);
      sCq[(c * L::NL1 + l1) * L::LM2 + q2 * LM + q3] = s;
    }
  } else {
    // Cq[k2][l1][q2] = sum_i Cb[e2(q2)+i-l2lo][l1] * beta2[k2][q2][i]
    const int tot2 = L::NCOMBO * nl1 * L2;
    for (int t = tid; t < tot2; t += NW * 32) {
      const int q2 = t % L2, l1 = (t / L2) % nl1, c = t / (L2 * nl1);
      const int e = sE23[q2] - l23lo[0];
      const R *bb = &sB23[((0 * 2 + c) * LM + q2) * 4];
      R s = 0;
#pragma unroll
      for (int i = 0; i < 4; i++) s = fma(sCb[(e + i) * nl1 + l1], bb[i], s);
      sCq[(c * L::NL1 + l1) * L::LM2 + q2] = s;
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- phase B
  R *wR = sU + warp * L::WARP;
  R *blkV = wR;                   // [kind][NP][NP]
  R *blkB = blkV + 2 * NP * NP;   // [kind][NP][4]
  R *bufA = blkB + 2 * NP * 4;
  R *bufB = bufA + L::BUFA;
  int *blkE = sI + L::I_P23 + warp * L::I_WARP;
  int *blkO = blkE + NP;

  const R *V1[2] = {static_cast<const R *>(A.V[0][0]), static_cast<const R *>(A.V[0][1])};
  const R *B1[2] = {static_cast<const R *>(A.beta[0][0]), static_cast<const R *>(A.beta[0][1])};
  constexpr int NPAIR = (D == 3) ? NB * NB : NB;
  constexpr int NSLOT = (NPAIR + 31) / 32;

  for (int r1 = a + warp; r1 < b; r1 += NW) {
    const int offM = A.off[0][0][r1], offS = A.off[0][1][r1];
    const int nblk = (A.off[0][0][r1 + 1] - offM) / NP;
    R accM[NSLOT][NB], accK[NSLOT][NB];
#pragma unroll
    for (int s = 0; s < NSLOT; s++)
#pragma unroll
      for (int j = 0; j < NB; j++) { accM[s][j] = 0; accK[s][j] = 0; }

    for (int blk = 0; blk < nblk; blk++) {
      __syncwarp();
      for (int t = lane; t < 2 * NP; t += 32) {
        const int kind = t / NP, qb = t % NP;
        const int gq = (kind ? offS : offM) + blk * NP + qb;
#pragma unroll
        for (int i = 0; i < NP; i++) blkV[(kind * NP + qb) * NP + i] = V1[kind][(size_t)gq * NP + i];
#pragma unroll
        for (int i = 0; i < 4; i++) blkB[(kind * NP + qb) * 4 + i] = B1[kind][(size_t)gq * 4 + i];
        if (kind == 0) {
          const int e = A.elem[0][0][gq];
          blkE[qb] = e - l1lo;
          blkO[qb] = e - r1 + P;
        }
      }
      __syncwarp();
      if constexpr (D == 3) {
        // C1: c[g][qb][q2][q3]
        const int totc = NG * NP * L2 * L3;
        for (int t = lane; t < totc; t += 32) {
          const int q3 = t % L3, q2 = (t / L3) % L2, qb = (t / (L3 * L2)) % NP, g = t / (L3 * L2 * NP);
          const int combo = (DO_K && g == G_K2) ? 1 : ((DO_K && g == G_K3) ? 2 : 0);
          const int k1 = (DO_K && g == G_K1) ? 1 : 0;
          const R *cq = &sCq[(combo * L::NL1 + blkE[qb]) * L::LM2 + q2 * LM + q3];
          const R *bb = &blkB[(k1 * NP + qb) * 4];
          R s = 0;
#pragma unroll
          for (int i = 0; i < 4; i++) s = fma(cq[i * L::LM2], bb[i], s);
          bufA[((g * NP + qb) * LM + q2) * LM + q3] = s;
        }
        __syncwarp();
        // X: contraction over q3 -> j3
        const int totx = NG * NP * L2;
        for (int t = lane; t < totx; t += 32) {
          const int q2 = t % L2, qb = (t / L2) % NP, g = t / (L2 * NP);
          const int k3 = (DO_K && g == G_K3) ? 1 : 0;
          R acc[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) acc[j] = 0;
          const R *cin = &bufA[((g * NP + qb) * LM + q2) * LM];
          for (int q3 = 0; q3 < L3; q3++)
            fiber_add<P>(acc, cin[q3], &sV23[((1 * 2 + k3) * LM + q3) * NP], sO23[LM + q3]);
          R *xo = &bufB[((g * NP + qb) * LM + q2) * NB];
#pragma unroll
          for (int j = 0; j < NB; j++) xo[j] = acc[j];
        }
        __syncwarp();
        // Y: contraction over q2 -> j2; output pair index j3*NB + j2
        const int toty = NG * NP * NB;
        for (int t = lane; t < toty; t += 32) {
          const int j3 = t % NB, qb = (t / NB) % NP, g = t / (NB * NP);
          const int k2 = (DO_K && g == G_K2) ? 1 : 0;
          R acc[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) acc[j] = 0;
          const R *xin = &bufB[((g * NP + qb) * LM) * NB + j3];
          for (int q2 = 0; q2 < L2; q2++)
            fiber_add<P>(acc, xin[q2 * NB], &sV23[((0 * 2 + k2) * LM + q2) * NP], sO23[q2]);
          R *yo = &bufA[(g * NP + qb) * NB * NB + j3 * NB];
#pragma unroll
          for (int j = 0; j < NB; j++) yo[j] = acc[j];
        }
      } else {
        // C1: c[g][qb][q2]
        const int totc = NG * NP * L2;
        for (int t = lane; t < totc; t += 32) {
          const int q2 = t % L2, qb = (t / L2) % NP, g = t / (L2 * NP);
          const int k2 = (DO_K && g == G_K2) ? 1 : 0;
          const int k1 = (DO_K && g == G_K1) ? 1 : 0;
          const R *cq = &sCq[(k2 * L::NL1 + blkE[qb]) * L::LM2 + q2];
          const R *bb = &blkB[(k1 * NP + qb) * 4];
          R s = 0;
#pragma unroll
          for (int i = 0; i < 4; i++) s = fma(cq[i * L::LM2], bb[i], s);
          bufA[(g * NP + qb) * LM + q2] = s;
        }
        __syncwarp();
        // Y: contraction over q2 -> j2
        const int toty = NG * NP;
        for (int t = lane; t < toty; t += 32) {
          const int qb = t % NP, g = t / NP;
          const int k2 = (DO_K && g == G_K2) ? 1 : 0;
          R acc[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) acc[j] = 0;
          const R *cin = &bufA[(g * NP + qb) * LM];
          for (int q2 = 0; q2 < L2; q2++)
            fiber_add<P>(acc, cin[q2], &sV23[((0 * 2 + k2) * LM + q2) * NP], sO23[q2]);
          R *yo = &bufB[(g * NP + qb) * NB];
#pragma unroll
          for (int j = 0; j < NB; j++) yo[j] = acc[j];
        }
      }
      __syncwarp();
      // F: contraction over q1 -> j1, accumulated per owned pair
      const R *Y = (D == 3) ? bufA : bufB;
      constexpr int YS = (D == 3) ? NB * NB : NB;  // stride of one (g, qb) slice
#pragma unroll
      for (int s = 0; s < NSLOT; s++) {
        const int pr = lane + 32 * s;
        if (pr < NPAIR) {
#pragma unroll
          for (int qb = 0; qb < NP; qb++) {
            const int o = blkO[qb];
            const R *vM = &blkV[(0 * NP + qb) * NP];
            if constexpr (DO_M) fiber_add<P>(accM[s], Y[(G_M * NP + qb) * YS + pr], vM, o);
            if constexpr (DO_K) {
              R y = Y[(G_K2 * NP + qb) * YS + pr];
              if constexpr (D == 3) y += Y[(G_K3 * NP + qb) * YS + pr];
              fiber_add<P>(accK[s], y, vM, o);
              fiber_add<P>(accK[s], Y[(G_K1 * NP + qb) * YS + pr], &blkV[(1 * NP + qb) * NP], o);
            }
          }
        }
      }
    }
    // write the row's band: entry pair*NB + j1
    const long long orow = base + r1 - A.row_begin;
    constexpr int BAND = (D == 3) ? NB * NB * NB : NB * NB;
#pragma unroll
    for (int s = 0; s < NSLOT; s++) {
      const int pr = lane + 32 * s;
      if (pr < NPAIR) {
        if constexpr (DO_M) {
          R *out = static_cast<R *>(A.M) + orow * BAND + pr * NB;
#pragma unroll
          for (int j = 0; j < NB; j++) out[j] = accM[s][j];
        }
        if constexpr (DO_K) {
          R *out = static_cast<R *>(A.K) + orow * BAND + pr * NB;
#pragma unroll
          for (int j = 0; j < NB; j++) out[j] = accK[s][j];
        }
      }
    }
  }
}

}  // namespace wq
