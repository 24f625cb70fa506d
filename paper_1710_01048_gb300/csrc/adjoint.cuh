// Adjoint of the row-wise assembly: the gradient of
//   J(c) = sum_rows sum_band G .* K(c) + H .* M(c)
// with respect to the coefficients C of the cubic spline c.  Every band entry
// is linear in C, so dJ/dC = A^T applied to (G, H), where A is the forward
// map of the row kernels.  The forward map factors as
//   C --(x3 then x2 stages)--> U --(x1 stage, per row)--> bands,
// and the adjoint runs the transposed stages in reverse order:
//   1. x1 stage transposed, per chunk of a line's rows and band fibre:
//        yM[q] = sum_j1 H[j1] V1M[q][j1],  yK[q] = sum_j1 G[j1] V1M[q][j1],
//        yS[q] = sum_j1 G[j1] V1S[q][j1]
//      accumulated into Ubar0[l1] += b1M[q][l1] yM[q] + b1S[q][l1] yS[q] and
//      Ubar1[l1] += b1M[q][l1] yK[q]: each thread takes one fibre of four
//      consecutive rows and keeps its columns in registers, and the threads'
//      windows are added to Ubar in three ordered rounds (adj_x1_stage).
//   2. 2D (adjoint_kernel, in the same CTA): the x2 stage transposed, one warp
//      per coefficient column, giving the chunk's block of dJ/dC in its own
//      slot of a scratch array; adjoint_gather_kernel adds the blocks of the
//      chunks that touch each coefficient in a fixed order.
//      3D (adjoint_x1_kernel): the chunk's Ubar goes to its own slot;
//      adjoint_u_kernel (adjoint_u.cuh) runs the x2 and x3 stages transposed
//      once per block of lines and columns, adjoint_gather3_kernel adds the
//      blocks in a fixed order.
// No step depends on the order in which CTAs ran.
#pragma once

#include "assemble.cuh"

namespace wq {

struct AdjArgs {
  RowsArgs rows;         // tables, sizes, row range, line list, chunking (M, K, coef unused)
  const void *G, *H;     // band weights, OutT<R>, rows [row_begin, row_end); either may be null
  double *partial;       // 2D: chunk blocks, slot (line * nch_max + chunk) of blk values
  int nch_max, nl1max;   // slots per line; the l1 extent of a block
  long long blk;         // values per slot: NL * nl1max (2D)
  void *ubar;            // 3D: chunk slots of Ubar in R, slot (line * nch_max + chunk) of ubar_slot values
  long long ubar_slot;   // 2 * nl1max * (2P+1)^2: [u][column - the chunk's first column][(j3, j2)]
};

// The chunks of a line: its class's chunk length T (rows per chunk), clipped
// to the call's rows, as the adjoint (and forward) kernels cut them.
struct GatherArgs {
  const double *partial;  // 2D: chunk blocks; 3D: the line-block slots of adjoint_u_kernel
  double *grad;  // prod(nc_a) coefficients, overwritten
  int dim, p;
  int n[3], N[3], nc[3];
  long long row_begin, row_end;
  int T_int, T_bnd;  // chunk lengths of interior and boundary lines (2D)
  int nch_max, nl1max;
  long long blk;
  int r3_lo, r3_hi, nblk2, nblk1;  // 3D: planes of the call, line and column blocks per plane
};

template <int P, int D, int LM, int TMAX, typename R>
struct AdjLayout {
  using F = RowsLayout<P, D, LM, TMAX, true, true, R>;
  static constexpr int NP = P + 1, NB = 2 * P + 1;
  static constexpr int NPAIR = F::NPAIR, BAND = F::BAND;
  static constexpr int NL1 = F::NL1, NL = P + 4, NW = F::NW, NT = F::NT, MAXPTS1 = F::MAXPTS1;
  // per-warp scratch of phase 2 (the column work)
  static constexpr int WQ = (D == 3) ? 3 * LM * NB : 2 * LM;               // Cqbar
  static constexpr int WT = (D == 3) ? 2 * NL * NB : 0;                    // T3bar
  static constexpr int WZ = (D == 3) ? 2 * NL * LM : 0;                    // Zbar
  static constexpr int WS = pad16<R>(WQ + WT + WZ);
  static constexpr int V23 = F::V23, V23D = F::V23D, B23 = F::B23, V1 = F::V1, B1 = F::B1;
  static constexpr int UB = pad16<R>(2 * NL1 * NPAIR);                     // [u][l1][pair]
  static constexpr int R_TOTAL = V23 + V23D + B23 + V1 + B1 + UB + NW * WS;
  static constexpr int I_TOTAL = 4 * LM + MAXPTS1 + TMAX + 1;
  static constexpr size_t BYTES = sizeof(R) * (size_t)R_TOTAL + sizeof(int) * (size_t)I_TOTAL;
};

__device__ __forceinline__ double r_to_double(double a) { return a; }
__device__ __forceinline__ double r_to_double(float a) { return (double)a; }
__device__ __forceinline__ double r_to_double(dd a) { return dd_to_double(a); }

// One x1 point of the transposed x1 stage at band offset O for window row K
// (the point's columns are window columns K + O .. K + O + 3).
template <int P, int O, int K, int WN, typename R>
__device__ __forceinline__ void adj_x1_point(R (&w0)[WN], R (&w1)[WN], const R (&hv)[2 * P + 1],
                                             const R (&gv)[2 * P + 1], const R *vm, const R *vs, const R *bm,
                                             const R *bs) {
  R yM = r_zero<R>(), yK = r_zero<R>(), yS = r_zero<R>();
#pragma unroll
  for (int i = 0; i <= P; i++) {
    yM = r_fma(hv[O + i], vm[i], yM);
    yK = r_fma(gv[O + i], vm[i], yK);
    yS = r_fma(gv[O + i], vs[i], yS);
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    w0[K + O + i] = r_fma(bs[i], yS, r_fma(bm[i], yM, w0[K + O + i]));
    w1[K + O + i] = r_fma(bm[i], yK, w1[K + O + i]);
  }
}

// Row K of a segment starting at chunk row rl (x1 index a + rl + K): the
// fibre's H and G entries (grow: the fibre's first entry in row rl; a null
// weight is zero), then the row's points through a switch on the band offset.
template <int P, int K, int WN, int MAXPTS1, int BAND, typename R, typename O>
__device__ __forceinline__ void adj_x1_row(R (&w0)[WN], R (&w1)[WN], const int rl, const int T, const int a,
                                           const O *Hg, const O *Gg, const long long grow, const int *sOff1,
                                           const int *sE1, const R *sV1, const R *sB1) {
  constexpr int NP = P + 1, NB = 2 * P + 1;
  if (rl + K >= T) return;
  const long long g = grow + (long long)K * BAND;
  R hv[NB], gv[NB];
#pragma unroll
  for (int j = 0; j < NB; j++) {
    hv[j] = Hg ? r_from_out<R>(Hg[g + j]) : r_zero<R>();
    gv[j] = Gg ? r_from_out<R>(Gg[g + j]) : r_zero<R>();
  }
  const int q0 = sOff1[rl + K], q1e = sOff1[rl + K + 1];
  for (int q = q0; q < q1e; q++) {
    const int o = sE1[q] - (a + rl + K) + P;
    const R *vm = &sV1[(0 * MAXPTS1 + q) * NP], *vs = &sV1[(1 * MAXPTS1 + q) * NP];
    const R *bm = &sB1[(0 * MAXPTS1 + q) * 4], *bs = &sB1[(1 * MAXPTS1 + q) * 4];
    switch (o) {
      case 0: adj_x1_point<P, 0, K, WN>(w0, w1, hv, gv, vm, vs, bm, bs); break;
      case 1: adj_x1_point<P, 1, K, WN>(w0, w1, hv, gv, vm, vs, bm, bs); break;
      case 2: adj_x1_point<P, 2, K, WN>(w0, w1, hv, gv, vm, vs, bm, bs); break;
      default:
        if constexpr (P >= 3) adj_x1_point<P, (P >= 3 ? 3 : 0), K, WN>(w0, w1, hv, gv, vm, vs, bm, bs);
        break;
    }
  }
}

// The x1 stage transposed for the chunk of rows [a, a + T) of the line whose
// first row is `base` (D = 2 or 3: a row has (2P+1)^(D-1) band fibres of
// 2P+1 entries): Ubar (shared memory, [u][NL1][fibre], zeroed and
// visible to the CTA on entry) receives, for window columns 0 .. nl1-1 (column
// l1lo + c), the contributions of the chunk's rows and band fibres:
//   yM = sum_i H[o+i] V1M[q][i], yK = sum_i G[o+i] V1M[q][i], yS = sum_i G[o+i] V1S[q][i]
//   Ubar0[e+i] += b1M[q][i] yM + b1S[q][i] yS, Ubar1[e+i] += b1M[q][i] yK
// per row and x1 point q (element e, band offset o = e - r1 + P).  A thread
// takes one fibre of four consecutive rows and keeps its columns in a
// register window; the windows are added to Ubar in three ordered rounds
// (segments s, s+3, ... touch disjoint columns), so the result does not
// depend on thread timing.  Every thread of the CTA must call it; it ends
// with a barrier.
template <int P, int D, int MAXPTS1, int NL1, int NT, typename R>
__device__ __forceinline__ void adj_x1_stage(const AdjArgs &AA, const R *sV1, const R *sB1, const int *sE1,
                                             const int *sOff1, R *sUb, int a, int T, long long base, int l1lo,
                                             int nl1) {
  using O = typename OutT<R>::type;
  constexpr int NB = 2 * P + 1, NPAIR = (D == 3) ? NB * NB : NB, BAND = NPAIR * NB;
  const RowsArgs &A = AA.rows;
  const int tid = threadIdx.x;
  const bool hasG = AA.G != nullptr, hasH = AA.H != nullptr;
  R *Ub0 = sUb, *Ub1 = sUb + NL1 * NPAIR;
  constexpr int RS = 4, WN = RS + P + 3;
  const O *Hg = hasH ? static_cast<const O *>(AA.H) : nullptr;
  const O *Gg = hasG ? static_cast<const O *>(AA.G) : nullptr;
  const int nseg = (T + RS - 1) / RS, nitems = nseg * NPAIR;
  for (int it0 = 0; it0 < nitems; it0 += NT) {  // uniform trip count: every thread meets the barriers
    const int it = it0 + tid;
    const bool act = it < nitems;
    const int sg = it / NPAIR, pr = it - sg * NPAIR;
    R w0[WN], w1[WN];
#pragma unroll
    for (int c = 0; c < WN; c++) {
      w0[c] = r_zero<R>();
      w1[c] = r_zero<R>();
    }
    if (act) {
      const long long grow = (base + a + sg * RS - A.row_begin) * BAND + (long long)pr * NB;
      const int rl = sg * RS;
      static_assert(RS == 4, "four rows per segment");
      adj_x1_row<P, 0, WN, MAXPTS1, BAND>(w0, w1, rl, T, a, Hg, Gg, grow, sOff1, sE1, sV1, sB1);
      adj_x1_row<P, 1, WN, MAXPTS1, BAND>(w0, w1, rl, T, a, Hg, Gg, grow, sOff1, sE1, sV1, sB1);
      adj_x1_row<P, 2, WN, MAXPTS1, BAND>(w0, w1, rl, T, a, Hg, Gg, grow, sOff1, sE1, sV1, sB1);
      adj_x1_row<P, 3, WN, MAXPTS1, BAND>(w0, w1, rl, T, a, Hg, Gg, grow, sOff1, sE1, sV1, sB1);
    }
    // window column c is coefficient column a + sg*RS - P + c
    const int cbase = a + sg * RS - P - l1lo;
    for (int round = 0; round < 3; round++) {
      if (act && sg % 3 == round) {
#pragma unroll
        for (int c = 0; c < WN; c++) {
          const int col = cbase + c;
          if (col >= 0 && col < nl1) {
            Ub0[col * NPAIR + pr] = r_add(Ub0[col * NPAIR + pr], w0[c]);
            Ub1[col * NPAIR + pr] = r_add(Ub1[col * NPAIR + pr], w1[c]);
          }
        }
      }
      __syncthreads();
    }
  }
}

// Resident CTAs per SM the register allocation is sized for (measured at
// 96^3: four for float, three for double, two for double-float, whose
// register windows spill at three).
#ifndef WQ_ADJ_MIN_BLOCKS_F32
#define WQ_ADJ_MIN_BLOCKS_F32 4
#endif
#ifndef WQ_ADJ_MIN_BLOCKS_F64
#define WQ_ADJ_MIN_BLOCKS_F64 3
#endif
#ifndef WQ_ADJ_MIN_BLOCKS_DD
#define WQ_ADJ_MIN_BLOCKS_DD 2
#endif
template <typename R> constexpr int adj_min_blocks() {
  return sizeof(R) == 4 ? WQ_ADJ_MIN_BLOCKS_F32 : std::is_same<R, dd>::value ? WQ_ADJ_MIN_BLOCKS_DD : WQ_ADJ_MIN_BLOCKS_F64;
}
template <int P, int D, int LM, int TMAX, typename R>
__global__ void __launch_bounds__(32 * kRowsWarps, adj_min_blocks<R>()) adjoint_kernel(const AdjArgs AA) {
  static_assert(D == 2, "3D runs adjoint_x1_kernel and adjoint_u_kernel");
  using L = AdjLayout<P, D, LM, TMAX, R>;
  const RowsArgs &A = AA.rows;
  constexpr int NP = L::NP, NB = L::NB, NT = L::NT, NW = L::NW, NL1 = L::NL1;
  constexpr int NPAIR = L::NPAIR;
  constexpr bool INNER_GAUSS = (LM == P + 1);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sV23 = reinterpret_cast<R *>(smem_raw);
  R *sV23d = sV23 + L::V23;
  R *sB23 = sV23d + L::V23D;
  R *sV1 = sB23 + L::B23;
  R *sB1 = sV1 + L::V1;
  R *sUb = sB1 + L::B1;  // [u][NL1][NPAIR]
  R *sW = sUb + L::UB;
  int *sE23 = reinterpret_cast<int *>(smem_raw + sizeof(R) * (size_t)L::R_TOTAL);
  int *sO23 = sE23 + 2 * LM;
  int *sE1 = sO23 + 2 * LM;
  int *sOff1 = sE1 + L::MAXPTS1;

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
  const int a = (int)lo, b = (int)hi, T = b - a;

  // ------------------------------------------------ tables (as in the forward kernel)
  const int rr[2] = {r2, r3};
  int L23[2] = {1, 1}, l23lo[2] = {0, 0}, nl23[2] = {1, 1};
#pragma unroll
  for (int di = 0; di < D - 1; di++) {
    const int dir = di + 1, r = rr[di];
    const int off0 = A.off[dir][0][r];
    const int off1 = A.off[dir][1][r];
    L23[di] = INNER_GAUSS ? P + 1 : A.off[dir][0][r + 1] - off0;
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
        if constexpr (!INNER_GAUSS) {
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
  const int p1lo = A.off[0][0][a], p1hi = A.off[0][0][b];
  const int np1 = p1hi - p1lo;
  for (int t = tid; t <= T; t += NT) sOff1[t] = A.off[0][0][a + t] - p1lo;
  const int elo1 = a - P < 0 ? 0 : a - P;
  const int ehi1 = (b - 1) > A.N[0] - 1 ? A.N[0] - 1 : (b - 1);
  const int l1lo = elo1, nl1 = ehi1 - elo1 + 4;
  for (int t = tid; t < 2 * NL1 * NPAIR; t += NT) sUb[t] = r_zero<R>();
  __syncthreads();  // sOff1 complete
  for (int t = tid; t < 2 * np1; t += NT) {
    const int kind = t >= np1 ? 1 : 0, q = t - kind * np1;
    const int gq = (kind ? A.off[0][1][a] : p1lo) + q;
    const R *Vg = static_cast<const R *>(A.V[0][kind]);
    const R *Bg = static_cast<const R *>(A.beta[0][kind]);
#pragma unroll
    for (int i = 0; i < NP; i++) sV1[(kind * L::MAXPTS1 + q) * NP + i] = Vg[(size_t)gq * NP + i];
#pragma unroll
    for (int i = 0; i < 4; i++) sB1[(kind * L::MAXPTS1 + q) * 4 + i] = Bg[(size_t)gq * 4 + i];
    if (kind == 0) sE1[q] = A.elem[0][0][p1lo + q];
  }
  const int L2 = L23[0];
  const int nl2 = nl23[0];
  __syncthreads();

  // ------------------------------------------------ 1. x1 stage transposed, register windows
  // Thread (segment s, fibre pr) takes rows s*RS .. s*RS+RS-1 of the chunk for
  // band fibre pr: per row and x1 point q (element e, band offset o = e - r1 + P)
  //   yM = sum_i H[o+i] V1M[q][i], yK = sum_i G[o+i] V1M[q][i], yS = sum_i G[o+i] V1S[q][i]
  // and Ubar0[e+i] += b1M[q][i] yM + b1S[q][i] yS, Ubar1[e+i] += b1M[q][i] yK,
  // kept in a register window over the columns its rows touch.  The windows
  // are then added to Ubar in three ordered rounds (segments s, s+3, ... touch
  // disjoint columns), so the result does not depend on thread timing.
  R *Ub0 = sUb, *Ub1 = sUb + NL1 * NPAIR;
  static_assert(NPAIR == ((D == 3) ? NB * NB : NB), "fibres per row");
  adj_x1_stage<P, D, L::MAXPTS1, NL1, NT, R>(AA, sV1, sB1, sE1, sOff1, sUb, a, T, base, l1lo, nl1);

  // ------------------------------------------------ 2. x2 stage transposed, warp per column
  // this chunk's slot of the block scratch
  const long long chunk_slot = ((long long)line * AA.nch_max + ch) * AA.blk;
  R *wq = sW + warp * L::WS;  // Cqbar
  for (int l1 = warp; l1 < nl1; l1 += NW) {
    {
      // Cqbar[c][q2] = sum_j2 Ubar[c][l1][j2] V2_c[q2][j2 - o2], c = kind2
      for (int t = lane; t < 2 * LM; t += 32) {
        const int q2 = t % LM, c = t / LM;
        if (q2 < L2) {
          const R *ub = (c == 0 ? Ub0 : Ub1) + l1 * NPAIR;
          R s = r_zero<R>();
          if constexpr (INNER_GAUSS) {
#pragma unroll
            for (int i = 0; i < NP; i++) s = r_fma(ub[q2 + i], sV23[(c * LM + q2) * NP + i], s);
          } else {
            const R *vd = &sV23d[(c * LM + q2) * NB];
#pragma unroll
            for (int j = 0; j < NB; j++) s = r_fma(ub[j], vd[j], s);
          }
          wq[t] = s;
        }
      }
      __syncwarp();
      // Cbar[l2] = sum_c sum_q2 Cqbar[c][q2] b2_c[q2][l2 - e2(q2)]
      if (lane < nl2) {
        const int l2 = lane;
        R s = r_zero<R>();
        for (int q2 = 0; q2 < L2; q2++) {
          const int i = l2 - (sE23[q2] - l23lo[0]);
          if (i >= 0 && i < 4) {
            s = r_fma(wq[0 * LM + q2], sB23[(0 * LM + q2) * 4 + i], s);
            s = r_fma(wq[1 * LM + q2], sB23[(1 * LM + q2) * 4 + i], s);
          }
        }
        const long long pidx = chunk_slot + (long long)l2 * AA.nl1max + l1;
        if (check_range(A.status, pidx, 1, (long long)A.n[1] * AA.nch_max * AA.blk)) AA.partial[pidx] = r_to_double(s);
      }
    }
    __syncwarp();
  }
}

template <int P, int D, int LM, int TMAX, typename R>
cudaError_t launch_adjoint_one(const AdjArgs &a, int nblocks, cudaStream_t s) {
  using L = AdjLayout<P, D, LM, TMAX, R>;
  auto kern = adjoint_kernel<P, D, LM, TMAX, R>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  kern<<<nblocks, L::NT, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

// 3D: the x1 stage transposed of one chunk, its Ubar stored in the chunk's
// slot of AA.ubar; the x2 and x3 stages run afterwards, once per block of
// lines and coefficient columns (adjoint_u_kernel), instead of per chunk.
template <int P, int TMAX, typename R> struct AdjX1Layout {
  static constexpr int NP = P + 1, NB = 2 * P + 1, NPAIR = NB * NB;
  static constexpr int NL1 = TMAX + P + 3;
  static constexpr int MAXPTS1 = TMAX * NP + P * NP * (P - 1);
  static constexpr int NT = 32 * kRowsWarps;
  static constexpr int V1 = pad16<R>(2 * MAXPTS1 * NP);
  static constexpr int B1 = pad16<R>(2 * MAXPTS1 * 4);
  static constexpr int UB = pad16<R>(2 * NL1 * NPAIR);  // [u][NL1][pair]
  static constexpr int R_TOTAL = V1 + B1 + UB;
  static constexpr int I_TOTAL = MAXPTS1 + TMAX + 1;
  static constexpr size_t BYTES = sizeof(R) * (size_t)R_TOTAL + sizeof(int) * (size_t)I_TOTAL;
};

template <int P, int TMAX, typename R>
__global__ void __launch_bounds__(32 * kRowsWarps, adj_min_blocks<R>()) adjoint_x1_kernel(const AdjArgs AA) {
  using L = AdjX1Layout<P, TMAX, R>;
  const RowsArgs &A = AA.rows;
  constexpr int NP = L::NP, NT = L::NT, NL1 = L::NL1, NPAIR = L::NPAIR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sV1 = reinterpret_cast<R *>(smem_raw);
  R *sB1 = sV1 + L::V1;
  R *sUb = sB1 + L::B1;
  int *sE1 = reinterpret_cast<int *>(smem_raw + sizeof(R) * (size_t)L::R_TOTAL);
  int *sOff1 = sE1 + L::MAXPTS1;

  const int tid = threadIdx.x;
  const int line = A.lines[blockIdx.x / A.nch];
  const int ch = blockIdx.x % A.nch;
  const int n1 = A.n[0];
  const long long base = (long long)line * n1;
  long long lo = (long long)ch * A.T, hi = lo + A.T;
  if (hi > n1) hi = n1;
  if (lo < A.row_begin - base) lo = A.row_begin - base;
  if (hi > A.row_end - base) hi = A.row_end - base;
  if (lo >= hi) return;
  const int a = (int)lo, b = (int)hi, T = b - a;

  const int p1lo = A.off[0][0][a], p1hi = A.off[0][0][b];
  const int np1 = p1hi - p1lo;
  for (int t = tid; t <= T; t += NT) sOff1[t] = A.off[0][0][a + t] - p1lo;
  const int elo1 = a - P < 0 ? 0 : a - P;
  const int ehi1 = (b - 1) > A.N[0] - 1 ? A.N[0] - 1 : (b - 1);
  const int l1lo = elo1, nl1 = ehi1 - elo1 + 4;
  for (int t = tid; t < 2 * NL1 * NPAIR; t += NT) sUb[t] = r_zero<R>();
  for (int t = tid; t < 2 * np1; t += NT) {
    const int kind = t >= np1 ? 1 : 0, q = t - kind * np1;
    const int gq = (kind ? A.off[0][1][a] : p1lo) + q;
    const R *Vg = static_cast<const R *>(A.V[0][kind]);
    const R *Bg = static_cast<const R *>(A.beta[0][kind]);
#pragma unroll
    for (int i = 0; i < NP; i++) sV1[(kind * L::MAXPTS1 + q) * NP + i] = Vg[(size_t)gq * NP + i];
#pragma unroll
    for (int i = 0; i < 4; i++) sB1[(kind * L::MAXPTS1 + q) * 4 + i] = Bg[(size_t)gq * 4 + i];
    if (kind == 0) sE1[q] = A.elem[0][0][p1lo + q];
  }
  __syncthreads();

  adj_x1_stage<P, 3, L::MAXPTS1, NL1, NT, R>(AA, sV1, sB1, sE1, sOff1, sUb, a, T, base, l1lo, nl1);

  // the chunk's window columns to its slot, [u][column][pair]
  R *Ug = static_cast<R *>(AA.ubar);
  const long long slot = ((long long)line * AA.nch_max + ch) * AA.ubar_slot;
  const long long total = (long long)A.n[1] * A.n[2] * AA.nch_max * AA.ubar_slot;
  const int run = nl1 * NPAIR;
  for (int t = tid; t < 2 * run; t += NT) {
    const int u = t >= run ? 1 : 0, rem = t - u * run;
    const long long di = slot + (long long)u * AA.nl1max * NPAIR + rem;
    if (check_range(A.status, di, 1, total)) Ug[di] = sUb[u * NL1 * NPAIR + rem];
  }
}

template <int P, int TMAX, typename R>
cudaError_t launch_adjoint_x1_one(const AdjArgs &a, int nblocks, cudaStream_t s) {
  using L = AdjX1Layout<P, TMAX, R>;
  auto kern = adjoint_x1_kernel<P, TMAX, R>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  kern<<<nblocks, L::NT, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wq
