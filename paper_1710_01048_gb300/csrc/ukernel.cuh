// The 3D assembly split in two kernels.
//
// u_kernel computes, for every line (r2, r3) in a range and every coefficient
// column l1, the two partial contractions of the row kernel's first phase
// (Eq. Decompo applied to the weighted sums of Eq. GaussQuadSys and
// Eq. GaussQuadSysStiff, with the coefficient spline c as the integrand's
// factor):
//   T3_k3[l1][l2][j3] = sum_q3 (sum_i3 C[l1][l2][e3(q3)+i3] b3_k3[q3][i3]) V3_k3[q3][j3-o3]
//   U0[l1][j3][j2] = sum_q2 Cq_MM[q2][j3] V2M[q2][j2-o2]
//   U1[l1][j3][j2] = sum_q2 Cq_SM[q2][j3] V2S[q2][j2-o2] + Cq_MS[q2][j3] V2M[q2][j2-o2]
//   Cq_c[q2][j3]   = sum_i2 T3_k3(c)[l1][e2(q2)+i2][j3] b2_k2(c)[q2][i2]
// and stores U in global memory, [line][u][l1][j3*(2P+1)+j2].  T3 depends on
// r3 only, so a CTA takes a block of kULines lines of one plane (same r3) and
// kUCols columns and computes T3 once for all of them; each line's x2 stage
// then reads it from shared memory.  Each warp stages its items' U values in
// shared memory and writes them with consecutive lanes on consecutive
// addresses.  The operation order of every value is
// the row kernel's, so the split and the fused path give the same bits.
//
// rows_ug_kernel is the row kernel without its first phase: it copies the
// chunk's U columns from global memory and runs phase B.  All lines take the
// same path (the x2/x3 rule lengths no longer matter), so one launch covers a
// range of lines.
#pragma once

#include "assemble.cuh"

namespace wq {

#ifndef WQ_UCOLS
#define WQ_UCOLS 8
#endif
constexpr int kULines = 8, kUCols = WQ_UCOLS;

// A table row of N values from shared memory into registers: as 16-byte
// loads where the row is four floats (rows start on 16-byte boundaries),
// else value by value.
template <int N, typename R> __device__ __forceinline__ void load_row(R (&d)[N], const R *s) {
  if constexpr (std::is_same<R, float>::value && N == 4) {
    const float4 x = *reinterpret_cast<const float4 *>(s);
    d[0] = x.x;
    d[1] = x.y;
    d[2] = x.z;
    d[3] = x.w;
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) d[i] = s[i];
  }
}
template <typename R> __device__ __forceinline__ void load_row4(R (&d)[4], const R *s) { load_row<4>(d, s); }

struct UArgs {
  const int *off[3][2];
  const int *elem[3][2];
  const void *V[3][2];
  const void *beta[3][2];
  int n[3], N[3], nc[3];
  const double *coef;  // may be null: c = 1
  const void *coefR;   // the same in R (checked), or null
  void *U;             // [line][2][nc1][(2P+1)^2] in R
  int line_lo, line_hi;  // lines [line_lo, line_hi] are written
  int r3_lo;             // plane of the launch's first CTA
  int nblk2, nblk1;      // line blocks per plane, column blocks
  unsigned *status;
  float zero;  // 0.0f, read at run time by the packed double-float path (dd2_fma)
};

template <int P, typename R> struct ULayout {
  static constexpr int NP = P + 1, NB = 2 * P + 1;
  static constexpr int LM = P * (P + 1);          // most points of one row in one direction
  static constexpr int NL2 = kULines + P + 3;      // x2 coefficient indices of the CTA's lines
  static constexpr int NL3 = P + 4;                // x3 coefficient indices of one row
  static constexpr int V3 = pad16<R>(2 * LM * NP);             // [k3][q3][i]
  static constexpr int B3 = pad16<R>(2 * LM * 4);              // [k3][q3][i]
  static constexpr int V2 = pad16<R>(kULines * 2 * LM * NP);   // [b][k2][q2][i]
  static constexpr int B2 = pad16<R>(kULines * 2 * LM * 4);    // [b][k2][q2][i]
  static constexpr int CB = pad16<R>(kUCols * NL2 * NL3);      // [l1][l2][l3]
  // T3 [k3][l1] blocks of NL2 * NB values, padded to a stride = NB (mod 32):
  // the x2 stage's 32 lanes read runs of NB values from consecutive l1
  // blocks, which then fall in disjoint shared-memory banks
  static constexpr int T3S = NL2 * NB + ((NB - NL2 * NB) % 32 + 32) % 32;
  static constexpr int T3 = pad16<R>(2 * kUCols * T3S);          // [k3][l1][l2][j3]
  // per-warp stage: float, one buffer per u written by bulk copies (a run of
  // 32 items plus alignment slack); otherwise one buffer for both in turn
  static constexpr bool BULK = std::is_same<R, float>::value;
  static constexpr int WSTB = pad16<R>(32 * NB + 3);
  static constexpr int WST = BULK ? 2 * WSTB : pad16<R>(32 * NB);
  static constexpr int R_TOTAL = V3 + B3 + V2 + B2 + CB + T3 + 8 * WST;
  // int region: e3[LM], o3[LM], L2[kULines], e2[kULines][LM], o2[kULines][LM]
  static constexpr int I_TOTAL = 2 * LM + kULines + 2 * kULines * LM;
  static constexpr size_t BYTES = sizeof(R) * (size_t)R_TOTAL + sizeof(int) * (size_t)I_TOTAL;
};

// The work of one u_kernel CTA: block `bid` (plane, line block, column
// block) in the dynamic shared memory `smem_raw` (ULayout::BYTES).
template <int P, typename R>
__device__ __forceinline__ void u_block(const UArgs &A, int bid, unsigned char *smem_raw) {
  using L = ULayout<P, R>;
  constexpr int NP = L::NP, NB = L::NB, NPAIR = NB * NB, LM = L::LM, NL2 = L::NL2, NL3 = L::NL3;
  constexpr int NT = 256;
  R *sV3 = reinterpret_cast<R *>(smem_raw);
  R *sB3 = sV3 + L::V3;
  R *sV2 = sB3 + L::B3;
  R *sB2 = sV2 + L::V2;
  R *sCb = sB2 + L::B2;
  R *sT3 = sCb + L::CB;
  R *sSt = sT3 + L::T3;
  int *sE3 = reinterpret_cast<int *>(smem_raw + sizeof(R) * (size_t)L::R_TOTAL);
  int *sO3 = sE3 + LM;
  int *sL2 = sO3 + LM;
  int *sE2 = sL2 + kULines;

  const int tid = threadIdx.x;
  const int n2 = A.n[1], nc1 = A.nc[0], nc2 = A.nc[1];
  const int b1 = bid % A.nblk1;
  bid /= A.nblk1;
  const int b2 = bid % A.nblk2;
  const int r3 = A.r3_lo + bid / A.nblk2;
  const int r2a = b2 * kULines;
  const int nlines = (n2 - r2a) < kULines ? (n2 - r2a) : kULines;
  const int lid0 = r2a + n2 * r3;
  if (lid0 + nlines - 1 < A.line_lo || lid0 > A.line_hi) return;
  const int l1a = b1 * kUCols;
  const int ncols = (nc1 - l1a) < kUCols ? (nc1 - l1a) : kUCols;

  // x3 rule of row r3
  const int off30 = A.off[2][0][r3], off31 = A.off[2][1][r3];
  const int L3 = A.off[2][0][r3 + 1] - off30;
  // (tables and the coefficient block by asynchronous copies, all in flight
  // together; the offsets o = e - r + P are formed where they are used)
#pragma unroll
  for (int kind = 0; kind < 2; kind++) {
    const int o = kind ? off31 : off30;
    cp_async_n(&sV3[kind * LM * NP], static_cast<const R *>(A.V[2][kind]) + (size_t)o * NP, L3 * NP, tid, NT);
    cp_async_n(&sB3[kind * LM * 4], static_cast<const R *>(A.beta[2][kind]) + (size_t)o * 4, L3 * 4, tid, NT);
  }
  cp_async_n(sE3, A.elem[2][0] + off30, L3, tid, NT);
  // x2 rules of the block's lines
  for (int t = tid; t < kULines * 2 * LM; t += NT) {
    const int b = t / (2 * LM), kind = (t / LM) % 2, q = t % LM;
    if (b < nlines) {
      const int r2 = r2a + b;
      const int off0 = A.off[1][0][r2];
      const int L2b = A.off[1][0][r2 + 1] - off0;
      if (kind == 0 && q == 0) sL2[b] = L2b;
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
    }
  }
  // the coefficient block: columns l1a.., x2 indices l2lo.., x3 indices l3lo..
  const int l2lo = (r2a - P) > 0 ? (r2a - P) : 0;
  const int l2hi = ((r2a + nlines - 1) < (A.N[1] - 1) ? (r2a + nlines - 1) : (A.N[1] - 1)) + 3;
  const int nl2 = l2hi - l2lo + 1;
  const int l3lo = (r3 - P) > 0 ? (r3 - P) : 0;
  const int nl3 = (r3 < A.N[2] - 1 ? r3 : A.N[2] - 1) - l3lo + 4;
  {
    unsigned bad = 0;
    const double *cg = A.coef;
    const R *cr = static_cast<const R *>(A.coefR);
    for (int t = tid; t < NL3 * NL2 * kUCols; t += NT) {
      const int l1 = t % kUCols, l2 = (t / kUCols) % NL2, l3 = t / (kUCols * NL2);
      if (l1 < ncols && l2 < nl2 && l3 < nl3) {
        const long long g = (long long)(l1a + l1) + (long long)nc1 * ((long long)(l2lo + l2) + (long long)nc2 * (l3lo + l3));
        R *dst = &sCb[(l1 * NL2 + l2) * NL3 + l3];
        if (cr) {
          cp_async_el(dst, &cr[g]);
        } else if (cg) {
          const double x = cg[g];
          if (!isfinite(x)) bad = 1;
          *dst = r_from_double<R>(x);
        } else {
          *dst = r_from_double<R>(1.0);
        }
      }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (tid & 31) == 0) atomicOr(A.status, 2u);
  }
  cp_async_wait_all();
  __syncthreads();

  // x3 stage, once for the block: items (k3, l1, l2)
  const bool in3 = r3 >= P && r3 <= A.N[2] - 1;
  for (int t = tid; t < 2 * kUCols * NL2; t += NT) {
    const int l2 = t % NL2, l1 = (t / NL2) % kUCols, k3 = t / (NL2 * kUCols);
    if (l1 < ncols && l2 < nl2) {
      const R *cb = &sCb[(l1 * NL2 + l2) * NL3];
      R acc[NB];
#pragma unroll
      for (int j = 0; j < NB; j++) acc[j] = r_zero<R>();
      if (in3) {
        // interior plane: point q3 in element e0 + q3
        const int e0 = sE3[0] - l3lo;
        R c[NP + 3];
#pragma unroll
        for (int i = 0; i < NP + 3; i++) c[i] = cb[e0 + i];
#pragma unroll
        for (int q3 = 0; q3 < NP; q3++) {
          R bb[4], v[NP];
          load_row4(bb, &sB3[(k3 * LM + q3) * 4]);
          load_row<NP>(v, &sV3[(k3 * LM + q3) * NP]);
          R z = r_zero<R>();
#pragma unroll
          for (int i = 0; i < 4; i++) z = r_fma(c[q3 + i], bb[i], z);
#pragma unroll
          for (int i = 0; i < NP; i++) acc[q3 + i] = r_fma(z, v[i], acc[q3 + i]);
        }
      } else {
        for (int q3 = 0; q3 < L3; q3++) {
          const int e = sE3[q3] - l3lo;
          const R *bb = &sB3[(k3 * LM + q3) * 4];
          R z = r_zero<R>();
#pragma unroll
          for (int i = 0; i < 4; i++) z = r_fma(cb[e + i], bb[i], z);
          fiber_shift<P>(acc, z, &sV3[(k3 * LM + q3) * NP], sE3[q3] - r3 + P);
        }
      }
#pragma unroll
      for (int j = 0; j < NB; j++) sT3[(k3 * kUCols + l1) * L::T3S + l2 * NB + j] = acc[j];
    }
  }
  __syncthreads();

  // x2 stage: warp w takes line w of the block, items (l1, j3) of that line
  // 32 at a time; item i's NB values of U sit at offset i * NB of the line's
  // run of the block's columns, so the warp's outputs are one contiguous run
  static_assert(kULines == kRowsWarps, "one warp per line of the block");
  R *Ug = static_cast<R *>(A.U);
  const int lane = tid & 31, warp = tid >> 5;
  R *wst = sSt + warp * L::WST;
  const int b = warp;
  const int nitem = ncols * NB;
  const bool line_ok = b < nlines && lid0 + b >= A.line_lo && lid0 + b <= A.line_hi;
  for (int i0 = 0; line_ok && i0 < nitem; i0 += 32) {
    const int t = i0 + lane;
    const bool ok = t < nitem;
    const int l1 = t / NB, j3 = t - l1 * NB;
    R u0[NB], u1[NB];
#pragma unroll
    for (int j = 0; j < NB; j++) {
      u0[j] = r_zero<R>();
      u1[j] = r_zero<R>();
    }
    if (ok) {
      const int r2 = r2a + b, L2 = sL2[b];
      const bool in2 = r2 >= P && r2 <= A.N[1] - 1;
      const R *t3m = &sT3[(0 * kUCols + l1) * L::T3S + j3];  // k3 = 0, index by l2 * NB
      const R *t3s = &sT3[(1 * kUCols + l1) * L::T3S + j3];  // k3 = 1
      const R *v2 = &sV2[(b * 2) * LM * NP];
      const R *b2 = &sB2[(b * 2) * LM * 4];
      if (std::is_same<R, dd>::value && in2 && in3) {
        // interior line in double-float: the same order, with the updates
        // that share a table entry as packed pairs (s0, s2) and (u0, u1)
        if constexpr (std::is_same<R, dd>::value) {
          const unsigned long long z = f2_pack(A.zero, A.zero);
          dd2 c02[NP];
          dd c1[NP];
#pragma unroll
          for (int q2 = 0; q2 < NP; q2++) {
            const int e = sE2[b * LM + q2] - l2lo;
            const R *bm = &b2[(0 * LM + q2) * 4], *bs = &b2[(1 * LM + q2) * 4];
            dd2 s02{z, z};
            dd s1 = r_zero<dd>();
#pragma unroll
            for (int i = 0; i < 4; i++) {
              const dd tm = t3m[(e + i) * NB], ts = t3s[(e + i) * NB], bb = bm[i];
              s02 = dd2_fma(dd2_pack(tm, ts), dd2_pack(bb, bb), s02, z);
              s1 = dd_fma(tm, bs[i], s1);
            }
            c02[q2] = s02;
            c1[q2] = s1;
          }
#pragma unroll
          for (int q2 = 0; q2 < NP; q2++) {
            const R *vs = &v2[(1 * LM + q2) * NP];
#pragma unroll
            for (int i = 0; i < NP; i++) u1[q2 + i] = dd_fma(c1[q2], vs[i], u1[q2 + i]);
          }
          dd2 u01[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) u01[j] = dd2{f2_pack(A.zero, u1[j].hi), f2_pack(A.zero, u1[j].lo)};
#pragma unroll
          for (int q2 = 0; q2 < NP; q2++) {
            const R *vm = &v2[(0 * LM + q2) * NP];
#pragma unroll
            for (int i = 0; i < NP; i++) {
              const dd v = vm[i];
              u01[q2 + i] = dd2_fma(c02[q2], dd2_pack(v, v), u01[q2 + i], z);
            }
          }
#pragma unroll
          for (int j = 0; j < NB; j++) {
            u0[j] = dd2_first(u01[j]);
            u1[j] = dd2_second(u01[j]);
          }
        }
      } else if (in2 && in3) {
        // interior line: the row kernel's order, all q2 of (S, M) before (M, S);
        // point q2 lies in element e0 + q2, so the item's T3 values are read
        // once, and the line's tables row by row (16-byte loads in float)
        const int e0 = sE2[b * LM] - l2lo;
        R tm[NP + 3], ts[NP + 3];
#pragma unroll
        for (int i = 0; i < NP + 3; i++) {
          tm[i] = t3m[(e0 + i) * NB];
          ts[i] = t3s[(e0 + i) * NB];
        }
        if constexpr (std::is_same<R, float>::value) {
          // float: the pairs that share a table entry as packed fma.rn.f32x2,
          // (s0, s2) += (tm, ts) b2M and (u0, u1) += (c0, c2) V2M, each lane
          // in the scalar order below (u1 takes all of (S, M) first)
          const unsigned long long z = f2_pack(A.zero, A.zero);
          unsigned long long c02[NP];
          float c1f[NP];
#pragma unroll
          for (int q2 = 0; q2 < NP; q2++) {
            float bm[4], bs[4];
            load_row4(bm, &b2[(0 * LM + q2) * 4]);
            load_row4(bs, &b2[(1 * LM + q2) * 4]);
            unsigned long long s02 = z;
            float s1 = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; i++) {
              s02 = f2_fma(f2_pack(tm[q2 + i], ts[q2 + i]), f2_pack(bm[i], bm[i]), s02);
              s1 = fmaf(tm[q2 + i], bs[i], s1);
            }
            c02[q2] = s02;
            c1f[q2] = s1;
          }
#pragma unroll
          for (int q2 = 0; q2 < NP; q2++) {
            float vs[NP];
            load_row<NP>(vs, &v2[(1 * LM + q2) * NP]);
#pragma unroll
            for (int i = 0; i < NP; i++) u1[q2 + i] = fmaf(c1f[q2], vs[i], u1[q2 + i]);
          }
          unsigned long long u01[NB];
#pragma unroll
          for (int j = 0; j < NB; j++) u01[j] = f2_pack(A.zero, u1[j]);
#pragma unroll
          for (int q2 = 0; q2 < NP; q2++) {
            float vm[NP];
            load_row<NP>(vm, &v2[(0 * LM + q2) * NP]);
#pragma unroll
            for (int i = 0; i < NP; i++) u01[q2 + i] = f2_fma(c02[q2], f2_pack(vm[i], vm[i]), u01[q2 + i]);
          }
#pragma unroll
          for (int j = 0; j < NB; j++) f2_unpack(u01[j], u0[j], u1[j]);
        } else {
        R c0[NP], c1[NP], c2[NP];
#pragma unroll
        for (int q2 = 0; q2 < NP; q2++) {
          R bm[4], bs[4];
          load_row4(bm, &b2[(0 * LM + q2) * 4]);
          load_row4(bs, &b2[(1 * LM + q2) * 4]);
          R s0 = r_zero<R>(), s1 = r_zero<R>(), s2 = r_zero<R>();
#pragma unroll
          for (int i = 0; i < 4; i++) {
            s0 = r_fma(tm[q2 + i], bm[i], s0);
            s1 = r_fma(tm[q2 + i], bs[i], s1);
            s2 = r_fma(ts[q2 + i], bm[i], s2);
          }
          c0[q2] = s0;
          c1[q2] = s1;
          c2[q2] = s2;
        }
        R vm[NP][NP], vs[NP][NP];
#pragma unroll
        for (int q2 = 0; q2 < NP; q2++) {
          load_row<NP>(vm[q2], &v2[(0 * LM + q2) * NP]);
          load_row<NP>(vs[q2], &v2[(1 * LM + q2) * NP]);
        }
#pragma unroll
        for (int q2 = 0; q2 < NP; q2++)
#pragma unroll
          for (int i = 0; i < NP; i++) u0[q2 + i] = r_fma(c0[q2], vm[q2][i], u0[q2 + i]);
#pragma unroll
        for (int q2 = 0; q2 < NP; q2++)
#pragma unroll
          for (int i = 0; i < NP; i++) u1[q2 + i] = r_fma(c1[q2], vs[q2][i], u1[q2 + i]);
#pragma unroll
        for (int q2 = 0; q2 < NP; q2++)
#pragma unroll
          for (int i = 0; i < NP; i++) u1[q2 + i] = r_fma(c2[q2], vm[q2][i], u1[q2 + i]);
        }
      } else {
        // boundary line: per point, (S, M) then (M, S)
        for (int q2 = 0; q2 < L2; q2++) {
          const int e = sE2[b * LM + q2] - l2lo, o = sE2[b * LM + q2] - r2 + P;
          const R *bm = &b2[(0 * LM + q2) * 4], *bs = &b2[(1 * LM + q2) * 4];
          R s0 = r_zero<R>(), s1 = r_zero<R>(), s2 = r_zero<R>();
#pragma unroll
          for (int i = 0; i < 4; i++) {
            s0 = r_fma(t3m[(e + i) * NB], bm[i], s0);
            s1 = r_fma(t3m[(e + i) * NB], bs[i], s1);
            s2 = r_fma(t3s[(e + i) * NB], bm[i], s2);
          }
          fiber_shift<P>(u0, s0, &v2[(0 * LM + q2) * NP], o);
          fiber_shift<P>(u1, s1, &v2[(1 * LM + q2) * NP], o);
          fiber_shift<P>(u1, s2, &v2[(0 * LM + q2) * NP], o);
        }
      }
    }
    // U[line][u][l1][j3*NB+j2]: contiguous from column l1a, item i0 onwards
    const int nent = ((nitem - i0) < 32 ? (nitem - i0) : 32) * NB;
    if constexpr (L::BULK) {
      // both runs staged, written by bulk copies (lane 0) and plain stores of
      // their unaligned ends; the previous runs' copies have read the stage
      if (lane == 0) bulk_wait_read();
      __syncwarp();
      float *dst[2], *st[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        dst[u] = Ug + (((size_t)(lid0 + b) * 2 + u) * nc1 + l1a) * NPAIR + (size_t)i0 * NB;
        st[u] = wst + u * L::WSTB + (int)(((uintptr_t)dst[u] >> 2) & 3);
        if (ok) {
#pragma unroll
          for (int j = 0; j < NB; j++) st[u][lane * NB + j] = u ? u1[j] : u0[j];
        }
      }
      fence_proxy_async();
      __syncwarp();
      const long long utot = (long long)A.n[1] * A.n[2] * 2 * nc1 * NPAIR;
      if (check_range(A.status, (((long long)(lid0 + b) * 2 + 0) * nc1 + l1a) * NPAIR + (long long)i0 * NB, nent, utot))
        stage_out(dst[0], st[0], nent, lane, 0, 1);
      if (check_range(A.status, (((long long)(lid0 + b) * 2 + 1) * nc1 + l1a) * NPAIR + (long long)i0 * NB, nent, utot))
        stage_out(dst[1], st[1], nent, lane, 0, 8);
      if (lane == 0) bulk_commit();
    } else {
#pragma unroll
      for (int u = 0; u < 2; u++) {
        if (ok) {
#pragma unroll
          for (int j = 0; j < NB; j++) wst[lane * NB + j] = u ? u1[j] : u0[j];
        }
        __syncwarp();
        R *dst = Ug + (((size_t)(lid0 + b) * 2 + u) * nc1 + l1a) * NPAIR + (size_t)i0 * NB;
        if (check_range(A.status, (((long long)(lid0 + b) * 2 + u) * nc1 + l1a) * NPAIR + (long long)i0 * NB, nent,
                        (long long)A.n[1] * A.n[2] * 2 * nc1 * NPAIR))
          for (int e = lane; e < nent; e += 32) dst[e] = wst[e];
        __syncwarp();
      }
    }
  }
  if constexpr (L::BULK) {
    if (lane == 0) bulk_wait_read();  // the stage is read before the CTA's shared memory is released
    __syncwarp();
  }
}

// Four resident CTAs per SM (the shared-memory limit as well).
#ifndef WQ_U_MIN_BLOCKS
#define WQ_U_MIN_BLOCKS 4
#endif
template <int P, typename R> __global__ void __launch_bounds__(256, WQ_U_MIN_BLOCKS) u_kernel(const UArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  u_block<P, R>(A, blockIdx.x, smem_raw);
}

// Row kernel of the split path: x1 tables and U columns in shared memory, then phase B.
template <int P, int TMAX, bool DO_M, bool DO_K, typename R> struct RowsLayoutUG {
  static constexpr int NP = P + 1, NB = 2 * P + 1, NPAIR = NB * NB;
  static constexpr int NL1 = TMAX + P + 3;
  static constexpr int NU = DO_K ? 2 : 1;
  static constexpr int NW = kRowsWarps;
  static constexpr int MAXPTS1 = TMAX * NP + P * NP * (P - 1);
  static constexpr int V1 = pad16<R>(2 * MAXPTS1 * NP);
  static constexpr int B1 = pad16<R>(2 * MAXPTS1 * 4);
  static constexpr int US = pad16<R>(NU * NL1 * NPAIR);
  static constexpr int STAGE = NW * stage_per_warp<R, NB, false>();
  static constexpr int R_TOTAL = V1 + B1 + US + STAGE;
  static constexpr int I_TOTAL = MAXPTS1 + TMAX + 1;
  static constexpr size_t BYTES = sizeof(R) * (size_t)R_TOTAL + sizeof(int) * (size_t)I_TOTAL;
};

// The work of one rows_ug_kernel CTA: chunk `bid` of lines line0, line0+1, ...
template <int P, int TMAX, bool DO_M, bool DO_K, typename R>
__device__ __forceinline__ void rows_ug_block(const RowsArgs &A, int bid, unsigned char *smem_raw) {
  using L = RowsLayoutUG<P, TMAX, DO_M, DO_K, R>;
  constexpr int NPAIR = L::NPAIR, NL1 = L::NL1, NT = 32 * kRowsWarps;
  R *sV1 = reinterpret_cast<R *>(smem_raw);
  R *sB1 = sV1 + L::V1;
  R *sU = sB1 + L::B1;
  R *sW = sU + L::US;
  int *sE1 = reinterpret_cast<int *>(smem_raw + sizeof(R) * (size_t)L::R_TOTAL);
  int *sOff1 = sE1 + L::MAXPTS1;

  const int tid = threadIdx.x;
  const int line = A.line0 + bid / A.nch;
  const int ch = bid % A.nch;
  const int n1 = A.n[0];
  const long long base = (long long)line * n1;
  long long lo = (long long)ch * A.T, hi = lo + A.T;
  if (hi > n1) hi = n1;
  if (lo < A.row_begin - base) lo = A.row_begin - base;
  if (hi > A.row_end - base) hi = A.row_end - base;
  if (lo >= hi) return;
  const int a = (int)lo, b = (int)hi, T = b - a;

  load_x1_tables<P, L::MAXPTS1, R>(A, a, T, sV1, sB1, sE1, sOff1);
  const int elo1 = a - P < 0 ? 0 : a - P;
  const int ehi1 = (b - 1) > A.N[0] - 1 ? A.N[0] - 1 : (b - 1);
  const int l1lo = elo1, nl1 = ehi1 - elo1 + 4;
  const R *Ug = static_cast<const R *>(A.Ug);
  const int nc1 = A.nc[0];
#pragma unroll
  for (int u = 0; u < L::NU; u++)
    if (check_range(A.status, (((long long)line * 2 + u) * nc1 + l1lo) * NPAIR, (long long)nl1 * NPAIR,
                    (long long)A.n[1] * A.n[2] * 2 * nc1 * NPAIR))
      cp_async_n(sU + u * NL1 * NPAIR, Ug + (((size_t)line * 2 + u) * nc1 + l1lo) * NPAIR, nl1 * NPAIR, tid, NT);
  cp_async_wait_all();
  __syncthreads();
  rows_phase_b<P, 3, L::MAXPTS1, NL1, false, DO_M, DO_K, R>(A, sU, sV1, sB1, sE1, sOff1, sW, a, T, l1lo, base);
}

template <int P, int TMAX, bool DO_M, bool DO_K, typename R>
__global__ void __launch_bounds__(32 * kRowsWarps, rows_min_blocks<R>()) rows_ug_kernel(const RowsArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_ug_block<P, TMAX, DO_M, DO_K, R>(A, blockIdx.x, smem_raw);
}

// Chunk length of the split row kernel (every line, any rule lengths in x2, x3).
#ifndef WQ_UG_CHUNK
#define WQ_UG_CHUNK 32
#endif
constexpr int kUGChunk = WQ_UG_CHUNK;

template <int P, typename R> cudaError_t launch_u(const UArgs &a, int nblocks, cudaStream_t s) {
  using L = ULayout<P, R>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(u_kernel<P, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  u_kernel<P, R><<<nblocks, 256, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int P, bool DO_M, bool DO_K, typename R>
cudaError_t launch_ug_one(const RowsArgs &a, int nblocks, cudaStream_t s) {
  using L = RowsLayoutUG<P, kUGChunk, DO_M, DO_K, R>;
  auto kern = rows_ug_kernel<P, kUGChunk, DO_M, DO_K, R>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  kern<<<nblocks, 32 * kRowsWarps, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int P, typename R>
cudaError_t launch_rows_ug(bool do_m, bool do_k, const RowsArgs &a, int nblocks, cudaStream_t s) {
  if (do_m && do_k) return launch_ug_one<P, true, true, R>(a, nblocks, s);
  if (do_m) return launch_ug_one<P, true, false, R>(a, nblocks, s);
  return launch_ug_one<P, false, true, R>(a, nblocks, s);
}

// ---------------------------------------------------------------- matrix-free apply
// The split row kernel with y = M x, y = K x in place of the band: per chunk
// of up to kApplyChunk rows of one line, the x1 tables, the U columns and x
// at the chunk's columns in shared memory, then phase B in APPLY mode (the
// band entries of a fibre meet x in registers; per-row sums by one warp).
#ifndef WQ_APPLY_CHUNK
#define WQ_APPLY_CHUNK 24
#endif
constexpr int kApplyChunk = WQ_APPLY_CHUNK;

template <int P, bool DO_M, bool DO_K, typename R> struct ApplyLayoutUG {
  static constexpr int TMAX = kApplyChunk;
  static constexpr int NP = P + 1, NB = 2 * P + 1, NPAIR = NB * NB;
  static constexpr int NL1 = TMAX + P + 3;
  static constexpr int XL = TMAX + 2 * P;  // x columns a - P .. a + TMAX - 1 + P
  static constexpr int NU = DO_K ? 2 : 1;
  static constexpr int MAXPTS1 = TMAX * NP + P * NP * (P - 1);
  static constexpr int V1 = pad16<R>(2 * MAXPTS1 * NP);
  static constexpr int B1 = pad16<R>(2 * MAXPTS1 * 4);
  static constexpr int US = pad16<R>(NU * NL1 * NPAIR);
  static constexpr int XS = pad16<R>(NPAIR * XL);
  static constexpr int PART = pad16<R>(2 * TMAX * NPAIR);  // per-fibre partial sums (M, K)
  static constexpr int R_TOTAL = V1 + B1 + US + XS + PART;
  static constexpr int I_TOTAL = MAXPTS1 + TMAX + 1;
  static constexpr size_t BYTES = sizeof(R) * (size_t)R_TOTAL + sizeof(int) * (size_t)I_TOTAL;
};

template <int P, bool DO_M, bool DO_K, typename R>
__device__ __forceinline__ void apply_ug_block(const RowsArgs &A, int bid, unsigned char *smem_raw) {
  using L = ApplyLayoutUG<P, DO_M, DO_K, R>;
  constexpr int NPAIR = L::NPAIR, NL1 = L::NL1, XL = L::XL, NT = 32 * kRowsWarps;
  static_assert(NL1 + P - 3 == XL, "x row length seen by phase B");
  R *sV1 = reinterpret_cast<R *>(smem_raw);
  R *sB1 = sV1 + L::V1;
  R *sU = sB1 + L::B1;
  R *sX = sU + L::US;
  R *sP = sX + L::XS;
  int *sE1 = reinterpret_cast<int *>(smem_raw + sizeof(R) * (size_t)L::R_TOTAL);
  int *sOff1 = sE1 + L::MAXPTS1;

  const int tid = threadIdx.x;
  const int line = A.line0 + bid / A.nch;
  const int ch = bid % A.nch;
  const int n1 = A.n[0];
  const long long base = (long long)line * n1;
  long long lo = (long long)ch * A.T, hi = lo + A.T;
  if (hi > n1) hi = n1;
  if (lo < A.row_begin - base) lo = A.row_begin - base;
  if (hi > A.row_end - base) hi = A.row_end - base;
  if (lo >= hi) return;  // uniform across the CTA: no thread reaches the barriers below
  const int a = (int)lo, b = (int)hi, T = b - a;

  load_x1_tables<P, L::MAXPTS1, R>(A, a, T, sV1, sB1, sE1, sOff1);
  const int elo1 = a - P < 0 ? 0 : a - P;
  const int ehi1 = (b - 1) > A.N[0] - 1 ? A.N[0] - 1 : (b - 1);
  const int l1lo = elo1, nl1 = ehi1 - elo1 + 4;
  const R *Ug = static_cast<const R *>(A.Ug);
  const int nc1 = A.nc[0];
#pragma unroll
  for (int u = 0; u < L::NU; u++)
    if (check_range(A.status, (((long long)line * 2 + u) * nc1 + l1lo) * NPAIR, (long long)nl1 * NPAIR,
                    (long long)A.n[1] * A.n[2] * 2 * nc1 * NPAIR))
      cp_async_n(sU + u * NL1 * NPAIR, Ug + (((size_t)line * 2 + u) * nc1 + l1lo) * NPAIR, nl1 * NPAIR, tid, NT);
  stage_x<P, 3, XL>(A, line, a, T, sX);
  cp_async_wait_all();
  __syncthreads();
  rows_phase_b<P, 3, L::MAXPTS1, NL1, false, DO_M, DO_K, R, true>(A, sU, sV1, sB1, sE1, sOff1, sP, a, T, l1lo,
                                                                    base, sX);
}

template <int P, bool DO_M, bool DO_K, typename R>
__global__ void __launch_bounds__(32 * kRowsWarps, rows_min_blocks<R>()) apply_ug_kernel(const RowsArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  apply_ug_block<P, DO_M, DO_K, R>(A, blockIdx.x, smem_raw);
}

template <int P, bool DO_M, bool DO_K, typename R>
cudaError_t launch_apply_one(const RowsArgs &a, int nblocks, cudaStream_t s) {
  using L = ApplyLayoutUG<P, DO_M, DO_K, R>;
  auto kern = apply_ug_kernel<P, DO_M, DO_K, R>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nblocks <= 0) return cudaSuccess;
  kern<<<nblocks, 32 * kRowsWarps, L::BYTES, s>>>(a);
  return cudaGetLastError();
}

// y = M x and y = K x (do_k), or y = M x only (the load vector's form).
template <int P, typename R>
cudaError_t launch_apply_ug(bool do_k, const RowsArgs &a, int nblocks, cudaStream_t s) {
  if (do_k) return launch_apply_one<P, true, true, R>(a, nblocks, s);
  return launch_apply_one<P, true, false, R>(a, nblocks, s);
}

}  // namespace wq
