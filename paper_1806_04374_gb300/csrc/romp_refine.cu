// romp_refine.cu -- per-patch steps of the FP16 path between scoring passes:
// candidate certification, exact re-scoring, the least-squares update and the
// residual (steps (c)-(e) of OMP, Sec. II-C), one thread per patch.
//
// romp_init_kernel writes each patch's packed residual (= x) in fp16 for the
// first scoring pass and initialises its state.  Rows are scaled by a power
// of two chosen from a bound on their norm (rsc_internal.h), so that scores
// come back as 2^(16 - e) times their true value.  romp_refine_kernel then,
// after every scoring pass (romp_score.cu):
//   * certifies the scoring pass's candidates (per column slice: kept blocks
//     of 32 rows and a mask of columns): E bounds the fp16 error of a score
//     (rounding of both operands, accumulation, and the FP32 residual's own
//     error); every row with |score| >= s1 - 2E is row b + u of a kept block
//     b and a masked column u, unless a slice's bound on what it left out
//     (disc) is >= s1 - 2E, in which case the patch is handed to the FP32
//     path;
//   * re-scores those rows exactly in double-float as
//     <A_c, x> - sum_i a_i <A_c, A_i> (ties: smallest m*R + r): the slice's
//     best row first, the others (K <= 5) only when their FP32 score plus its
//     error bound reaches the exact best;
//   * adds the Cholesky row of the winner (Gram entries and right-hand side
//     in double-float, factor and solve in FP64) and writes the new residual
//     row; after the last step the reported residual norm comes from the
//     factor instead (||x||^2 - z^T z, L z = b).
// Per-patch state lives in HBM as structure-of-arrays (coalesced over
// threads); stopped and finished patches write their outputs.
#include "rsc_internal.h"
#include "tc_common.cuh"

namespace {


// State arrays (each of length P, element i of patch p at [field * P + p]).
template <int KK>
struct StateIdx {
  static constexpr int nL = KK * (KK + 1) / 2;
  // doubles: L, inv, z, a
  static constexpr int dL = 0, dInv = nL, dZ = nL + KK, dA = nL + 2 * KK, nD = nL + 3 * KK;
  // floats: ahi, alo, xnorm, rnorm, dr, ||x||^2 in double-float (hi, lo)
  static constexpr int fHi = 0, fLo = KK, fX = 2 * KK, fR = 2 * KK + 1, fDr = 2 * KK + 2,
                       fX2h = 2 * KK + 3, fX2l = 2 * KK + 4, nF = 2 * KK + 5;
  // ints: m, r, t, e (exponent of the current row's scale)
  static constexpr int iM = 0, iR = KK, iT = 2 * KK, iE = 2 * KK + 1, nI = 2 * KK + 2;
};

// The selection state (atoms, angles, weights, norms) is loaded when a patch
// starts; the FP64 factor only right before the Cholesky update, so that it
// does not hold registers through the scoring code.
template <int KK>
__device__ __forceinline__ void load_state(const RefineArgs &a, int64_t p, Ls<KK> &S, int &t,
                                           int &e, float &xnorm, float &rnorm, float &dr) {
  using I = StateIdx<KK>;
  const int64_t P = a.P;
  t = a.sI[I::iT * P + p];
  e = a.sI[I::iE * P + p];
#pragma unroll
  for (int i = 0; i < KK; ++i) {
    S.ahi[i] = a.sF[(I::fHi + i) * P + p];
    S.alo[i] = a.sF[(I::fLo + i) * P + p];
    S.m[i] = a.sI[(I::iM + i) * P + p];
    S.r[i] = a.sI[(I::iR + i) * P + p];
  }
  xnorm = a.sF[I::fX * P + p];
  rnorm = a.sF[I::fR * P + p];
  dr = a.sF[I::fDr * P + p];
}

template <int KK>
__device__ __forceinline__ void load_factor(const RefineArgs &a, int64_t p, Ls<KK> &S) {
  using I = StateIdx<KK>;
  const int64_t P = a.P;
#pragma unroll
  for (int q = 0; q < I::nL; ++q) S.L[q] = a.sD[(I::dL + q) * P + p];
#pragma unroll
  for (int i = 0; i < KK; ++i) {
    S.inv[i] = a.sD[(I::dInv + i) * P + p];
    S.z[i] = a.sD[(I::dZ + i) * P + p];
    S.a[i] = a.sD[(I::dA + i) * P + p];
  }
}

template <int KK>
__device__ __forceinline__ void store_state(const RefineArgs &a, int64_t p, const Ls<KK> &S, int t,
                                            int e, float rnorm, float dr) {
  using I = StateIdx<KK>;
  const int64_t P = a.P;
  a.sI[I::iT * P + p] = t;
  a.sI[I::iE * P + p] = e;
#pragma unroll
  for (int q = 0; q < I::nL; ++q) a.sD[(I::dL + q) * P + p] = S.L[q];
#pragma unroll
  for (int i = 0; i < KK; ++i) {
    a.sD[(I::dInv + i) * P + p] = S.inv[i];
    a.sD[(I::dZ + i) * P + p] = S.z[i];
    a.sD[(I::dA + i) * P + p] = S.a[i];
    a.sF[(I::fHi + i) * P + p] = S.ahi[i];
    a.sF[(I::fLo + i) * P + p] = S.alo[i];
    a.sI[(I::iM + i) * P + p] = S.m[i];
    a.sI[(I::iR + i) * P + p] = S.r[i];
  }
  a.sF[I::fR * P + p] = rnorm;
  a.sF[I::fDr * P + p] = dr;
}

template <int KK>
__device__ void write_outputs(const RefineArgs &a, int64_t p, const Ls<KK> &S, int t,
                              float rnorm) {
  const int K = a.K;
#pragma unroll
  for (int i = 0; i < KK; ++i) {
    if (i < K) {
      const int64_t o = p * K + i;
      if (i < t) {
        a.atom[o] = S.m[i];
        a.angle_idx[o] = S.r[i];
        if (a.angle) a.angle[o] = (float)(6.283185307179586 * S.r[i] / a.R);
        a.coef[o] = S.a[i];
      } else {
        a.atom[o] = -1;
        a.angle_idx[o] = -1;
        if (a.angle) a.angle[o] = 0.0f;
        a.coef[o] = 0.0;
      }
    }
  }
  if (a.resid_norm2) a.resid_norm2[p] = rnorm * rnorm;
}

// Shared memory of the init/refine kernels: the steering-factor table
// [4][H][R], then the packed-slot table qtab[q] = rsc_slot_code (slot q holds
// Re (c = 0) or Im (c = 1) of entry e = k*J + j, or zero for -1) of the
// plain or paired row layout.
__device__ __forceinline__ TwS load_tw(const RefineArgs &a, const int *&qtab) {
  extern __shared__ __align__(16) float tws[];
  const int n = 4 * a.H * a.R;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = a.tw[i];
  int *qt = reinterpret_cast<int *>(tws + ((n + 3) & ~3));
  for (int q = threadIdx.x; q < a.L; q += blockDim.x)
    qt[q] = rsc_slot_code(q, a.J, a.kmax, a.paired != 0);
  __syncthreads();
  qtab = qt;
  return TwS{tws, a.H, a.R};
}

// Packed residual x - sum_i a_i S_{r_i} d_{m_i} of this thread's patch (FP32)
// written times `scale` as fp16 (L slots, zero-padded) to `row` if not
// null, slot by slot in packed order; the Im slot of an entry reuses the value
// computed with its Re slot.  Returns ||r||^2 (unscaled).
template <int KK>
__device__ __forceinline__ float residual_q(uint4 *row, int L, float scale,
                                            const float *__restrict__ xp,
                                            const float *__restrict__ d, int HJ, int t,
                                            const Ls<KK> &S, const TwS &tw, const int *qtab) {
  float n2 = 0.0f, pend = 0.0f;
#pragma unroll 1
  for (int cq = 0; cq < L / 8; ++cq) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int code = qtab[cq * 8 + u];
      float val = 0.0f;
      if (code >= 0) {
        const int e = code >> 8, k = (code >> 1) & 127;
        if (code & 1) {
          val = pend;
        } else {
          const float2 xv = __ldg(reinterpret_cast<const float2 *>(xp) + e);
          float re = xv.x, im = k ? xv.y : 0.0f;
#pragma unroll
          for (int i = 0; i < KK; ++i) {
            if (i < t) {
              const float2 dv =
                  __ldg(reinterpret_cast<const float2 *>(d) + (size_t)S.m[i] * HJ + e);
              const float dim = k ? dv.y : 0.0f;
              const float c = tw.cos32(k, S.r[i]), sn = tw.sin32(k, S.r[i]);
              re = fmaf(-S.ahi[i], fmaf(c, dv.x, sn * dim), re);
              im = fmaf(-S.ahi[i], fmaf(c, dim, -sn * dv.x), im);
            }
          }
          if (k) {
            re *= 1.41421356237309515f;
            pend = im * 1.41421356237309515f;
          }
          val = re;
        }
        n2 = fmaf(val, val, n2);
      }
      v[u] = val;
    }
    if (row) {
      uint4 pk;
      __half2 b0 = __floats2half2_rn(v[0] * scale, v[1] * scale);
      __half2 b1 = __floats2half2_rn(v[2] * scale, v[3] * scale);
      __half2 b2 = __floats2half2_rn(v[4] * scale, v[5] * scale);
      __half2 b3 = __floats2half2_rn(v[6] * scale, v[7] * scale);
      pk.x = *reinterpret_cast<uint32_t *>(&b0);
      pk.y = *reinterpret_cast<uint32_t *>(&b1);
      pk.z = *reinterpret_cast<uint32_t *>(&b2);
      pk.w = *reinterpret_cast<uint32_t *>(&b3);
      row[cq] = pk;
    }
  }
  return n2;
}

// Error bound of one fp16 score of a row of L slots, times 1.25, without the
// key term: 2^-10 ||r|| (both operands rounded, unit atoms) + 2^-18 ||r||
// (second order) + L 2^-21 ||r|| (the accumulation, at 4x unit roundoff) +
// s 2^-33 ||r|| and s 2^(e-33) (subnormal rounding of a dictionary entry,
// <= 2^-25 / kDictScale, and of a row entry, <= 2^-25 / row scale, over
// sqrt(L) <= s entries: s = 11 for 112 slots, 16 for 256); plus the FP32
// residual's own error 2 dr.
__device__ __forceinline__ float score_err_base(float rnorm, float dr, int e, int L) {
  const float sq = L <= kTcKst ? 11.0f : 16.0f;
  return 1.25f * (9.765625e-4f + 3.814697265625e-6f + (float)L * 4.76837158203125e-7f +
                  sq * 1.16415321826934814e-10f) *
             rnorm +
         1.25f * sq * ldexpf(1.0f, e - 33) + 2.0f * dr;
}

// The scoring pass's window for a row: 2.02 E in accumulator units
// (2^(16 - e) times true scores), with the key term 2^-16 s1 bounded through
// s1 <= 1.01 ||r|| (Cauchy-Schwarz over unit atoms plus the score error).
__device__ __forceinline__ float score_window(float rnorm, float dr, int e, int L) {
  return 2.02f * (score_err_base(rnorm, dr, e, L) + 1.52587890625e-5f * 1.01f * rnorm) *
         ldexpf(1.0f, 16 - e);
}

template <int KK>
__global__ void __launch_bounds__(128) romp_init_kernel(const RefineArgs a) {
  using I = StateIdx<KK>;
  const int H = a.H, J = a.J, HJ = H * J;
  const int *qtab;
  const TwS tw = load_tw(a, qtab);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float *xp = a.x + p * (int64_t)(2 * HJ);
    df acc = df_make(0.0f);
    for (int e = 0; e < HJ; ++e) {
      float2 v = __ldg(reinterpret_cast<const float2 *>(xp) + e);
      if (e < J) v.y = 0.0f;
      df q = df_add(two_prod(v.x, v.x), two_prod(v.y, v.y));
      acc = df_add(acc, e < J ? q : df_mul_f(q, 2.0f));
    }
    const float xnorm = sqrtf(fmaxf(acc.hi + acc.lo, 0.0f));
    Ls<KK> S;
    const int e = rsc_row_exponent(xnorm);
    const float rn = sqrtf(residual_q<KK>(reinterpret_cast<uint4 *>(a.A + p * (a.L * 2)), a.L,
                                          ldexpf(1.0f, kRowLog2 - e), xp, a.d, HJ, 0, S, tw,
                                          qtab));
    a.sI[I::iT * a.P + p] = 0;
    a.sI[I::iE * a.P + p] = e;
    a.sF[I::fX * a.P + p] = xnorm;
    a.sF[I::fX2h * a.P + p] = acc.hi;
    a.sF[I::fX2l * a.P + p] = acc.lo;
    a.sF[I::fR * a.P + p] = rn;
    a.sF[I::fDr * a.P + p] = 2.0f * kU32 * xnorm;
    a.win[p] = score_window(rn, 2.0f * kU32 * xnorm, e, a.L);
    a.status[p] = 1;
  }
}

// Register budget: 5 blocks of 128 threads per SM (<= 102 registers) up to
// K = 5; for K = 8 the state (Cholesky row, weights, Gram entries of up to 8
// atoms) spills 1.8 KB a thread at that budget.  Measured on the 21 x 21-patch
// image workload: 4 blocks (<= 128 registers, 0.8 KB of spills) 1.9% faster
// than 3 (<= 168) and 4% faster than 2 (no spills).
//
// Two passes per step: a thread re-scores every unit of its patch in one loop,
// so a warp runs that loop max(units per lane) times.  Nearly all patches have
// one unit in the window, but among 32 lanes one with several is common, so
// the first pass (PASS = 1) finishes only the patches with one unit and
// appends the others to a list, which the second pass (PASS = 2) finishes with
// every lane on a patch that needs the loop.
template <int KK, bool PAIRED, int PASS>
__global__ void __launch_bounds__(128, KK > 5 ? 4 : 5) romp_refine_kernel(const RefineArgs a) {
  const int H = a.H, J = a.J, R = a.R, M = a.M, HJ = H * J;
  const int *qtab;
  const TwS tw = load_tw(a, qtab);
  const int64_t nwork = PASS == 2 ? (int64_t)*a.slow_count : a.P;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwork;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = PASS == 2 ? (int64_t)a.slow_list[w] : w;
    if (a.status[p] <= 0) continue;
    const float *xp = a.x + p * (int64_t)(2 * HJ);
    // the patch's row is read by the re-scoring and the residual writer:
    // start bringing its cache lines into L1 before the state loads
    // (measured 2.5% on omp_1m)
    {
      const uintptr_t b0 = reinterpret_cast<uintptr_t>(xp) & ~(uintptr_t)127;
      const uintptr_t b1 = reinterpret_cast<uintptr_t>(xp + 2 * HJ - 1);
      for (uintptr_t q = b0; q <= b1; q += 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(q));
    }
    Ls<KK> S;
    int t, e;
    float xnorm, rnorm, dr;
    load_state<KK>(a, p, S, t, e, xnorm, rnorm, dr);
    // accumulator scores are 2^(16 - e) times the true scores
    const float unscale = ldexpf(1.0f, e - 16);
    // the scoring pass's lists of kept blocks (one per column slice of each
    // chunk, each sorted by block maximum in descending order): their heads
    // give the best value; the entries are read again by the re-scoring loop
    // below
    static_assert(kTcTop == 4, "slots read as float4 / int4 per slice");
    const float *cvp = a.cand_val + p * kTcCand;
    const int *cip = a.cand_idx + p * kTcCand;
    float discm = -INFINITY, head = -INFINITY;
#pragma unroll
    for (int sl = 0; sl < kTcSplit; ++sl) {
      discm = fmaxf(discm, a.cand_disc[kTcSplit * p + sl]);
      head = fmaxf(head, cvp[kTcTop * sl]);
    }
    const float disc = discm * unscale;
    const float stop_level = 1e-10f * xnorm;
    const float s1 = head * unscale;
    // fp16 error of a score (score_err_base) plus a spare 2^-16 s1
    const float E = score_err_base(rnorm, dr, e, a.L) + 1.52587890625e-5f * fabsf(s1);
    int outcome = 0;  // 0 continue, 1 finished/stopped, 2 hand-off
    bool have_factor = false;
    if (!(s1 + E > stop_level)) {
      outcome = 1;
    } else {
      const float thr = s1 - 2.0f * E;
      if (disc >= thr) {
        outcome = 2;
      } else {
        // a candidate unit is one steered atom (row r*M + m), or in the
        // paired layout the two angles r and r + R/2 of atom m (row r*M + m,
        // r < R/2, scored by max(|s(r)|, |s(r + R/2)|)).  Every unit in the
        // certified window is row b + u of a kept block b (slot q) whose
        // maximum reaches the window and a column u in its slice's class mask;
        // the best slice's best unit (the block with the largest maximum and
        // that slice's best column) is re-scored exactly first.
        constexpr int NP = PAIRED ? 2 : 1;
        const int Rh = R / 2;
        const int MR = PAIRED ? M * Rh : M * R;
        df best = df_make(0.0f), best_ax = df_make(0.0f);
        df bg[KK];
#pragma unroll
        for (int i = 0; i < KK; ++i) bg[i] = df_make(0.0f);
        int bm = -1, br = 0, bflat = 0;
        // the kept blocks inside the window as a bit mask (slot q = slice q / 4);
        // the loop below runs over (block, column) pairs, so that a warp runs
        // the re-scoring body max(units per lane) times
        unsigned bmask = 0;
        int qf = -1;  // the block with the largest maximum
        // column mask and best column of slice sl
        unsigned umk[kTcSplit], ubk[kTcSplit];
#pragma unroll
        for (int sl = 0; sl < kTcSplit; ++sl) {
          const uint2 v = *reinterpret_cast<const uint2 *>(a.cand_mask + 2 * (kTcSplit * p + sl));
          umk[sl] = v.x;
          ubk[sl] = v.y;
        }
        auto umask_of = [&](int sl) {
          unsigned r = umk[0];
#pragma unroll
          for (int i = 1; i < kTcSplit; ++i) r = sl == i ? umk[i] : r;
          return r;
        };
        auto ubest_of = [&](int sl) {
          unsigned r = ubk[0];
#pragma unroll
          for (int i = 1; i < kTcSplit; ++i) r = sl == i ? ubk[i] : r;
          return (int)r;
        };
        {
          float vbest = -1.0f;
#pragma unroll
          for (int sl = 0; sl < kTcSplit; ++sl) {
            const int4 iq = *reinterpret_cast<const int4 *>(cip + kTcTop * sl);
            const float4 vq = *reinterpret_cast<const float4 *>(cvp + kTcTop * sl);
            const int iv[kTcTop] = {iq.x, iq.y, iq.z, iq.w};
            const float vv[kTcTop] = {vq.x, vq.y, vq.z, vq.w};
#pragma unroll
            for (int j = 0; j < kTcTop; ++j)
              if (iv[j] >= 0 && vv[j] * unscale >= thr) {
                bmask |= 1u << (sl * kTcTop + j);
                if (vv[j] > vbest) {
                  vbest = vv[j];
                  qf = sl * kTcTop + j;
                }
              }
          }
        }
        // (the masks' columns are < 32 by construction; the best column is
        // masked too, so that candidates left undefined by a scoring pass that
        // gave up cannot name a row outside the table)
        const int uf = qf < 0 ? 0 : (ubest_of(qf / kTcTop) & 31);
        if (PASS == 1) {
          // units in the window: columns of the masks over the kept blocks
          int nunits = 0;
#pragma unroll
          for (int q = 0; q < kTcCand; ++q)
            if (bmask & (1u << q)) nunits += __popc(umask_of(q / kTcTop));
          if (nunits > 1) {
            a.slow_list[atomicAdd(a.slow_count, 1)] = (int)p;
            continue;
          }
        }
        // The other units are first scored in FP32 and re-scored exactly only
        // if they can reach the exact best so far.  Error of the FP32 score:
        // each per-harmonic dot product of J complex entries and the angle
        // transform over H harmonics round at most 2J + 2H + 8 times, on
        // terms bounded by ||x|| (unit atoms, Cauchy-Schwarz) and by |a_i| for
        // the Gram terms, and the weights carry only their hi part; x4 margin.
        // (only the second pass runs more than one unit; at K = 8 the screen
        // is built into that pass alone: 2.55 -> 2.18 ms per refine launch on
        // the 21 x 21 image sizes, where windows hold many units)
        constexpr bool kScreen = KK <= 5 || PASS == 2;
        float asum = 0.0f;
#pragma unroll
        for (int i = 0; i < KK; ++i)
          if (i < t) asum += fabsf(S.ahi[i]) + fabsf(S.alo[i]);
        const float E32 = 4.0f * (float)(2 * J + 2 * H + 8) * kU32 * (xnorm + asum) + asum * kU32;
        // unit iterator: (q, u) starts at the half's best unit; the rest of
        // its block's columns, then the other kept blocks' columns follow, so a
        // lane with one unit runs the body once
        int q = qf, u = qf < 0 ? 0 : uf;
        unsigned uleft = qf < 0 ? 0u : (umask_of(qf / kTcTop) & ~(1u << uf));
        unsigned bleft = qf < 0 ? 0u : (bmask & ~(1u << qf));
        bool more = qf >= 0, first = true;
#pragma unroll 1
        while (more) {
          const int id = cip[q] + u;
          bool go = cip[q] >= 0 && cip[q] < MR && id < MR;
          const int m = id % M, r = id / M;
          if (PASS != 1 && kScreen && go && !first) {
            float f;
            if (PAIRED) {
              const float2 f2 = score32_pair<KK>(a.d + (size_t)m * HJ * 2, xp, a.xgram, M, J, H,
                                                 R, m, r, t, S, tw);
              f = fmaxf(fabsf(f2.x), fabsf(f2.y));
            } else {
              f = fabsf(score32<KK>(a.d + (size_t)m * HJ * 2, xp, a.xgram, M, J, H, R, m, r, t, S,
                                    tw));
            }
            // cannot reach (or tie) the best: |best| >= |best.hi| (1 - 2^-22)
            go = !(f + E32 < fabsf(best.hi) * 0.99999976f);
          }
          first = false;
          if (go) {
            df ax[NP], sc[NP], gq[NP][KK];
            if (PAIRED) {
              const DF2 x2 = score_x_pair(a.d + (size_t)m * HJ * 2, xp, J, H, r, tw);
              ax[0] = x2.a;
              ax[NP - 1] = x2.b;
            } else {
              ax[0] = score_x(a.d + (size_t)m * HJ * 2, xp, J, H, r, tw);
            }
#pragma unroll
            for (int h = 0; h < NP; ++h) sc[h] = ax[h];
#pragma unroll
            for (int i = 0; i < KK; ++i) {
#pragma unroll
              for (int h = 0; h < NP; ++h) gq[h][i] = df_make(0.0f);
              if (i < t) {
                if (PAIRED) {
                  const DF2 g2 = gram_entry_pair(a.xgram, M, H, R, m, r, S.m[i], S.r[i], tw);
                  gq[0][i] = g2.a;
                  gq[NP - 1][i] = g2.b;
                } else {
                  gq[0][i] = gram_entry(a.xgram, M, H, R, m, r, S.m[i], S.r[i], tw);
                }
#pragma unroll
                for (int h = 0; h < NP; ++h)
                  sc[h] = df_sub(sc[h], df_mul(df{S.ahi[i], S.alo[i]}, gq[h][i]));
              }
            }
#pragma unroll
            for (int h = 0; h < NP; ++h) {
              const int rr = r + h * Rh, flat = m * R + rr;
              if (bm < 0 || df_abs_gt(sc[h], best) || (df_abs_eq(sc[h], best) && flat < bflat)) {
                best = sc[h];
                bm = m;
                br = rr;
                bflat = flat;
                best_ax = ax[h];
#pragma unroll
                for (int i = 0; i < KK; ++i) bg[i] = gq[h][i];
              }
            }
          }
          if (PASS == 1) break;  // the first pass keeps one-unit patches only
          // next unit: the next column of this block, else the first column
          // of the next kept block with a non-empty mask
          while (uleft == 0 && bleft != 0) {
            q = __ffs(bleft) - 1;
            bleft &= bleft - 1;
            uleft = umask_of(q / kTcTop);
          }
          more = uleft != 0;
          if (more) {
            u = __ffs(uleft) - 1;
            uleft &= uleft - 1;
          }
        }
        if (bm < 0 || !(fabsf(best.hi) > stop_level)) {
          outcome = 1;
        } else {
          const int mb = bm, rb = br;
          double gr[KK];
#pragma unroll
          for (int i = 0; i < KK; ++i) gr[i] = (i < t) ? df_to_d(bg[i]) : 0.0;
          // <S_r d_m, S_r d_m> = ||d_m||^2: steering preserves the norm
          const double diag = (double)a.anorm[mb].x + (double)a.anorm[mb].y;
          const double rhs = df_to_d(best_ax);
          load_factor<KK>(a, p, S);
          have_factor = true;
          if (!CholAt<KK, 0>::run(t, S, gr, diag, rhs)) {
            outcome = 1;
          } else {
#pragma unroll
            for (int i = 0; i < KK; ++i)
              if (i == t) {
                S.m[i] = mb;
                S.r[i] = rb;
              }
            ++t;
            float asum = 0.0f;
#pragma unroll
            for (int i = 0; i < KK; ++i)
              if (i < t) asum += fabsf(S.ahi[i]);
            dr = 2.0f * (t + 6) * kU32 * (xnorm + 1.5f * asum);
            if (t >= a.K) {
              outcome = 1;
              // final residual norm from the least-squares solution: with
              // L z = b (b_i = <A_i, x>, the factor of the Gram of the
              // selected steered atoms), ||x - sum_i a_i A_i||^2 =
              // ||x||^2 - z^T z, in FP64 from ||x||^2 in double-float (no
              // residual is formed: the fp16 row is not needed any more)
              double zz = 0.0;
#pragma unroll
              for (int i = 0; i < KK; ++i)
                if (i < t) zz = fma(S.z[i], S.z[i], zz);
              const double x2 = (double)a.sF[StateIdx<KK>::fX2h * a.P + p] +
                                (double)a.sF[StateIdx<KK>::fX2l * a.P + p];
              rnorm = (float)sqrt(fmax(x2 - zz, 0.0));
            } else {
              // the previous residual's norm bounds the new one (least squares
              // over a larger support)
              const int en = rsc_row_exponent(rnorm);
              rnorm = sqrtf(residual_q<KK>(reinterpret_cast<uint4 *>(a.A + p * (a.L * 2)), a.L,
                                           ldexpf(1.0f, kRowLog2 - en), xp, a.d, HJ, t, S,
                                           tw, qtab));
              store_state<KK>(a, p, S, t, en, rnorm, dr);
              a.win[p] = score_window(rnorm, dr, en, a.L);
            }
          }
        }
      }
    }
    if (outcome == 1) {
      if (!have_factor) {
#pragma unroll
        for (int i = 0; i < KK; ++i)
          if (i < t) S.a[i] = a.sD[(StateIdx<KK>::dA + i) * a.P + p];
      }
      write_outputs<KK>(a, p, S, t, rnorm);
      a.status[p] = 0;
    } else if (outcome == 2) {
      const int slot = atomicAdd(a.redo_count, 1);
      a.redo_list[slot] = (int)p;
      if (a.fallbacks) atomicAdd(a.fallbacks, 1ull);
      a.status[p] = -1;
    }
  }
}

template <int KK>
int launch_refine_t(const RefineArgs &a, bool init, cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = (a.P + 127) / 128;
  const int64_t cap = (int64_t)nsm * (a.blocks_per_sm > 0 ? a.blocks_per_sm : 32);
  const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
  const size_t shm = (size_t)((4 * a.H * a.R + 3) & ~3) * 4 + (size_t)a.L * 4;
  if (init) {
    romp_init_kernel<KK><<<grid, 128, shm, stream>>>(a);
  } else {
    e = cudaMemsetAsync(a.slow_count, 0, sizeof(int), stream);
    if (e != cudaSuccess) return rsc_cuda_fail(e);
    // the second pass's list holds a few percent of the patches: a grid of
    // 4 blocks per SM walks it
    const unsigned grid2 = (unsigned)(grid < (unsigned)(nsm * 4) ? grid : (unsigned)(nsm * 4));
    if (a.paired) {
      romp_refine_kernel<KK, true, 1><<<grid, 128, shm, stream>>>(a);
      romp_refine_kernel<KK, true, 2><<<grid2, 128, shm, stream>>>(a);
    } else {
      romp_refine_kernel<KK, false, 1><<<grid, 128, shm, stream>>>(a);
      romp_refine_kernel<KK, false, 2><<<grid2, 128, shm, stream>>>(a);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return RSC_OK;
}

}  // namespace

namespace {
template <int KK>
int state_layout_t(int *nD, int *nF, int *nI) {
  *nD = StateIdx<KK>::nD;
  *nF = StateIdx<KK>::nF;
  *nI = StateIdx<KK>::nI;
  return KK;
}
}  // namespace

int rsc_state_layout(int K, int *nD, int *nF, int *nI) {
  if (K <= 3) return state_layout_t<3>(nD, nF, nI);
  if (K <= 5) return state_layout_t<5>(nD, nF, nI);
  return state_layout_t<8>(nD, nF, nI);
}

int rsc_launch_refine(const RefineArgs &a, bool init, cudaStream_t stream) {
  if (a.P == 0) return RSC_OK;
  if (a.K <= 3) return launch_refine_t<3>(a, init, stream);
  if (a.K <= 5) return launch_refine_t<5>(a, init, stream);
  if (a.K <= 8) return launch_refine_t<8>(a, init, stream);
  return RSC_ERR_UNSUPPORTED;
}
