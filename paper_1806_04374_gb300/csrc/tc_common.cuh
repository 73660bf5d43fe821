// tc_common.cuh -- per-patch arithmetic shared by the tensor-core coders:
// steering-factor table access, the FP64 Cholesky state, the double-float
// exact re-score <S_r d_m, x> - sum_i a_i <S_r d_m, S_{r_i} d_{m_i}>, its FP32
// screen, the candidate list of block maxima, and the packed residual.
#pragma once

#include <cuda_fp16.h>
#include <math.h>

#include "df.cuh"
#include "rsc_internal.h"

namespace {

constexpr float kU32 = 5.9604644775390625e-8f;  // 2^-24

struct TwS {
  const float *base;
  int H, stride;
  __device__ df cosv(int k, int r) const {
    return {base[(0 * H + k) * stride + r], base[(1 * H + k) * stride + r]};
  }
  __device__ df sinv(int k, int r) const {
    return {base[(2 * H + k) * stride + r], base[(3 * H + k) * stride + r]};
  }
  __device__ float cos32(int k, int r) const { return base[(0 * H + k) * stride + r]; }
  __device__ float sin32(int k, int r) const { return base[(2 * H + k) * stride + r]; }
};

template <int KK>
struct Ls {
  double L[KK * (KK + 1) / 2];  // packed lower Cholesky factor
  double inv[KK];               // 1 / L_ii
  double z[KK];                 // L z = b
  double a[KK];                 // weights
  float ahi[KK], alo[KK];       // weights in double-float
  int m[KK], r[KK];             // selected atom / angle
};

__device__ __forceinline__ bool df_abs_gt(df a, df b) {
  if (a.hi < 0.0f) a = df_neg(a);
  if (b.hi < 0.0f) b = df_neg(b);
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

__device__ __forceinline__ bool df_abs_eq(df a, df b) {
  if (a.hi < 0.0f) a = df_neg(a);
  if (b.hi < 0.0f) b = df_neg(b);
  return a.hi == b.hi && a.lo == b.lo;
}

constexpr int kTop = kTcTop;  // candidates kept per list, patch and step

// Inserts (x, idx) into the descending list (v, i) of NT entries; disc
// keeps the largest value that did not stay in the list.  Strict comparisons
// keep the earlier entry first among equal values.
template <int NT>
__device__ __forceinline__ void topn_insert(float (&v)[NT], int (&i)[NT], float &disc, float x,
                                            int idx) {
  if (x > v[NT - 1]) {
    disc = fmaxf(disc, v[NT - 1]);
    v[NT - 1] = x;
    i[NT - 1] = idx;
#pragma unroll
    for (int q = NT - 1; q > 0; --q) {
      if (v[q] > v[q - 1]) {
        const float tf = v[q - 1];
        v[q - 1] = v[q];
        v[q] = tf;
        const int tn = i[q - 1];
        i[q - 1] = i[q];
        i[q] = tn;
      }
    }
  } else {
    disc = fmaxf(disc, x);
  }
}

// Dot2-style accumulation (Ogita, Rump, Oishi): s + c carries the sum.
__device__ __forceinline__ void dot2_acc(float &s, float &c, float x, float y) {
  df p = two_prod(x, y);
  df q = two_sum(s, p.hi);
  s = q.hi;
  c = __fadd_rn(c, __fadd_rn(p.lo, q.lo));
}

// <S_r d_m, x> in double-float: sum_k w_k Re(e^{ik theta} Q_k),
// Q_k = sum_j conj(d_m[j,k]) x[j,k].
__device__ df score_x(const float *__restrict__ dm, const float *__restrict__ xp, int J, int H,
                      int r, const TwS &tw) {
  df acc = df_make(0.0f);
  for (int k = 0; k < H; ++k) {
    float qr = 0.f, qrc = 0.f, qi = 0.f, qic = 0.f;
    const float2 *d2 = reinterpret_cast<const float2 *>(dm) + k * J;
    const float2 *x2 = reinterpret_cast<const float2 *>(xp) + k * J;
    for (int j = 0; j < J; ++j) {
      const float2 dv = __ldg(d2 + j);
      const float2 xv = __ldg(x2 + j);
      const float dim = k ? dv.y : 0.0f, xim = k ? xv.y : 0.0f;
      dot2_acc(qr, qrc, dv.x, xv.x);
      dot2_acc(qr, qrc, dim, xim);
      dot2_acc(qi, qic, dv.x, xim);
      dot2_acc(qi, qic, -dim, xv.x);
    }
    const df Qr = fast_two_sum(qr, qrc), Qi = fast_two_sum(qi, qic);
    // Re(e^{ik theta} Q) = cos(k theta) Re Q - sin(k theta) Im Q
    df term = df_sub(df_mul(tw.cosv(k, r), Qr), df_mul(tw.sinv(k, r), Qi));
    acc = df_add(acc, k ? df_mul_f(term, 2.0f) : term);
  }
  return acc;
}

// FP32 estimate of <S_r d_m, x> - sum_i a_i <S_r d_m, S_{r_i} d_{m_i}>, the
// candidate's score against the current residual (used to screen candidates
// before the exact re-score; its error is bounded by the caller).
template <int KK>
__device__ float score32(const float *__restrict__ dm, const float *__restrict__ xp,
                         const float4 *__restrict__ xg, int M, int J, int H, int R, int m, int r,
                         int t, const Ls<KK> &S, const TwS &tw) {
  float acc = 0.0f;
  for (int k = 0; k < H; ++k) {
    float qr = 0.f, qi = 0.f;
    const float2 *d2 = reinterpret_cast<const float2 *>(dm) + k * J;
    const float2 *x2 = reinterpret_cast<const float2 *>(xp) + k * J;
    for (int j = 0; j < J; ++j) {
      const float2 dv = __ldg(d2 + j), xv = __ldg(x2 + j);
      const float dim = k ? dv.y : 0.0f, xim = k ? xv.y : 0.0f;
      qr = fmaf(dv.x, xv.x, fmaf(dim, xim, qr));
      qi = fmaf(dv.x, xim, fmaf(-dim, xv.x, qi));
    }
    const float term = fmaf(tw.cos32(k, r), qr, -tw.sin32(k, r) * qi);
    acc = fmaf(k ? 2.0f : 1.0f, term, acc);
  }
#pragma unroll
  for (int i = 0; i < KK; ++i) {
    if (i < t) {
      int dr = r - S.r[i];
      if (dr < 0) dr += R;
      const float4 *h = xg + ((size_t)m * M + S.m[i]) * H;
      float g = 0.0f;
      for (int k = 0; k < H; ++k) {
        const float4 v = __ldg(h + k);
        const float term = fmaf(tw.cos32(k, dr), v.x, -tw.sin32(k, dr) * v.z);
        g = fmaf(k ? 2.0f : 1.0f, term, g);
      }
      acc = fmaf(-S.ahi[i], g, acc);
    }
  }
  return acc;
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// <S_ra d_ma, S_rb d_mb> = sum_k w_k Re(e^{ik (theta_a - theta_b)} H_k(ma, mb)).
__device__ df gram_entry(const float4 *__restrict__ xg, int M, int H, int R, int ma, int ra,
                         int mb, int rb, const TwS &tw) {
  int dr = ra - rb;
  if (dr < 0) dr += R;
  const float4 *h = xg + ((size_t)ma * M + mb) * H;
  df acc = df_make(0.0f);
  for (int k = 0; k < H; ++k) {
    const float4 v = __ldg(h + k);
    // the table row k already holds the angles k * 2 pi r / R
    df term = df_sub(df_mul(tw.cosv(k, dr), df{v.x, v.y}), df_mul(tw.sinv(k, dr), df{v.z, v.w}));
    acc = df_add(acc, k ? df_mul_f(term, 2.0f) : term);
  }
  return acc;
}

// Paired forms (even R): the same quantities for the two angles r and
// r + R/2 at once.  Half a turn multiplies harmonic k by (-1)^k (Eq. (Sr)), so
// with the even-k and odd-k parts of a sum, value(r) = even + odd and
// value(r + R/2) = even - odd.
struct DF2 {
  df a, b;
};

// score32 for (m, r) and (m, r + R/2): the even-k and odd-k parts E and O
// of the FP32 estimate give s(r) = E + O and s(r + R/2) = E - O.
template <int KK>
__device__ float2 score32_pair(const float *__restrict__ dm, const float *__restrict__ xp,
                               const float4 *__restrict__ xg, int M, int J, int H, int R, int m,
                               int r, int t, const Ls<KK> &S, const TwS &tw) {
  float ev = 0.0f, od = 0.0f;
  for (int k = 0; k < H; ++k) {
    float qr = 0.f, qi = 0.f;
    const float2 *d2 = reinterpret_cast<const float2 *>(dm) + k * J;
    const float2 *x2 = reinterpret_cast<const float2 *>(xp) + k * J;
    for (int j = 0; j < J; ++j) {
      const float2 dv = __ldg(d2 + j), xv = __ldg(x2 + j);
      const float dim = k ? dv.y : 0.0f, xim = k ? xv.y : 0.0f;
      qr = fmaf(dv.x, xv.x, fmaf(dim, xim, qr));
      qi = fmaf(dv.x, xim, fmaf(-dim, xv.x, qi));
    }
    const float term = fmaf(tw.cos32(k, r), qr, -tw.sin32(k, r) * qi);
    if (k & 1)
      od = fmaf(2.0f, term, od);
    else
      ev = fmaf(k ? 2.0f : 1.0f, term, ev);
  }
  float sa = ev + od, sb = ev - od;
#pragma unroll
  for (int i = 0; i < KK; ++i) {
    if (i < t) {
      int dr = r - S.r[i];
      if (dr < 0) dr += R;
      const float4 *h = xg + ((size_t)m * M + S.m[i]) * H;
      float ge = 0.0f, go = 0.0f;
      for (int k = 0; k < H; ++k) {
        const float4 v = __ldg(h + k);
        const float term = fmaf(tw.cos32(k, dr), v.x, -tw.sin32(k, dr) * v.z);
        if (k & 1)
          go = fmaf(2.0f, term, go);
        else
          ge = fmaf(k ? 2.0f : 1.0f, term, ge);
      }
      sa = fmaf(-S.ahi[i], ge + go, sa);
      sb = fmaf(-S.ahi[i], ge - go, sb);
    }
  }
  return make_float2(sa, sb);
}

// score_x for (m, r) and (m, r + R/2), double-float.
__device__ DF2 score_x_pair(const float *__restrict__ dm, const float *__restrict__ xp, int J,
                            int H, int r, const TwS &tw) {
  df ev = df_make(0.0f), od = df_make(0.0f);
  for (int k = 0; k < H; ++k) {
    float qr = 0.f, qrc = 0.f, qi = 0.f, qic = 0.f;
    const float2 *d2 = reinterpret_cast<const float2 *>(dm) + k * J;
    const float2 *x2 = reinterpret_cast<const float2 *>(xp) + k * J;
    for (int j = 0; j < J; ++j) {
      const float2 dv = __ldg(d2 + j);
      const float2 xv = __ldg(x2 + j);
      const float dim = k ? dv.y : 0.0f, xim = k ? xv.y : 0.0f;
      dot2_acc(qr, qrc, dv.x, xv.x);
      dot2_acc(qr, qrc, dim, xim);
      dot2_acc(qi, qic, dv.x, xim);
      dot2_acc(qi, qic, -dim, xv.x);
    }
    const df Qr = fast_two_sum(qr, qrc), Qi = fast_two_sum(qi, qic);
    const df term = df_sub(df_mul(tw.cosv(k, r), Qr), df_mul(tw.sinv(k, r), Qi));
    if (k & 1)
      od = df_add(od, df_mul_f(term, 2.0f));
    else
      ev = df_add(ev, k ? df_mul_f(term, 2.0f) : term);
  }
  return DF2{df_add(ev, od), df_sub(ev, od)};
}

// gram_entry for (ma, ra) and (ma, ra + R/2) against (mb, rb), double-float.
__device__ DF2 gram_entry_pair(const float4 *__restrict__ xg, int M, int H, int R, int ma, int ra,
                               int mb, int rb, const TwS &tw) {
  int dr = ra - rb;
  if (dr < 0) dr += R;
  const float4 *h = xg + ((size_t)ma * M + mb) * H;
  df ev = df_make(0.0f), od = df_make(0.0f);
  for (int k = 0; k < H; ++k) {
    const float4 v = __ldg(h + k);
    const df term =
        df_sub(df_mul(tw.cosv(k, dr), df{v.x, v.y}), df_mul(tw.sinv(k, dr), df{v.z, v.w}));
    if (k & 1)
      od = df_add(od, df_mul_f(term, 2.0f));
    else
      ev = df_add(ev, k ? df_mul_f(term, 2.0f) : term);
  }
  return DF2{df_add(ev, od), df_sub(ev, od)};
}

// New Cholesky row TT (compile-time) and the solve of all TT+1 weights, FP64.
template <int KK, int TT>
__device__ __forceinline__ bool chol_add(Ls<KK> &S, const double (&g)[KK], double diag,
                                         double rhs) {
  double l[TT > 0 ? TT : 1];
  double p2 = diag;
#pragma unroll
  for (int i = 0; i < TT; ++i) {
    double v = g[i];
#pragma unroll
    for (int j = 0; j < i; ++j) v -= S.L[i * (i + 1) / 2 + j] * l[j];
    v *= S.inv[i];
    l[i] = v;
    p2 -= v * v;
  }
  if (!(p2 > kPivotRel * diag)) return false;
  const double ltt = sqrt(p2);
#pragma unroll
  for (int i = 0; i < TT; ++i) S.L[TT * (TT + 1) / 2 + i] = l[i];
  S.L[TT * (TT + 1) / 2 + TT] = ltt;
  S.inv[TT] = 1.0 / ltt;
  double zt = rhs;
#pragma unroll
  for (int i = 0; i < TT; ++i) zt -= l[i] * S.z[i];
  S.z[TT] = zt * S.inv[TT];
#pragma unroll
  for (int i = TT; i >= 0; --i) {
    double v = S.z[i];
#pragma unroll
    for (int q = i + 1; q <= TT; ++q) v -= S.L[q * (q + 1) / 2 + i] * S.a[q];
    v *= S.inv[i];
    S.a[i] = v;
    const float hi = __double2float_rn(v);
    S.ahi[i] = hi;
    S.alo[i] = __double2float_rn(v - (double)hi);
  }
  return true;
}

template <int KK, int TT>
struct CholAt {
  __device__ static bool run(int t, Ls<KK> &S, const double (&g)[KK], double diag, double rhs) {
    if (t == TT) return chol_add<KK, TT>(S, g, diag, rhs);
    return CholAt<KK, TT + 1>::run(t, S, g, diag, rhs);
  }
};
template <int KK>
struct CholAt<KK, KK> {
  __device__ static bool run(int, Ls<KK> &, const double (&)[KK], double, double) {
    return false;
  }
};

// Produces this thread's packed residual x - sum_i a_i S_{r_i} d_{m_i} (FP32,
// times `scale`, rounded to fp16) as 16-byte chunks sink(chunk index, 8 fp16)
// in packed order, zero-padded to a multiple of 16 slots; returns ||r||^2
// (unscaled).
// Entries are visited in packed order; a k >= 1 entry yields its two slots
// (sqrt(2) Re, sqrt(2) Im) from one pass over the selected atoms.
template <int KK, class Sink>
__device__ float write_residual(Sink &&sink, float scale, const float *__restrict__ xp,
                                const float *__restrict__ d, int J, int HJ, int n, int t,
                                const Ls<KK> &S, const TwS &tw) {
  float n2 = 0.0f;
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int fill = 0, cq = 0;
  float cs[KK], sn[KK];
  int kcur = -1;
  auto flush = [&]() {
    uint4 pk;
    __half2 b0 = __floats2half2_rn(v[0] * scale, v[1] * scale);
    __half2 b1 = __floats2half2_rn(v[2] * scale, v[3] * scale);
    __half2 b2 = __floats2half2_rn(v[4] * scale, v[5] * scale);
    __half2 b3 = __floats2half2_rn(v[6] * scale, v[7] * scale);
    pk.x = *reinterpret_cast<uint32_t *>(&b0);
    pk.y = *reinterpret_cast<uint32_t *>(&b1);
    pk.z = *reinterpret_cast<uint32_t *>(&b2);
    pk.w = *reinterpret_cast<uint32_t *>(&b3);
    sink(cq, pk);
    ++cq;
    fill = 0;
  };
  auto push = [&](float val) {
    n2 = fmaf(val, val, n2);
    // registers cannot be indexed at run time: shift the value in
#pragma unroll
    for (int u = 0; u < 7; ++u) v[u] = v[u + 1];
    v[7] = val;
    if (++fill == 8) flush();
  };
  for (int e = 0; e < HJ; ++e) {
    const int k = e / J;
    if (k != kcur) {
      kcur = k;
#pragma unroll
      for (int i = 0; i < KK; ++i)
        if (i < t) {
          cs[i] = tw.cos32(k, S.r[i]);
          sn[i] = tw.sin32(k, S.r[i]);
        }
    }
    const float2 xv = __ldg(reinterpret_cast<const float2 *>(xp) + e);
    float re = xv.x, im = k ? xv.y : 0.0f;
#pragma unroll
    for (int i = 0; i < KK; ++i) {
      if (i < t) {
        const float2 dv = __ldg(reinterpret_cast<const float2 *>(d) + (size_t)S.m[i] * HJ + e);
        const float dim = k ? dv.y : 0.0f;
        re = fmaf(-S.ahi[i], fmaf(cs[i], dv.x, sn[i] * dim), re);
        im = fmaf(-S.ahi[i], fmaf(cs[i], dim, -sn[i] * dv.x), im);
      }
    }
    if (k == 0) {
      push(re);
    } else {
      push(re * 1.41421356237309515f);
      push(im * 1.41421356237309515f);
    }
  }
  // zero the rest of the contraction depth (slots n .. 16*ceil(n/16))
  const int total = ((n + 15) / 16) * 16;
  for (int q = n; q < total; ++q) push(0.0f);
  return n2;
}

}  // namespace
