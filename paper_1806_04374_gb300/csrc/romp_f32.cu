// romp_f32.cu -- rotational OMP with an FP32 CUDA-core scoring pass.
//
// One warp codes one patch at a time (persistent grid, warps stride over the
// patches).  Per greedy step (OMP of Sec. II-C on the augmented dictionary of
// Fig. "code", rotations by the steering matrix of Eq. (Sr)):
//   (a) per-harmonic contraction G_k(m) = sum_j conj(d_m[j,k]) r[j,k], one
//       lane per atom, FP32 FMA, the residual broadcast from shared memory;
//   (b) angle transform score(m, r) = G_0 + 2 Re sum_k e^{ik 2 pi r / R} G_k,
//       one lane per angle with its cos/sin factors held in registers; with
//       RSC_FP32_PRUNE only for the atoms whose exact bound |G_0| +
//       2 sum_k |G_k| >= max_r |score(m, r)| can still reach the window of
//       the running best;
//   (c) per-lane top-4 of |score| plus the largest discarded value, merged
//       over the warp into every candidate within 2E of the best, where E
//       bounds the FP32 error of a score; the candidates are re-scored in
//       double-float arithmetic against the double-float residual (if a lane
//       discarded a value inside the window, all M*R candidates are
//       re-scored exactly instead);
//   (e) new row of the Cholesky factor of the Gram matrix of the selected
//       steered atoms (entries and right-hand side in double-float, factor and
//       solve in FP64 on lane 0);
//   (d) residual x - sum_i a_i S_{r_i} d_{m_i} in double-float, its high part
//       feeding the next scoring pass.
#include <math.h>

#include "df.cuh"
#include "rsc_internal.h"

namespace {

constexpr int kChunk = 32;     // atoms per contraction chunk (g buffer rows)
constexpr int kCandCap = 128;  // candidates kept per step (4 per lane)

template <int KM>
struct GStride {
  static constexpr int v = ((2 * KM + 1) + 3) & ~3;  // floats per atom row of g
};

struct Layout {
  // block-level
  int tw_off, tw_stride;  // twiddles [4][H][tw_stride]
  int dT_off;             // transposed atoms [2][HJ][M] or -1 (read from global)
  // per-warp
  int warp_off, warp_bytes;
  int x_off, rhi_off, rlo_off, g_off, ub_off, cand_off, L_off, inv_off, z_off, a_off, adf_off,
      sel_off, gram_off;
  int acache_off;  // [K][HJ] float4: steered selected atoms (re hi, re lo, im hi, im lo)
  int total;
};

__host__ __device__ inline int align16(int v) { return (v + 15) & ~15; }

template <int KM>
__host__ __device__ inline Layout make_layout(int M, int J, int H, int R, int K, int warps,
                                              bool dT_in_smem) {
  Layout L;
  const int HJ = H * J;
  int off = 0;
  L.tw_stride = R + 1;
  L.tw_off = off;
  off = align16(off + 4 * H * L.tw_stride * 4);
  L.dT_off = dT_in_smem ? off : -1;
  if (dT_in_smem) off = align16(off + 2 * HJ * M * 4);
  L.warp_off = off;
  int w = 0;
  L.x_off = w;    w = align16(w + 2 * HJ * 4);
  L.rhi_off = w;  w = align16(w + 2 * HJ * 4);
  L.rlo_off = w;  w = align16(w + 2 * HJ * 4);
  L.g_off = w;    w = align16(w + kChunk * GStride<KM>::v * 4);
  L.ub_off = w;   w = align16(w + kChunk * 4);
  L.cand_off = w; w = align16(w + kCandCap * 4);
  L.L_off = w;    w = align16(w + K * (K + 1) / 2 * 8);
  L.inv_off = w;  w = align16(w + K * 8);
  L.z_off = w;    w = align16(w + K * 8);
  L.a_off = w;    w = align16(w + K * 8);
  L.adf_off = w;  w = align16(w + 2 * K * 4);
  L.sel_off = w;  w = align16(w + K * 4);
  L.gram_off = w; w = align16(w + (2 * K + 2) * 8);
  L.acache_off = w; w = align16(w + K * HJ * 16);
  L.warp_bytes = w;
  L.total = off + warps * w;
  return L;
}

struct Tw {
  const float *base;
  int H, stride;
  __device__ df cosv(int k, int r) const {
    return {base[(0 * H + k) * stride + r], base[(1 * H + k) * stride + r]};
  }
  __device__ df sinv(int k, int r) const {
    return {base[(2 * H + k) * stride + r], base[(3 * H + k) * stride + r]};
  }
};

struct Cdf {
  df re, im;
};

// Entry e = k*J + j of the steered atom S_{2 pi r / R} d_m in double-float:
// e^{-ik theta} (dre + i dim) = (c dre + s dim) + i (c dim - s dre).
__device__ __forceinline__ Cdf steered_entry(const float *__restrict__ d, int HJ, int k, int m,
                                             int r, int e, const Tw &tw) {
  float2 dv = __ldg(reinterpret_cast<const float2 *>(d) + (size_t)m * HJ + e);
  float dim = (k == 0) ? 0.0f : dv.y;
  df c = tw.cosv(k, r), s = tw.sinv(k, r);
  Cdf out;
  out.re = df_add(df_mul_f(c, dv.x), df_mul_f(s, dim));
  out.im = df_sub(df_mul_f(c, dim), df_mul_f(s, dv.x));
  return out;
}

// |a| > |b| for normalised double-float values.
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

// Inserts (v, idx) into the descending top-4 (v, i); disc keeps the largest
// value that did not stay in the top-4.  Strict comparisons keep the earlier
// (smaller) flat index first among equal values.
__device__ __forceinline__ void top4_insert(float (&v)[4], int (&i)[4], float &disc, float x,
                                            int idx) {
  if (x > v[3]) {
    disc = fmaxf(disc, v[3]);
    v[3] = x;
    i[3] = idx;
    if (v[3] > v[2]) { float t = v[2]; v[2] = v[3]; v[3] = t; int u = i[2]; i[2] = i[3]; i[3] = u; }
    if (v[2] > v[1]) { float t = v[1]; v[1] = v[2]; v[2] = t; int u = i[1]; i[1] = i[2]; i[2] = u; }
    if (v[1] > v[0]) { float t = v[0]; v[0] = v[1]; v[1] = t; int u = i[0]; i[0] = i[1]; i[1] = u; }
  } else {
    disc = fmaxf(disc, x);
  }
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float4 cdf_pack(const Cdf &a) {
  return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo);
}

__device__ __forceinline__ Cdf cdf_unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }

template <int KM, int RPL, bool PRUNE>
__global__ void __launch_bounds__(256)
    romp_f32_kernel(RompArgs a, int dT_in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int GS = GStride<KM>::v;
  const int M = a.M, J = a.J, H = a.H, R = a.R, K = a.K, kmax = a.kmax;
  const int HJ = H * J;
  const int warps = blockDim.x >> 5;
  const Layout Lo = make_layout<KM>(M, J, H, R, K, warps, dT_in_smem != 0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // hand-off mode launches the whole persistent grid for a list whose length
  // only the device knows (a few patches): a block with no patch of the list
  // leaves before loading its tables (the whole block, before any barrier)
  if (a.redo_list && (int64_t)blockIdx.x * warps >= (int64_t)*a.redo_count) return;

  // ---- block setup: twiddles (padded stride) and transposed atoms
  float *s_tw = reinterpret_cast<float *>(smem + Lo.tw_off);
  for (int i = threadIdx.x; i < 4 * H * R; i += blockDim.x) {
    int plane_k = i / R, r = i - plane_k * R;
    s_tw[plane_k * Lo.tw_stride + r] = a.tw[i];
  }
  const float *dT = a.dT;
  if (dT_in_smem) {
    float *s_dT = reinterpret_cast<float *>(smem + Lo.dT_off);
    for (int i = threadIdx.x; i < 2 * HJ * M; i += blockDim.x) s_dT[i] = a.dT[i];
    dT = s_dT;
  }
  __syncthreads();
  const Tw tw{s_tw, H, Lo.tw_stride};

  unsigned char *wbase = smem + Lo.warp_off + warp * Lo.warp_bytes;
  float *s_x = reinterpret_cast<float *>(wbase + Lo.x_off);
  float *s_rhi = reinterpret_cast<float *>(wbase + Lo.rhi_off);
  float *s_rlo = reinterpret_cast<float *>(wbase + Lo.rlo_off);
  float *s_g = reinterpret_cast<float *>(wbase + Lo.g_off);
  float *s_ub = reinterpret_cast<float *>(wbase + Lo.ub_off);
  int *s_cand = reinterpret_cast<int *>(wbase + Lo.cand_off);
  double *s_L = reinterpret_cast<double *>(wbase + Lo.L_off);
  double *s_inv = reinterpret_cast<double *>(wbase + Lo.inv_off);  // 1 / L_ii
  double *s_z = reinterpret_cast<double *>(wbase + Lo.z_off);
  double *s_a = reinterpret_cast<double *>(wbase + Lo.a_off);
  float *s_adf = reinterpret_cast<float *>(wbase + Lo.adf_off);
  int *s_sel = reinterpret_cast<int *>(wbase + Lo.sel_off);
  double *s_gram = reinterpret_cast<double *>(wbase + Lo.gram_off);
  float4 *s_A = reinterpret_cast<float4 *>(wbase + Lo.acache_off);

  // FP32 angle factors of this lane's angles r = lane + 32 i, harmonics 1..KM
  float tc[RPL][KM], ts[RPL][KM];
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    int r = lane + 32 * i;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      bool ok = (r < R) && (k + 1 <= kmax);
      tc[i][k] = ok ? tw.cosv(k + 1, r).hi : 0.0f;
      ts[i][k] = ok ? tw.sinv(k + 1, r).hi : 0.0f;
    }
  }

  // FP32 error bound of one score per unit residual norm.  With u = 2^-24:
  // each G_k component carries <= gamma_2J sum_j |d_jk||r_jk|, the rounded
  // residual and cos/sin factors add u each, and the 2 kmax + 1 term FMA chain
  // of (b) adds gamma_{2kmax+1}; summed with the weights 1, 2 and bounded by
  // Cauchy-Schwarz (unit atoms) this is <= (4J + 4 kmax + 5) u ||r||.  The
  // factor 4 and the +8 are headroom.
  const float err_per_norm = 4.0f * (4.0f * J + 4.0f * kmax + 8.0f) * 5.9604644775390625e-8f;

  const int64_t nwarps = (int64_t)gridDim.x * warps;
  for (int64_t it = (int64_t)blockIdx.x * warps + warp;; it += nwarps) {
    int64_t p;
    if (a.redo_list) {
      if (it >= *a.redo_count) break;
      p = a.redo_list[it];
    } else {
      if (it >= a.P) break;
      p = it;
    }
    const float *xp = a.x + p * (int64_t)(2 * HJ);
    // ---- load the patch; residual = x
    df acc = df_make(0.0f);
    for (int e = lane; e < HJ; e += 32) {
      float2 v = *reinterpret_cast<const float2 *>(xp + 2 * e);
      const bool k0 = e < J;
      if (k0) v.y = 0.0f;
      s_x[2 * e] = v.x;
      s_x[2 * e + 1] = v.y;
      s_rhi[2 * e] = v.x;
      s_rhi[2 * e + 1] = v.y;
      s_rlo[2 * e] = 0.0f;
      s_rlo[2 * e + 1] = 0.0f;
      df q = df_add(two_prod(v.x, v.x), two_prod(v.y, v.y));
      acc = df_add(acc, k0 ? q : df_mul_f(q, 2.0f));
    }
    acc = df_warp_sum(acc);
    const float xnorm = sqrtf(fmaxf(acc.hi + acc.lo, 0.0f));
    const float stop_level = (float)kStopRel * xnorm;
    float rnorm = xnorm;
    __syncwarp();

    // steps already certified elsewhere are taken as given (no scoring)
    int t0 = 0;
    if (a.resume_sI) t0 = min(a.resume_sI[(int64_t)2 * a.resume_cap * a.resume_P + p], K);
    int t = 0;
    for (int step = 0; step < K; ++step) {
      int best_c = -1;
      if (step < t0) {
        best_c = a.resume_sI[(int64_t)step * a.resume_P + p] * R +
                 a.resume_sI[(int64_t)(a.resume_cap + step) * a.resume_P + p];
      } else {
        // ---- (a)+(b)+(c): FP32 scores, per-lane top-4
        float tv[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        int ti[4] = {-1, -1, -1, -1};
        float disc = -INFINITY;
        const float win2 = 2.0f * err_per_norm * rnorm;
        for (int mc = 0; mc < M; mc += kChunk) {
          const int mend = min(kChunk, M - mc);
          // (a) one lane per atom: G_k = sum_j conj(d[j,k]) r[j,k]
          for (int ml = lane; ml < mend; ml += 32) {
            const int m = mc + ml;
            float gv[GS];
#pragma unroll
            for (int q = 0; q < GS; ++q) gv[q] = 0.0f;
            const float *pre = dT + m;
            const float *pim = dT + (size_t)HJ * M + m;
            const float2 *r2 = reinterpret_cast<const float2 *>(s_rhi);
            int e = 0;
#pragma unroll
            for (int k = 0; k <= KM; ++k) {
              if (k < H) {
                float gre0 = 0.f, gre1 = 0.f, gim0 = 0.f, gim1 = 0.f;
                for (int j = 0; j < J; ++j, ++e) {
                  const float dre = pre[(size_t)e * M], dim = pim[(size_t)e * M];
                  const float2 rv = r2[e];
                  gre0 = fmaf(dre, rv.x, gre0);
                  gre1 = fmaf(dim, rv.y, gre1);
                  gim0 = fmaf(dre, rv.y, gim0);
                  gim1 = fmaf(-dim, rv.x, gim1);
                }
                if (k == 0) {
                  gv[0] = gre0 + gre1;
                } else {
                  gv[2 * k - 1] = 2.0f * (gre0 + gre1);
                  gv[2 * k] = -2.0f * (gim0 + gim1);
                }
              }
            }
            float4 *g4 = reinterpret_cast<float4 *>(s_g + ml * GS);
#pragma unroll
            for (int q = 0; q < GS / 4; ++q)
              g4[q] = make_float4(gv[4 * q], gv[4 * q + 1], gv[4 * q + 2], gv[4 * q + 3]);
            if constexpr (PRUNE) {
              // |score(m, r)| <= |G_0| + 2 sum_k |G_k| for every angle
              // (triangle inequality; gv holds G_0 and 2 Re / -2 Im of G_k),
              // times a slack covering the FP32 rounding of this sum and of
              // the transform below, so every FP32 score of the atom is <= ub
              float ub = fabsf(gv[0]);
#pragma unroll
              for (int k = 1; k <= KM; ++k)
                if (k <= kmax) ub += sqrtf(fmaf(gv[2 * k - 1], gv[2 * k - 1], gv[2 * k] * gv[2 * k]));
              s_ub[ml] = ub * (1.0f + 16.0f * (KM + 2) * 5.9604644775390625e-8f);
            }
          }
          __syncwarp();
          // (b) one lane per angle, (c) per-lane top-4
          auto transform = [&](int ml) {
            const float4 *g4 = reinterpret_cast<const float4 *>(s_g + ml * GS);
            float gv[GS];
#pragma unroll
            for (int q = 0; q < GS / 4; ++q) {
              float4 v = g4[q];
              gv[4 * q] = v.x;
              gv[4 * q + 1] = v.y;
              gv[4 * q + 2] = v.z;
              gv[4 * q + 3] = v.w;
            }
#pragma unroll
            for (int i = 0; i < RPL; ++i) {
              float sa = gv[0], sb = 0.0f;
#pragma unroll
              for (int k = 0; k < KM; ++k) {
                sa = fmaf(gv[2 * k + 1], tc[i][k], sa);
                sb = fmaf(gv[2 * k + 2], ts[i][k], sb);
              }
              const int r = lane + 32 * i;
              const float v = fabsf(sa + sb);
              // a value more than 2E below this lane's running best is below
              // the final window and need not be kept (the best only grows)
              if (r < R && !(v < tv[0] - win2)) top4_insert(tv, ti, disc, v, (mc + ml) * R + r);
            }
          };
          if constexpr (!PRUNE) {
            for (int ml = 0; ml < mend; ++ml) transform(ml);
          } else {
            // In index order, an atom whose bound is below the warp's running
            // best minus the window 2E (refreshed every 8 atoms; a stale best
            // is lower, so only more atoms are transformed) is skipped: every
            // FP32 score of it is below best - 2E <= the final threshold
            // s1 - 2E (the best only grows), so none of them could be a
            // candidate or raise a lane's discarded value to the threshold;
            // the best atom is never skipped (its bound is >= its score).
            // Measured at M = 64, R = 64, K = 5 (400,000 patches): with the
            // chunk's largest-bound atom first the bound rules out 52% of the
            // transforms, yet that loop takes 1.55x the plain loop's time and
            // this one 1.3x; the same loop transforming every atom takes
            // 1.06x.  The plain loop's unbroken run of short FMA chains
            // pipelines better than any loop with a data-dependent skip.
            float wbest = -INFINITY;
            for (int ml = 0; ml < mend; ++ml) {
              if ((ml & 7) == 0) wbest = warp_max(tv[0]);
              if (s_ub[ml] < wbest - win2) continue;
              transform(ml);
            }
          }
          __syncwarp();
        }
        const float s1 = warp_max(tv[0]);
        const float E = err_per_norm * rnorm;
        if (s1 + E <= stop_level) break;  // every exact score is below the stop level
        const float thr = s1 - 2.0f * E;
        const bool overflow = __any_sync(0xffffffffu, disc >= thr);

        // ---- candidates, re-scored in double-float against the exact residual
        int ncand = 0;
        if (!overflow) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const bool f = (tv[q] >= thr) && (ti[q] >= 0);
            const unsigned b = __ballot_sync(0xffffffffu, f);
            if (f) s_cand[ncand + __popc(b & ((1u << lane) - 1u))] = ti[q];
            ncand += __popc(b);
          }
        } else {
          if (lane == 0 && a.fallbacks) atomicAdd(a.fallbacks, 1ull);
          ncand = M * R;
        }
        __syncwarp();
        df best_v = df_make(0.0f);
        for (int ci = 0; ci < ncand; ++ci) {
          const int c = overflow ? ci : s_cand[ci];
          const int m = c / R, r = c - m * R;
          df s = df_make(0.0f);
          for (int e = lane; e < HJ; e += 32) {
            const int k = e / J;
            Cdf A = steered_entry(a.d, HJ, k, m, r, e, tw);
            df rr = {s_rhi[2 * e], s_rlo[2 * e]};
            df ri = {s_rhi[2 * e + 1], s_rlo[2 * e + 1]};
            df q = df_add(df_mul(A.re, rr), df_mul(A.im, ri));
            s = df_add(s, k ? df_mul_f(q, 2.0f) : q);
          }
          s = df_warp_sum(s);
          if (best_c < 0 || df_abs_gt(s, best_v) || (df_abs_eq(s, best_v) && c < best_c)) {
            best_v = s;
            best_c = c;
          }
        }
        if (best_c < 0 || !(fabsf(best_v.hi) > stop_level)) break;
      }

      // ---- (e) new steered atom (cached), its Gram row, diagonal, right-hand side
      const int mn = best_c / R, rn = best_c - mn * R;
      {
        df sd = df_make(0.0f), sb = df_make(0.0f);
        for (int e = lane; e < HJ; e += 32) {
          const int k = e / J;
          Cdf A = steered_entry(a.d, HJ, k, mn, rn, e, tw);
          s_A[t * HJ + e] = cdf_pack(A);
          df qd = df_add(df_mul(A.re, A.re), df_mul(A.im, A.im));
          df qb = df_add(df_mul_f(A.re, s_x[2 * e]), df_mul_f(A.im, s_x[2 * e + 1]));
          sd = df_add(sd, k ? df_mul_f(qd, 2.0f) : qd);
          sb = df_add(sb, k ? df_mul_f(qb, 2.0f) : qb);
        }
        sd = df_warp_sum(sd);
        sb = df_warp_sum(sb);
        if (lane == 0) {
          s_gram[t] = df_to_d(sd);
          s_gram[t + 1] = df_to_d(sb);
        }
      }
      __syncwarp();
      for (int i = 0; i < t; ++i) {
        df s = df_make(0.0f);
        for (int e = lane; e < HJ; e += 32) {
          const Cdf A = cdf_unpack(s_A[t * HJ + e]);
          const Cdf B = cdf_unpack(s_A[i * HJ + e]);
          df q = df_add(df_mul(A.re, B.re), df_mul(A.im, B.im));
          s = df_add(s, (e >= J) ? df_mul_f(q, 2.0f) : q);
        }
        s = df_warp_sum(s);
        if (lane == 0) s_gram[K + 1 + i] = df_to_d(s);  // Gram row, after diag/rhs slots
      }
      __syncwarp();
      int ok = 0;
      if (lane == 0) {
        // new row t of L (packed lower triangle, row i starts at i(i+1)/2); FP64
        const double diag = s_gram[t], rhs = s_gram[t + 1];
        double *Lt = s_L + t * (t + 1) / 2;
        double p2 = diag;
        for (int i = 0; i < t; ++i) {
          const double *Li = s_L + i * (i + 1) / 2;
          double v = s_gram[K + 1 + i];
          for (int j = 0; j < i; ++j) v -= Li[j] * Lt[j];
          v *= s_inv[i];
          Lt[i] = v;
          p2 -= v * v;
        }
        if (p2 > kPivotRel * diag) {
          ok = 1;
          const double ltt = sqrt(p2);
          Lt[t] = ltt;
          s_inv[t] = 1.0 / ltt;
          double zt = rhs;
          for (int i = 0; i < t; ++i) zt -= Lt[i] * s_z[i];
          s_z[t] = zt * s_inv[t];
          // back substitution L^T a = z over the t+1 selected atoms
          for (int i = t; i >= 0; --i) {
            double v = s_z[i];
            for (int q = i + 1; q <= t; ++q) v -= s_L[q * (q + 1) / 2 + i] * s_a[q];
            v *= s_inv[i];
            s_a[i] = v;
            const float hi = __double2float_rn(v);
            s_adf[2 * i] = hi;
            s_adf[2 * i + 1] = __double2float_rn(v - (double)hi);
          }
          s_sel[t] = best_c;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();
      if (!ok) break;
      ++t;

      // ---- (d) residual x - sum_i a_i S_{r_i} d_{m_i} (double-float)
      df nacc = df_make(0.0f);
      for (int e = lane; e < HJ; e += 32) {
        df rr = df_make(s_x[2 * e]);
        df ri = df_make(s_x[2 * e + 1]);
        for (int i = 0; i < t; ++i) {
          const Cdf A = cdf_unpack(s_A[i * HJ + e]);
          const df ai = {s_adf[2 * i], s_adf[2 * i + 1]};
          rr = df_sub(rr, df_mul(ai, A.re));
          ri = df_sub(ri, df_mul(ai, A.im));
        }
        const bool k0 = e < J;
        if (k0) ri = df_make(0.0f);
        s_rhi[2 * e] = rr.hi;
        s_rlo[2 * e] = rr.lo;
        s_rhi[2 * e + 1] = ri.hi;
        s_rlo[2 * e + 1] = ri.lo;
        df q = df_add(df_mul(rr, rr), df_mul(ri, ri));
        nacc = df_add(nacc, k0 ? q : df_mul_f(q, 2.0f));
      }
      nacc = df_warp_sum(nacc);
      rnorm = sqrtf(fmaxf(nacc.hi + nacc.lo, 0.0f));
      __syncwarp();
    }

    // ---- outputs
    for (int i = lane; i < K; i += 32) {
      const int64_t o = p * K + i;
      if (i < t) {
        const int c = s_sel[i];
        const int m = c / R, r = c - m * R;
        a.atom[o] = m;
        a.angle_idx[o] = r;
        if (a.angle) a.angle[o] = (float)(6.283185307179586 * r / R);
        a.coef[o] = s_a[i];
      } else {
        a.atom[o] = -1;
        a.angle_idx[o] = -1;
        if (a.angle) a.angle[o] = 0.0f;
        a.coef[o] = 0.0;
      }
    }
    if (lane == 0 && a.resid_norm2) a.resid_norm2[p] = rnorm * rnorm;
    __syncwarp();
  }
}

template <int KM, int RPL, bool PRUNE>
int launch_p(const RompArgs &a, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  int max_optin = 0, nsm = 0;
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int HJ = a.H * a.J;
  bool dT_smem = (size_t)2 * HJ * a.M * 4 <= 64 * 1024;
  int warps = 8;
  Layout L = make_layout<KM>(a.M, a.J, a.H, a.R, a.K, warps, dT_smem);
  while (L.total > max_optin && warps > 1) {
    warps >>= 1;
    L = make_layout<KM>(a.M, a.J, a.H, a.R, a.K, warps, dT_smem);
  }
  if (L.total > max_optin && dT_smem) {
    dT_smem = false;
    warps = 8;
    L = make_layout<KM>(a.M, a.J, a.H, a.R, a.K, warps, false);
    while (L.total > max_optin && warps > 1) {
      warps >>= 1;
      L = make_layout<KM>(a.M, a.J, a.H, a.R, a.K, warps, false);
    }
  }
  if (L.total > max_optin) return RSC_ERR_UNSUPPORTED;
  auto kern = romp_f32_kernel<KM, RPL, PRUNE>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, L.total);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (per_sm < 1) return RSC_ERR_UNSUPPORTED;
  int64_t grid = (int64_t)nsm * per_sm;
  if (!a.redo_list) {
    const int64_t need = (a.P + warps - 1) / warps;
    if (need < grid) grid = need;
  }
  kern<<<(unsigned)grid, warps * 32, L.total, stream>>>(a, dT_smem ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return RSC_OK;
}

template <int KM, int RPL>
int launch_t(const RompArgs &a, cudaStream_t stream) {
  return a.prune ? launch_p<KM, RPL, true>(a, stream) : launch_p<KM, RPL, false>(a, stream);
}

}  // namespace

int rsc_launch_f32(const RompArgs &a, cudaStream_t stream) {
  if (a.P == 0) return RSC_OK;
  const int rpl = (a.R + 31) / 32;
  if (a.kmax <= 8) {
    if (rpl == 1) return launch_t<8, 1>(a, stream);
    if (rpl == 2) return launch_t<8, 2>(a, stream);
    if (rpl <= 4) return launch_t<8, 4>(a, stream);
  } else if (a.kmax <= 12) {
    if (rpl <= 2) return launch_t<12, 2>(a, stream);
    if (rpl <= 4) return launch_t<12, 4>(a, stream);
  } else if (a.kmax <= 16) {
    if (rpl <= 2) return launch_t<16, 2>(a, stream);
  }
  return RSC_ERR_UNSUPPORTED;
}
