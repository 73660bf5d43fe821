// romp_tc.cu -- rotational OMP with a BF16 tensor-core (tcgen05) scoring pass.
//
// The scores of one greedy step, score(p, m, r) = <S_r d_m, r_p> (OMP of
// Sec. II-C over the augmented dictionary of Fig. "code"), are steps (a) and
// (b) of the method: the per-harmonic contraction G_k = sum_j conj(d) r and
// the angle transform sum_k e^{ik 2 pi r/R} G_k.  Both are linear, so their
// product is one dense contraction of the packed residual with the steered
// dictionary [S_0 D ... S_{R-1} D] (built once per dictionary by the host in
// FP64 and stored in bf16).  This kernel runs that contraction on the 5th
// generation tensor cores:
//
//   * a CTA owns TILES tiles of 128 patches; a tile's packed residuals are
//     the A operand (bf16, 128 x 112, 128-byte swizzled K-major in shared
//     memory) and every TMEM lane holds one patch;
//   * the steered dictionary streams through a ring of shared-memory stages
//     in chunks of 128 steered atoms, loaded by TMA (one thread issues the
//     loads and the MMAs); each chunk is multiplied into one of two TMEM
//     accumulator buffers per tile while the other buffer is read back;
//   * epilogue (c): every thread reads its patch's scores with tcgen05.ld and
//     keeps the top-4 |score| and the largest value it discarded;
//   * per patch, every candidate within 2E of the best (E bounds the bf16
//     error of a score) is re-scored exactly in double-float as
//     <A_c, x> - sum_i a_i <A_c, A_i>, the Gram entries coming from the
//     per-harmonic cross-Gram table; if the window holds more candidates
//     than were kept, the patch is handed to the FP32 path instead;
//   * (e) the Gram row and right-hand side of the winner in double-float,
//     the Cholesky row and solve in FP64, per thread;
//   * (d) the new residual in FP32, rounded to bf16 into the A tile.
#include <cuda_bf16.h>
#include <math.h>

#include "df.cuh"
#include "rsc_internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int kTile = 128;
constexpr int kStages = 3;
constexpr int kBlkA = kTile * 128;    // one 64-column block of A (bytes)
constexpr int kBlkB = kTcBN * 128;    // one 64-column block of a B stage (bytes)
constexpr int kStageBytes = 2 * kBlkB;
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits: 2 s
constexpr float kU32 = 5.9604644775390625e-8f;  // 2^-24

struct TcLayout {
  int a_off, b_off, tw_off, qtab_off, bar_off, misc_off, total;
};

__host__ __device__ inline int al(int v, int a) { return (v + a - 1) / a * a; }

template <int TILES>
__host__ __device__ inline TcLayout tc_layout(int H, int R) {
  TcLayout L;
  int off = 0;
  L.a_off = off;
  off += TILES * 2 * kBlkA;
  L.b_off = off;
  off += kStages * kStageBytes;
  L.tw_off = off;
  off = al(off + 4 * H * (R + 1) * 4, 16);
  L.qtab_off = off;
  off = al(off + kTcMaxN * 4, 16);
  L.bar_off = off;
  off = al(off + (kStages + 2) * 8, 16);
  L.misc_off = off;
  off += 16;
  L.total = off + 1024;  // slack for the 1024-byte alignment of the base
  return L;
}

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

// Writes this thread's packed residual x - sum_i a_i S_{r_i} d_{m_i} (FP32,
// rounded to bf16) into row `row` of the swizzled A tile; returns ||r||^2.
template <int KK>
__device__ float write_residual(unsigned char *sA, int row, const float *__restrict__ xp,
                                const float *__restrict__ d, int HJ, int n, int t,
                                const Ls<KK> &S, const int *qtab, const TwS &tw) {
  float n2 = 0.0f;
#pragma unroll 1
  for (int cq = 0; cq < kTcKst / 8; ++cq) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = cq * 8 + u;
      float val = 0.0f;
      if (q < n) {
        const int code = qtab[q];
        const int e = code >> 8, k = (code >> 1) & 127, comp = code & 1;
        val = xp[2 * e + comp];
#pragma unroll
        for (int i = 0; i < KK; ++i) {
          if (i < t) {
            const float2 dv = __ldg(reinterpret_cast<const float2 *>(d) + (size_t)S.m[i] * HJ + e);
            const float c = tw.cos32(k, S.r[i]), s = tw.sin32(k, S.r[i]);
            const float Ac = comp ? fmaf(c, dv.y, -s * dv.x) : fmaf(c, dv.x, s * dv.y);
            val = fmaf(-S.ahi[i], Ac, val);
          }
        }
        if (k) val *= 1.41421356237309515f;
      }
      v[u] = val;
      n2 = fmaf(val, val, n2);
    }
    uint4 pk;
    __nv_bfloat162 b0 = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 b1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 b2 = __floats2bfloat162_rn(v[4], v[5]);
    __nv_bfloat162 b3 = __floats2bfloat162_rn(v[6], v[7]);
    pk.x = *reinterpret_cast<uint32_t *>(&b0);
    pk.y = *reinterpret_cast<uint32_t *>(&b1);
    pk.z = *reinterpret_cast<uint32_t *>(&b2);
    pk.w = *reinterpret_cast<uint32_t *>(&b3);
    const int blk = cq >> 3, ch = cq & 7;
    *reinterpret_cast<uint4 *>(sA + blk * kBlkA + row * 128 + ((ch ^ (row & 7)) << 4)) = pk;
  }
  return n2;
}

__device__ __forceinline__ void record_error(int *err, int code) {
  if (err) atomicCAS(err, 0, code);
}

template <int TILES, int KK>
__global__ void __launch_bounds__(TILES * 128, 1)
    romp_tc_kernel(const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int H = a.H, J = a.J, R = a.R, M = a.M, K = a.K, HJ = H * J;
  const TcLayout Lo = tc_layout<TILES>(H, R);
  unsigned char *sA = smem + Lo.a_off;
  unsigned char *sB = smem + Lo.b_off;
  float *s_tw = reinterpret_cast<float *>(smem + Lo.tw_off);
  int *s_qtab = reinterpret_cast<int *>(smem + Lo.qtab_off);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lo.bar_off);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + Lo.misc_off);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile_id = tid >> 7, row = tid & 127;
  const uint32_t full_bar0 = tc::smem_u32(bars);
  const uint32_t done_bar0 = tc::smem_u32(bars + kStages);
  constexpr uint32_t kCols = TILES * 2 * kTcBN;
  constexpr uint32_t kIdesc = tc::idesc_bf16_f32(128, kTcBN);

  // ---- set-up: tables, barriers, TMEM
  for (int i = tid; i < 4 * H * R; i += blockDim.x) {
    const int pk = i / R, r = i - pk * R;
    s_tw[pk * (R + 1) + r] = a.tw[i];
  }
  for (int q = tid; q < kTcMaxN; q += blockDim.x) {
    int code = 0;
    if (q < a.n) {
      int e, k, comp;
      if (q < J) {
        e = q; k = 0; comp = 0;
      } else {
        const int qq = q - J, kj = qq >> 1;
        comp = qq & 1;
        k = 1 + kj / J;
        e = k * J + (kj - (k - 1) * J);
      }
      code = (e << 8) | (k << 1) | comp;
    }
    s_qtab[q] = code;
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) tc::mbar_init(full_bar0 + 8 * s, 1);
    for (int b = 0; b < 2; ++b) tc::mbar_init(done_bar0 + 8 * b, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;
  const TwS tw{s_tw, H, R + 1};

  // producer / MMA state, meaningful in thread 0 only
  uint32_t g = 0;              // global chunk counter (MMA order)
  uint32_t tma_next = 0;       // next chunk to load
  uint32_t mma_issued = 0;     // chunks whose MMAs were issued
  uint32_t mma_waited = 0;     // chunks whose completion was observed by thread 0

  auto issue_tma = [&](uint32_t gg) {
    const int s = gg % kStages;
    const int chunk = gg % a.nchunks;
    const uint32_t bar = full_bar0 + 8 * s;
    const uint32_t dst = tc::smem_u32(sB + s * kStageBytes);
    tc::mbar_arrive_expect_tx(bar, kStageBytes);
    tc::tma_load_2d(dst, &tmB, bar, 0, chunk * kTcBN);
    tc::tma_load_2d(dst + kBlkB, &tmB, bar, 64, chunk * kTcBN);
  };
  auto issue_mma = [&](uint32_t gg) -> bool {
    const int s = gg % kStages;
    if (!tc::mbar_wait_bounded(full_bar0 + 8 * s, (gg / kStages) & 1, kWaitNs)) return false;
    tc::fence_after_sync();
    const uint32_t buf = gg & 1;
    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB + s * kStageBytes);
#pragma unroll
    for (int tl = 0; tl < TILES; ++tl) {
      const uint32_t d = tmem + (uint32_t)(tl * 2 + buf) * kTcBN;
      for (int ks = 0; ks < a.ksteps; ++ks) {
        const uint32_t off = (ks >> 2) * kBlkA + (ks & 3) * 32;
        const uint32_t boff = (ks >> 2) * kBlkB + (ks & 3) * 32;
        tc::mma_bf16(d, tc::smem_desc_sw128(a0 + tl * 2 * kBlkA + off),
                     tc::smem_desc_sw128(b0 + boff), kIdesc, ks > 0 ? 1u : 0u);
      }
    }
    tc::mma_commit(done_bar0 + 8 * buf);
    mma_issued = gg + 1;
    return true;
  };

  if (tid == 0) {
    for (; tma_next < (uint32_t)kStages; ++tma_next) issue_tma(tma_next);
  }

  const int64_t ngroups = (a.P + (int64_t)TILES * kTile - 1) / ((int64_t)TILES * kTile);
  bool aborted = false;
  for (int64_t grp = blockIdx.x; grp < ngroups && !aborted; grp += gridDim.x) {
    const int64_t p = (grp * TILES + tile_id) * kTile + row;
    const bool valid = p < a.P;
    unsigned char *myA = sA + tile_id * 2 * kBlkA;
    const float *xp = a.x + (valid ? p : 0) * (int64_t)(2 * HJ);
    Ls<KK> S;
    int t = 0;
    bool active = valid, redo = false;
    float xnorm = 0.0f, rnorm = 0.0f, dr = 0.0f;
    if (valid) {
      df acc = df_make(0.0f);
      for (int e = 0; e < HJ; ++e) {
        float2 v = __ldg(reinterpret_cast<const float2 *>(xp) + e);
        if (e < J) v.y = 0.0f;
        df q = df_add(two_prod(v.x, v.x), two_prod(v.y, v.y));
        acc = df_add(acc, e < J ? q : df_mul_f(q, 2.0f));
      }
      xnorm = sqrtf(fmaxf(acc.hi + acc.lo, 0.0f));
      rnorm = sqrtf(write_residual<KK>(myA, row, xp, a.d, HJ, a.n, 0, S, s_qtab, tw));
      dr = 2.0f * kU32 * xnorm;
    } else {
      // rows of absent patches: zeros
      for (int cq = 0; cq < kTcKst / 8; ++cq) {
        const int blk = cq >> 3, ch = cq & 7;
        *reinterpret_cast<uint4 *>(myA + blk * kBlkA + row * 128 + ((ch ^ (row & 7)) << 4)) =
            make_uint4(0, 0, 0, 0);
      }
    }
    const float stop_level = 1e-10f * xnorm;

    for (int step = 0; step < K; ++step) {
      tc::fence_proxy_async_smem();
      const int any = __syncthreads_or(active ? 1 : 0);
      if (!any) break;
      // ---- scoring: MMAs chunk by chunk, epilogue keeps the per-patch top-4
      float tv[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
      int ti[4] = {-1, -1, -1, -1};
      float disc = -INFINITY;
      for (int c = 0; c < a.nchunks; ++c) {
        const uint32_t gg = g + c;
        int fail = 0;
        if (tid == 0) {
          bool ok = true;
          if (c == 0) ok = issue_mma(gg);
          if (ok && c + 1 < a.nchunks) ok = issue_mma(gg + 1);
          if (!ok) fail = 1;
        }
        // completion of chunk gg (every thread observes the barrier)
        bool done = false;
        if (!fail) done = tc::mbar_wait_bounded(done_bar0 + 8 * (gg & 1), (gg >> 1) & 1, kWaitNs);
        if (!done) {
          fail = 1;
          record_error(a.err, RSC_ERR_TIMEOUT);
        }
        tc::fence_after_sync();
        if (tid == 0 && done) {
          mma_waited = gg + 1;
          // stage gg % kStages is free again: prefetch chunk gg + kStages
          issue_tma(tma_next);
          ++tma_next;
        }
        // tcgen05.ld is warp-collective: a warp reads back only if none of its
        // threads saw a failed wait
        if (!__any_sync(0xffffffffu, fail)) {
          const uint32_t col0 = (uint32_t)(tile_id * 2 + (gg & 1)) * kTcBN;
          const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + col0;
          const int nvalid = min(kTcBN, a.MR - c * kTcBN);
#pragma unroll 1
          for (int piece = 0; piece < kTcBN / 32; ++piece) {
            uint32_t v[32];
            tc::tmem_ld32(taddr + piece * 32, v);
            tc::tmem_wait_ld();
            if (active) {
              const int base = c * kTcBN + piece * 32;
              if ((piece + 1) * 32 <= nvalid) {
                float mx = 0.0f;
#pragma unroll
                for (int u = 0; u < 32; ++u) mx = fmaxf(mx, fabsf(__uint_as_float(v[u])));
                if (mx > tv[3]) {
#pragma unroll
                  for (int u = 0; u < 32; ++u)
                    top4_insert(tv, ti, disc, fabsf(__uint_as_float(v[u])), base + u);
                } else {
                  disc = fmaxf(disc, mx);
                }
              } else {
#pragma unroll
                for (int u = 0; u < 32; ++u)
                  if (piece * 32 + u < nvalid)
                    top4_insert(tv, ti, disc, fabsf(__uint_as_float(v[u])), base + u);
              }
            }
          }
        }
        tc::fence_before_sync();
        // one CTA-wide decision: a failed wait anywhere ends the kernel
        if (__syncthreads_or(fail)) {
          aborted = true;
          break;
        }
      }
      g += a.nchunks;
      if (aborted) break;

      // ---- per patch: certify, re-score, least squares, residual
      if (active) {
        const float s1 = tv[0];
        const float E = 1.25f * (3.90625e-3f + 3.814697265625e-6f + 112.0f * 4.76837158203125e-7f) *
                            rnorm + 2.0f * dr;
        if (!(s1 + E > stop_level)) {
          active = false;
        } else {
          const float thr = s1 - 2.0f * E;
          if (disc >= thr) {
            redo = true;
            active = false;
          } else {
            df best = df_make(0.0f), best_ax = df_make(0.0f);
            int bc = -1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (ti[q] >= 0 && tv[q] >= thr) {
                const int c = ti[q], m = c / R, r = c - m * R;
                const df ax = score_x(a.d + (size_t)m * HJ * 2, xp, J, H, r, tw);
                df s = ax;
#pragma unroll
                for (int i = 0; i < KK; ++i)
                  if (i < t)
                    s = df_sub(s, df_mul(df{S.ahi[i], S.alo[i]},
                                         gram_entry(a.xgram, M, H, R, m, r, S.m[i], S.r[i], tw)));
                if (bc < 0 || df_abs_gt(s, best) || (df_abs_eq(s, best) && c < bc)) {
                  best = s;
                  bc = c;
                  best_ax = ax;
                }
              }
            }
            if (bc < 0 || !(fabsf(best.hi) > stop_level)) {
              active = false;
            } else {
              const int mb = bc / R, rb = bc - mb * R;
              double gr[KK];
#pragma unroll
              for (int i = 0; i < KK; ++i)
                gr[i] = (i < t) ? df_to_d(gram_entry(a.xgram, M, H, R, mb, rb, S.m[i], S.r[i], tw))
                                : 0.0;
              const double diag = df_to_d(gram_entry(a.xgram, M, H, R, mb, rb, mb, rb, tw));
              const double rhs = df_to_d(best_ax);
              if (!CholAt<KK, 0>::run(t, S, gr, diag, rhs)) {
                active = false;
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
                rnorm = sqrtf(write_residual<KK>(myA, row, xp, a.d, HJ, a.n, t, S, s_qtab, tw));
                dr = 2.0f * (t + 6) * kU32 * (xnorm + 1.5f * asum);
              }
            }
          }
        }
        if (redo) {
          const int slot = atomicAdd(a.redo_count, 1);
          a.redo_list[slot] = (int)p;
          if (a.fallbacks) atomicAdd(a.fallbacks, 1ull);
        }
      }
    }

    // ---- outputs of this thread's patch
    if (valid && !redo && !aborted) {
#pragma unroll
      for (int i = 0; i < KK; ++i) {
        if (i < K) {
          const int64_t o = p * K + i;
          if (i < t) {
            a.atom[o] = S.m[i];
            a.angle_idx[o] = S.r[i];
            if (a.angle) a.angle[o] = (float)(6.283185307179586 * S.r[i] / R);
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
  }

  // ---- drain: every issued TMA load and MMA completes before TMEM is freed
  if (tid == 0) {
    for (uint32_t gg = mma_waited; gg < mma_issued; ++gg)
      tc::mbar_wait_bounded(done_bar0 + 8 * (gg & 1), (gg >> 1) & 1, kWaitNs);
    for (uint32_t gg = mma_issued; gg < tma_next; ++gg)
      tc::mbar_wait_bounded(full_bar0 + 8 * (gg % kStages), (gg / kStages) & 1, kWaitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

template <int TILES, int KK>
int launch_tc_t(const TcArgs &a, const CUtensorMap &tmap, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  int max_optin = 0, nsm = 0;
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const TcLayout L = tc_layout<TILES>(a.H, a.R);
  if (L.total > max_optin) return RSC_ERR_UNSUPPORTED;
  auto kern = romp_tc_kernel<TILES, KK>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  const int64_t groups = (a.P + (int64_t)TILES * kTile - 1) / ((int64_t)TILES * kTile);
  const int64_t grid = groups < nsm ? groups : nsm;
  kern<<<(unsigned)grid, TILES * kTile, L.total, stream>>>(tmap, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return RSC_OK;
}

}  // namespace

int rsc_launch_tc(const TcArgs &a, const CUtensorMap &tmap, cudaStream_t stream) {
  if (a.P == 0) return RSC_OK;
  if (a.K <= 3) return launch_tc_t<2, 3>(a, tmap, stream);
  if (a.K <= 5) return launch_tc_t<2, 5>(a, tmap, stream);
  if (a.K <= 8) return launch_tc_t<2, 8>(a, tmap, stream);
  return RSC_ERR_UNSUPPORTED;
}
